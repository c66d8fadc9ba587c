// rbd_grad.cu -- rbd_grad: the adjoint of the differentiation form.
//
// For the FIXED pivot set P of a compression (A = X(:, P) = Y R, Y = Q of the Gram-Schmidt
// factorisation in pivot order, R = T(:, P) upper triangular, T = Y' X) and fixed out-of-sample
// data Xo:
//     L(X) = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2.
// With P_A = A A^+ the projector onto span A, L = w_rec tr(X'(I - P_A) X) + w_proj tr(Xo' P_A Xo),
// and dP_A = (I - P_A) dA A^+ + (A^+)' dA' (I - P_A), A^+ = R^-1 Y', the gradient is
//     G = 2 w_rec E                                             E = X - Y T
//     G(:, P) += [-2 w_rec E T' + 2 w_proj (Xo - Y C) C'] R^-T, C = Y' Xo.
// Kernels (one stream, in order; rbd_grad_batched launches each once for a whole batch, the CTA's
// blockIdx.y picking the instance, and C = Y' Xo once per instance):
//   grad_pass_kernel   one pass over X by 32-row blocks: E = X - Y T (float-float), G = 2 w_rec E,
//                      M1 = E T' (m x d, float-float, from E held in shared memory), ||E||^2
//   project_kernel     C = Y' Xo (rbd_project's kernel)
//   grad_small_kernel  CC = C C', ||C||^2 (one CTA)
//   grad_pivot_kernel  Z = -2 w_rec M1 + 2 w_proj (Xo C' - Y CC), W = Z R^-T (back substitution
//                      per row, FP64), G(:, P(l)) += W(:, l)
//   grad_loss_kernel   loss = w_rec ||E||^2 + w_proj ||C||^2 (fixed order)
// The contractions have inner dimensions n, k and d of a few hundred at most and need FP64-grade
// results, so they run as float-float on the FP32 pipes (FP64 is 1/64 rate on GB300; BF16 tensor
// products would lose the accuracy).
#include <algorithm>
#include <vector>

#include "../../include/rbd.h"
#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

namespace {

constexpr int kGR = 32;        // rows per CTA
constexpr int kGCT = 32;       // columns per tile of the pass
constexpr int kGThreads = 256;
constexpr int kGradMaxD = 256;

struct GradParams {
    const void* X;
    int xt;
    int64_t m, n, ldx;
    const double* Y;
    int64_t ldy;
    const double* T;
    int64_t ldt;
    const int64_t* piv;
    int64_t d;
    const void* Xo;
    int64_t k, ldxo;
    double w_rec, w_proj;
    double* G;
    int64_t ldg;
    double* M1;     // m x d (ld m)
    double* C;      // d x k (ld d)
    double* CC;     // d x d
    double* epart;  // per row block ||E||^2
    double* c2;     // ||C||^2
    double* loss;
};

__device__ __forceinline__ double load_elem(const void* A, int t, int64_t idx) { return load_x_elem(A, t, idx); }

// Shared memory of grad_pass_kernel (all arrays row-index fastest, so that the 32 lanes of a warp,
// which hold 32 consecutive rows, touch 32 banks): Ys [2][d][kGR], Ts [2][d][kGCT + 1] (padded),
// Es [2][kGCT][kGR], Ms [2][d][kGR], then kGThreads doubles for the reduction.
constexpr int kTP = kGCT + 1;
size_t grad_pass_smem(int64_t d) {
    return (size_t)(2 * kGR * d + 2 * d * kTP + 2 * kGR * kGCT + 2 * kGR * d) * 4 + (size_t)kGThreads * 8;
}

template <bool WITH_G>
__device__ __forceinline__ void grad_pass_body(const GradParams& p) {
    extern __shared__ __align__(16) float gsm[];
    const int d = (int)p.d;
    float* Ysh = gsm;                       // [d][kGR]
    float* Ysl = Ysh + kGR * d;
    float* Tsh = Ysl + kGR * d;             // [d][kTP]
    float* Tsl = Tsh + d * kTP;
    float* Esh = Tsl + d * kTP;             // [kGCT][kGR]
    float* Esl = Esh + kGR * kGCT;
    float* Msh = Esl + kGR * kGCT;          // [d][kGR]
    float* Msl = Msh + kGR * d;
    double* red = reinterpret_cast<double*>(Msl + kGR * d);

    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kGR;
    const int rr = tid % kGR, cq = tid / kGR;  // row of the block, column slot (0..7) = warp
    const int nrows = (int)min((int64_t)kGR, p.m - r0);

    for (int i = tid; i < kGR * d; i += kGThreads) {
        const int r = i % kGR, l = i / kGR;
        float hi = 0.f, lo = 0.f;
        if (r < nrows) split_double(p.Y[(r0 + r) + l * p.ldy], hi, lo);
        Ysh[l * kGR + r] = hi;
        Ysl[l * kGR + r] = lo;
        Msh[l * kGR + r] = 0.f;
        Msl[l * kGR + r] = 0.f;
    }
    double e2 = 0.0;
    for (int64_t j0 = 0; j0 < p.n; j0 += kGCT) {
        const int ncols = (int)min((int64_t)kGCT, p.n - j0);
        __syncthreads();  // the previous tile is consumed
        for (int i = tid; i < d * kGCT; i += kGThreads) {
            const int l = i % d, jj = i / d;
            float hi = 0.f, lo = 0.f;
            if (jj < ncols) split_double(p.T[(j0 + jj) * p.ldt + l], hi, lo);
            Tsh[l * kTP + jj] = hi;
            Tsl[l * kTP + jj] = lo;
        }
        __syncthreads();
        // E = X - Y T for the kGR x kGCT entries of the tile: 4 per thread
#pragma unroll
        for (int q = 0; q < kGCT / 8; ++q) {
            const int jj = cq + 8 * q;
            float s = 0.f, c = 0.f;
            if (jj < ncols && rr < nrows) {
                split_double(load_elem(p.X, p.xt, (j0 + jj) * p.ldx + r0 + rr), s, c);
                for (int l = 0; l < d; ++l)
                    ff_mac2(s, c, -Ysh[l * kGR + rr], -Ysl[l * kGR + rr], Tsh[l * kTP + jj], Tsl[l * kTP + jj]);
            }
            const double e = ff_to_double(s, c);
            float eh, el;
            split_double(e, eh, el);
            Esh[jj * kGR + rr] = eh;
            Esl[jj * kGR + rr] = el;
            e2 += e * e;
            if (WITH_G && jj < ncols && rr < nrows) p.G[(j0 + jj) * p.ldg + r0 + rr] = 2.0 * p.w_rec * e;
        }
        if (WITH_G) {
            __syncthreads();
            // M1 += E T' for this tile: outputs (rr, l), l = cq + 8 q
            for (int l = cq; l < d; l += 8) {
                float s = Msh[l * kGR + rr], c = Msl[l * kGR + rr];
                for (int jj = 0; jj < ncols; ++jj)
                    ff_mac2(s, c, Esh[jj * kGR + rr], Esl[jj * kGR + rr], Tsh[l * kTP + jj], Tsl[l * kTP + jj]);
                Msh[l * kGR + rr] = s;
                Msl[l * kGR + rr] = c;
            }
        }
    }
    if (WITH_G) {
        for (int l = cq; l < d; l += 8)
            if (rr < nrows) p.M1[(r0 + rr) + l * p.m] = ff_to_double(Msh[l * kGR + rr], Msl[l * kGR + rr]);
    }
    // ||E||^2 of this row block, fixed-order tree
    red[tid] = e2;
    __syncthreads();
    for (int o = kGThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) p.epart[blockIdx.x] = red[0];
}

template <bool WITH_G>
__global__ void __launch_bounds__(kGThreads) grad_pass_kernel(GradParams p) {
    grad_pass_body<WITH_G>(p);
}

// Batched: instance blockIdx.y; the grid is as wide as the tallest instance needs.
template <bool WITH_G>
__global__ void __launch_bounds__(kGThreads) grad_pass_batched(const GradParams* ps) {
    const GradParams& p = ps[blockIdx.y];
    if ((int64_t)blockIdx.x * kGR >= p.m) return;
    grad_pass_body<WITH_G>(p);
}

// CC = C C' (d x d) and ||C||^2, one CTA, float-float over k.
__device__ __forceinline__ void grad_small_body(const GradParams& p) {
    __shared__ double red[kGThreads];
    const int tid = threadIdx.x;
    const int64_t d = p.d, k = p.k;
    for (int64_t o = tid; o < d * d; o += kGThreads) {
        const int64_t a = o % d, b = o / d;
        float s = 0.f, c = 0.f;
        for (int64_t q = 0; q < k; ++q) {
            float ah, al, bh, bl;
            split_double(p.C[a + q * d], ah, al);
            split_double(p.C[b + q * d], bh, bl);
            ff_mac2(s, c, ah, al, bh, bl);
        }
        p.CC[a + b * d] = ff_to_double(s, c);
    }
    double acc = 0.0;
    for (int64_t o = tid; o < d * k; o += kGThreads) acc += p.C[o] * p.C[o];
    red[tid] = acc;
    __syncthreads();
    for (int o = kGThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) *p.c2 = red[0];
}

__global__ void __launch_bounds__(kGThreads) grad_small_kernel(GradParams p) { grad_small_body(p); }

// Batched: one CTA per instance; instances without both Y and Xo get CC = 0.
__global__ void __launch_bounds__(kGThreads) grad_small_batched(const GradParams* ps) {
    const GradParams& p = ps[blockIdx.y];
    if (p.d > 0 && p.k > 0) {
        grad_small_body(p);
    } else {
        for (int64_t o = threadIdx.x; o < p.d * p.d; o += kGThreads) p.CC[o] = 0.0;
    }
}

// Pivot columns: Z = -2 w_rec M1 + 2 w_proj (Xo C' - Y CC), W = Z R^-T, G(:, P(l)) += W(:, l).
// Shared memory: Z [d][kGR] doubles, Xo tile [kGCT][kGR] and C tile [d][kGCT] (split floats).
size_t grad_pivot_smem(int64_t d) {
    return (size_t)kGR * d * 8 + (size_t)2 * kGR * kGCT * 4 + (size_t)2 * d * kGCT * 4;
}

__device__ __forceinline__ void grad_pivot_body(const GradParams& p) {
    extern __shared__ __align__(16) unsigned char psm[];
    const int d = (int)p.d;
    double* Z = reinterpret_cast<double*>(psm);         // [d][kGR]
    float* Xoh = reinterpret_cast<float*>(Z + kGR * d);  // [kGCT][kGR]
    float* Xol = Xoh + kGR * kGCT;
    float* Ch = Xol + kGR * kGCT;                        // [d][kGCT]
    float* Cl = Ch + d * kGCT;
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * kGR;
    const int rr = tid % kGR, cq = tid / kGR;
    const int nrows = (int)min((int64_t)kGR, p.m - r0);

    // Z over chunks of 32 coefficients: outputs (rr, l), l = l0 + cq + 8 q, q < 4
    for (int l0 = 0; l0 < d; l0 += 32) {
        float as[4], ac[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) as[q] = ac[q] = 0.f;
        for (int64_t q0 = 0; q0 < p.k; q0 += kGCT) {
            const int nq = (int)min((int64_t)kGCT, p.k - q0);
            __syncthreads();
            for (int i = tid; i < kGR * kGCT; i += kGThreads) {
                const int r = i % kGR, qq = i / kGR;
                float hi = 0.f, lo = 0.f;
                if (r < nrows && qq < nq) split_double(load_elem(p.Xo, p.xt, (q0 + qq) * p.ldxo + r0 + r), hi, lo);
                Xoh[qq * kGR + r] = hi;
                Xol[qq * kGR + r] = lo;
            }
            for (int i = tid; i < d * kGCT; i += kGThreads) {
                const int l = i % d, qq = i / d;
                float hi = 0.f, lo = 0.f;
                if (qq < nq) split_double(p.C[l + (q0 + qq) * p.d], hi, lo);
                Ch[l * kGCT + qq] = hi;
                Cl[l * kGCT + qq] = lo;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int l = l0 + cq + 8 * q;
                if (l < d)
                    for (int qq = 0; qq < nq; ++qq)
                        ff_mac2(as[q], ac[q], Xoh[qq * kGR + rr], Xol[qq * kGR + rr], Ch[l * kGCT + qq],
                                Cl[l * kGCT + qq]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = l0 + cq + 8 * q;
            if (l < d) {
                double z = 0.0;
                if (rr < nrows) {
                    float s = as[q], c = ac[q];
                    for (int l2 = 0; l2 < d; ++l2) {
                        float yh, yl, ch, cl;
                        split_double(p.Y[(r0 + rr) + l2 * p.ldy], yh, yl);
                        split_double(p.CC[l2 + l * p.d], ch, cl);
                        ff_mac2(s, c, -yh, -yl, ch, cl);
                    }
                    z = -2.0 * p.w_rec * p.M1[(r0 + rr) + l * p.m] + 2.0 * p.w_proj * ff_to_double(s, c);
                }
                Z[l * kGR + rr] = z;
            }
        }
    }
    __syncthreads();
    // W = Z R^-T: per row, W R' = Z with R(a, b) = T(a, P(b)), a <= b; back substitution in FP64
    if (tid < nrows) {
        for (int a = d - 1; a >= 0; --a) {
            double v = Z[a * kGR + tid];
            for (int b = a + 1; b < d; ++b) v -= Z[b * kGR + tid] * __ldg(&p.T[__ldg(&p.piv[b]) * p.ldt + a]);
            Z[a * kGR + tid] = v / __ldg(&p.T[__ldg(&p.piv[a]) * p.ldt + a]);
        }
    }
    __syncthreads();
    for (int i = tid; i < kGR * d; i += kGThreads) {
        const int r = i % kGR, l = i / kGR;
        if (r < nrows) p.G[p.piv[l] * p.ldg + r0 + r] += Z[l * kGR + r];
    }
}

__global__ void __launch_bounds__(kGThreads) grad_pivot_kernel(GradParams p) { grad_pivot_body(p); }

__global__ void __launch_bounds__(kGThreads) grad_pivot_batched(const GradParams* ps) {
    const GradParams& p = ps[blockIdx.y];
    if ((int64_t)blockIdx.x * kGR >= p.m || p.d == 0 || !p.G) return;
    grad_pivot_body(p);
}

__device__ __forceinline__ void grad_loss_body(const GradParams& p, int64_t nblocks) {
    double e2 = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) e2 += p.epart[b];
    *p.loss = p.w_rec * e2 + p.w_proj * (p.k > 0 && p.d > 0 ? *p.c2 : 0.0);
}

__global__ void grad_loss_kernel(GradParams p, int nblocks) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    grad_loss_body(p, nblocks);
}

// Batched: thread i sums instance i's row-block partials (the same order as grad_loss_kernel).
__global__ void grad_loss_batched(const GradParams* ps, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) grad_loss_body(ps[i], ceil_div(ps[i].m, (int64_t)kGR));
}

rbd_status map_cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RBD_OK;
    if (e == cudaErrorMemoryAllocation) return RBD_ENOMEM;
    return RBD_ECUDA;
}

}  // namespace
}  // namespace rbd

using namespace rbd;

extern "C" rbd_status rbd_grad(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, const double* Y,
                               int64_t ldy, const double* T, int64_t ldt, const int64_t* pivots, int64_t d,
                               const void* Xo, int64_t k, int64_t ldxo, double w_rec, double w_proj, double* G,
                               int64_t ldg, double* loss, void* stream) {
    if (!X || !loss || m < 1 || n < 1 || ldx < m || d < 0 || d > m || d > n || k < 0) return RBD_EINVAL;
    if (xt != RBD_F64 && xt != RBD_F32 && xt != RBD_BF16) return RBD_EINVAL;
    if (d > 0 && (!Y || !T || !pivots || ldy < m || ldt < d)) return RBD_EINVAL;
    if (k > 0 && (!Xo || ldxo < m)) return RBD_EINVAL;
    if (G && ldg < m) return RBD_EINVAL;
    if (!(w_rec == w_rec) || !(w_proj == w_proj)) return RBD_EINVAL;
    if (d > kGradMaxD) return RBD_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nb = ceil_div(m, (int64_t)kGR);
    if (nb > (int64_t)1 << 31) return RBD_EUNSUPPORTED;
    const int64_t dd = std::max<int64_t>(d, 1), kk = std::max<int64_t>(k, 1);
    // workspace: M1 (m x d), C (d x k), CC (d x d), epart (nb), c2
    const size_t b_m1 = (size_t)m * dd * 8, b_c = (size_t)dd * kk * 8, b_cc = (size_t)dd * dd * 8;
    const size_t b_ep = (size_t)nb * 8;
    const size_t total = b_m1 + b_c + b_cc + b_ep + 64;
    void* ws = nullptr;
    cudaError_t ce = lib_malloc_async(&ws, total, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return RBD_ENOMEM;
    }
    unsigned char* w = (unsigned char*)ws;
    GradParams p;
    p.X = X;
    p.xt = (int)xt;
    p.m = m;
    p.n = n;
    p.ldx = ldx;
    p.Y = Y;
    p.ldy = ldy;
    p.T = T;
    p.ldt = ldt;
    p.piv = pivots;
    p.d = d;
    p.Xo = Xo;
    p.k = k;
    p.ldxo = ldxo;
    p.w_rec = w_rec;
    p.w_proj = w_proj;
    p.G = G;
    p.ldg = ldg;
    p.M1 = (double*)w;
    p.C = (double*)(w + b_m1);
    p.CC = (double*)(w + b_m1 + b_c);
    p.epart = (double*)(w + b_m1 + b_c + b_cc);
    p.c2 = (double*)(w + b_m1 + b_c + b_cc + b_ep);
    p.loss = loss;

    const size_t sm_pass = grad_pass_smem(d);
    const size_t sm_piv = grad_pivot_smem(d);
    if (G) {
        ce = cudaFuncSetAttribute(grad_pass_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pass);
        if (ce == cudaSuccess)
            ce = cudaFuncSetAttribute(grad_pivot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_piv);
        if (ce == cudaSuccess) {
            grad_pass_kernel<true><<<(unsigned)nb, kGThreads, sm_pass, st>>>(p);
            ce = cudaGetLastError();
        }
    } else {
        ce = cudaFuncSetAttribute(grad_pass_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pass);
        if (ce == cudaSuccess) {
            grad_pass_kernel<false><<<(unsigned)nb, kGThreads, sm_pass, st>>>(p);
            ce = cudaGetLastError();
        }
    }
    if (ce == cudaSuccess && d > 0 && k > 0) {
        ce = launch_project(Y, m, d, ldy, Xo, (int)xt, k, ldxo, p.C, d, st);
        if (ce == cudaSuccess) {
            grad_small_kernel<<<1, kGThreads, 0, st>>>(p);
            ce = cudaGetLastError();
        }
    } else if (ce == cudaSuccess && d > 0) {
        ce = cudaMemsetAsync(p.CC, 0, b_cc, st);
    }
    if (ce == cudaSuccess && G && d > 0) {
        grad_pivot_kernel<<<(unsigned)nb, kGThreads, sm_piv, st>>>(p);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        grad_loss_kernel<<<1, 32, 0, st>>>(p, (int)nb);
        ce = cudaGetLastError();
    }
    cudaError_t fe = cudaFreeAsync(ws, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) cudaGetLastError();
    return map_cuda_status(ce);
}

extern "C" rbd_status rbd_grad_batched(const rbd_grad_item* items, int64_t count, rbd_dtype xt, double w_rec,
                                       double w_proj, void* stream) {
    if (!items || count < 1 || count > 65535) return RBD_EINVAL;
    if (xt != RBD_F64 && xt != RBD_F32 && xt != RBD_BF16) return RBD_EINVAL;
    if (!(w_rec == w_rec) || !(w_proj == w_proj)) return RBD_EINVAL;
    const bool with_g = items[0].G != nullptr;
    int64_t max_nb = 1, max_d = 1;
    size_t total = ((size_t)count * sizeof(GradParams) + 255) & ~(size_t)255;
    std::vector<size_t> off((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const rbd_grad_item& it = items[i];
        if (!it.X || !it.loss || it.m < 1 || it.n < 1 || it.ldx < it.m || it.d < 0 || it.d > it.m || it.d > it.n ||
            it.k < 0)
            return RBD_EINVAL;
        if (it.d > 0 && (!it.Y || !it.T || !it.pivots || it.ldy < it.m || it.ldt < it.d)) return RBD_EINVAL;
        if (it.k > 0 && (!it.Xo || it.ldxo < it.m)) return RBD_EINVAL;
        if ((it.G != nullptr) != with_g || (it.G && it.ldg < it.m)) return RBD_EINVAL;
        if (it.d > kGradMaxD) return RBD_EUNSUPPORTED;
        const int64_t nb = ceil_div(it.m, (int64_t)kGR);
        if (nb > (int64_t)1 << 31) return RBD_EUNSUPPORTED;
        max_nb = std::max(max_nb, nb);
        max_d = std::max(max_d, it.d);
        const int64_t dd = std::max<int64_t>(it.d, 1), kk = std::max<int64_t>(it.k, 1);
        off[(size_t)i] = total;
        total += ((size_t)it.m * dd * 8 + (size_t)dd * kk * 8 + (size_t)dd * dd * 8 + (size_t)nb * 8 + 64 + 255) &
                 ~(size_t)255;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = nullptr;
    cudaError_t ce = lib_malloc_async(&ws, total, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return RBD_ENOMEM;
    }
    unsigned char* w = (unsigned char*)ws;
    std::vector<GradParams> hp((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const rbd_grad_item& it = items[i];
        GradParams& p = hp[(size_t)i];
        const int64_t dd = std::max<int64_t>(it.d, 1), kk = std::max<int64_t>(it.k, 1);
        const int64_t nb = ceil_div(it.m, (int64_t)kGR);
        unsigned char* b = w + off[(size_t)i];
        p.X = it.X;
        p.xt = (int)xt;
        p.m = it.m;
        p.n = it.n;
        p.ldx = it.ldx;
        p.Y = it.Y;
        p.ldy = it.ldy;
        p.T = it.T;
        p.ldt = it.ldt;
        p.piv = it.pivots;
        p.d = it.d;
        p.Xo = it.Xo;
        p.k = it.k;
        p.ldxo = it.ldxo;
        p.w_rec = w_rec;
        p.w_proj = w_proj;
        p.G = it.G;
        p.ldg = it.ldg;
        p.M1 = (double*)b;
        p.C = (double*)(b + (size_t)it.m * dd * 8);
        p.CC = (double*)(b + (size_t)it.m * dd * 8 + (size_t)dd * kk * 8);
        p.epart = (double*)(b + (size_t)it.m * dd * 8 + (size_t)dd * kk * 8 + (size_t)dd * dd * 8);
        p.c2 = (double*)(b + (size_t)it.m * dd * 8 + (size_t)dd * kk * 8 + (size_t)dd * dd * 8 + (size_t)nb * 8);
        p.loss = it.loss;
    }
    const GradParams* dp = (const GradParams*)w;
    // a pageable source: the call returns once the table is staged, so hp may go out of scope
    ce = cudaMemcpyAsync(w, hp.data(), (size_t)count * sizeof(GradParams), cudaMemcpyHostToDevice, st);
    const size_t sm_pass = grad_pass_smem(max_d), sm_piv = grad_pivot_smem(max_d);
    const dim3 grid_rows((unsigned)max_nb, (unsigned)count);
    if (ce == cudaSuccess) {
        if (with_g) {
            ce = cudaFuncSetAttribute(grad_pass_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pass);
            if (ce == cudaSuccess)
                ce = cudaFuncSetAttribute(grad_pivot_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_piv);
            if (ce == cudaSuccess) {
                grad_pass_batched<true><<<grid_rows, kGThreads, sm_pass, st>>>(dp);
                ce = cudaGetLastError();
            }
        } else {
            ce = cudaFuncSetAttribute(grad_pass_batched<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pass);
            if (ce == cudaSuccess) {
                grad_pass_batched<false><<<grid_rows, kGThreads, sm_pass, st>>>(dp);
                ce = cudaGetLastError();
            }
        }
    }
    for (int64_t i = 0; i < count && ce == cudaSuccess; ++i) {
        const rbd_grad_item& it = items[i];
        if (it.d > 0 && it.k > 0)
            ce = launch_project(it.Y, it.m, it.d, it.ldy, it.Xo, (int)xt, it.k, it.ldxo, hp[(size_t)i].C, it.d, st);
    }
    if (ce == cudaSuccess) {
        grad_small_batched<<<dim3(1, (unsigned)count), kGThreads, 0, st>>>(dp);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess && with_g) {
        grad_pivot_batched<<<grid_rows, kGThreads, sm_piv, st>>>(dp);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) {
        grad_loss_batched<<<(unsigned)ceil_div(count, 128), 128, 0, st>>>(dp, count);
        ce = cudaGetLastError();
    }
    cudaError_t fe = cudaFreeAsync(ws, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) cudaGetLastError();
    return map_cuda_status(ce);
}
