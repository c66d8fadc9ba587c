// rbd_project.cu -- the out-of-sample map of Section 3.1, v_C = Y' v (Section 3.3 "Online":
// cost m d per vector), for a block of k vectors: C = Y' V.
//
// Each CTA owns a 32 x 32 tile of C and a range of rows, walked in 32-row chunks staged in shared
// memory and split into float-float form on load; each thread accumulates 4 outputs over its rows
// in order.  Tall Y are split into row ranges (enough CTAs to fill the GPU) whose partial tiles a
// second kernel adds in range order: deterministic, FP64-grade accuracy on the FP32 pipes.
#include <algorithm>

#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

struct ProjParams {
    const double* Y;
    int64_t m, d, ldy;
    const void* V;
    int vt;
    int64_t k, ldv;
    double* C;
    int64_t ldc;
};

__device__ __forceinline__ double load_v(const void* V, int vt, int64_t idx) {
    if (vt == 0) return ((const double*)V)[idx];
    if (vt == 1) return (double)((const float*)V)[idx];
    return (double)__bfloat162float(((const __nv_bfloat16*)V)[idx]);
}

constexpr int kPT = 32;  // tile edge

// grid (ceil(d/32), ceil(k/32), nsplit), 256 threads; thread (ty = tid / 8, tx = tid % 8) computes
// C(l0 + ty, c0 + tx + 8 q), q = 0..3, over rows [z * rows_per, (z + 1) * rows_per).  With one
// split it writes C; with several it writes its partial tile to part[z] (FP64, d x k, ld d).
__global__ void __launch_bounds__(256) project_kernel(ProjParams p, int64_t rows_per, double* part) {
    __shared__ float yh[kPT][kPT + 1], yl[kPT][kPT + 1];   // [row][basis]
    __shared__ float vh[kPT][kPT + 1], vl[kPT][kPT + 1];   // [row][vector]
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;
    const int64_t l0 = (int64_t)blockIdx.x * kPT, c0 = (int64_t)blockIdx.y * kPT;
    const int64_t rbeg = (int64_t)blockIdx.z * rows_per, rend = min(p.m, rbeg + rows_per);
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t r0 = rbeg; r0 < rend; r0 += kPT) {
        // stage a 32-row chunk of Y(:, l0:l0+32) and V(:, c0:c0+32); element (row, col) is
        // loaded by thread (col * 32 + row) % 256 four times over.
        for (int idx = tid; idx < kPT * kPT; idx += 256) {
            const int row = idx % kPT, col = idx / kPT;
            const int64_t r = r0 + row;
            double y = 0.0, v = 0.0;
            if (r < rend) {
                if (l0 + col < p.d) y = p.Y[(l0 + col) * p.ldy + r];
                if (c0 + col < p.k) v = load_v(p.V, p.vt, (c0 + col) * p.ldv + r);
            }
            float a, b;
            split_f64_fast(y, a, b);  // integer splits (FP64 arithmetic is slow on this part)
            yh[row][col] = a;
            yl[row][col] = b;
            split_f64_fast(v, a, b);
            vh[row][col] = a;
            vl[row][col] = b;
        }
        __syncthreads();
#pragma unroll 4
        for (int row = 0; row < kPT; ++row) {
            const float ah = yh[row][ty], al = yl[row][ty];
#pragma unroll
            for (int q = 0; q < 4; ++q) ff_mac2(s[q], c[q], ah, al, vh[row][tx + 8 * q], vl[row][tx + 8 * q]);
        }
        __syncthreads();
    }
    const int64_t l = l0 + ty;
    if (l < p.d) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t col = c0 + tx + 8 * q;
            if (col >= p.k) continue;
            if (part)
                part[((int64_t)blockIdx.z * p.k + col) * p.d + l] = ff_to_double(s[q], c[q]);
            else
                p.C[col * p.ldc + l] = ff_to_double(s[q], c[q]);
        }
    }
}

// C = sum of the row splits' partial products, in split order.
__global__ void __launch_bounds__(256) project_reduce_kernel(ProjParams p, int nsplit, const double* part) {
    const int64_t total = p.d * p.k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i % p.d, col = i / p.d;
        double acc = 0.0;
        for (int z = 0; z < nsplit; ++z) acc += part[((int64_t)z * p.k + col) * p.d + l];
        p.C[col * p.ldc + l] = acc;
    }
}

cudaError_t launch_project(const double* Y, int64_t m, int64_t d, int64_t ldy, const void* V, int vt,
                           int64_t k, int64_t ldv, double* C, int64_t ldc, cudaStream_t st) {
    ProjParams p{Y, m, d, ldy, V, vt, k, ldv, C, ldc};
    const int64_t tiles = ceil_div(d, (int64_t)kPT) * ceil_div(k, (int64_t)kPT);
    // split the rows so that the grid covers the GPU twice over, each split at least 256 rows
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(ceil_div(2 * 152, tiles), m / 256));
    nsplit = std::min<int64_t>(nsplit, 64);
    const int64_t rows_per = round_up(ceil_div(m, nsplit), (int64_t)kPT);
    nsplit = ceil_div(m, rows_per);
    double* part = nullptr;
    if (nsplit > 1) {
        cudaError_t e = lib_malloc_async((void**)&part, (size_t)nsplit * d * k * 8, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            part = nullptr;
            nsplit = 1;
        }
    }
    const int64_t rp = (nsplit > 1) ? rows_per : m;
    dim3 grid((unsigned)ceil_div(d, (int64_t)kPT), (unsigned)ceil_div(k, (int64_t)kPT), (unsigned)nsplit);
    project_kernel<<<grid, 256, 0, st>>>(p, rp, part);
    cudaError_t e = cudaGetLastError();
    if (part) {
        if (e == cudaSuccess) {
            const int64_t total = d * k;
            const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, (int64_t)256), 4096));
            project_reduce_kernel<<<blocks, 256, 0, st>>>(p, (int)nsplit, part);
            e = cudaGetLastError();
        }
        cudaError_t fe = cudaFreeAsync(part, st);
        if (e == cudaSuccess) e = fe;
    }
    return e;
}

}  // namespace rbd

namespace rbd {

// ---------------------------------------------------------------------------------------------
// Uncompress (Section 3.1): Xr = Y T, column j of the approximation = Y T(:, j) (Section 3.3:
// m d per column).  Each CTA owns a 64 x 64 tile of Xr and walks the d bases in chunks of 32,
// staged in shared memory as float-float; thread (tx = tid % 16, ty = tid / 16) accumulates the
// 4 x 4 outputs of rows 4 tx .. 4 tx + 3 and columns 4 ty .. 4 ty + 3 over the bases in order:
// deterministic, FP64-grade on the FP32 pipes.  Per basis a thread reads its 4 rows of Y as two
// 16-byte loads and its 4 columns of T as 8 broadcast words, for 16 float-float products.
// ---------------------------------------------------------------------------------------------
struct ReconParams {
    const double* Y;
    int64_t m, d, ldy;
    const double* T;
    int64_t n, ldt;
    double* Xr;
    int64_t ldxr;
};

constexpr int kRT = 64;  // tile edge (rows and columns of Xr)
constexpr int kRL = 32;  // bases per staged chunk

__global__ void __launch_bounds__(256) reconstruct_kernel(ReconParams p) {
    __shared__ __align__(16) float yh[kRL][kRT];  // [basis][row]
    __shared__ __align__(16) float yl[kRL][kRT];
    __shared__ float th[kRT][kRL + 1], tl[kRT][kRL + 1];         // [col][basis]
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t r0 = (int64_t)blockIdx.x * kRT;
    // column tiles blockIdx.y, blockIdx.y + gridDim.y, ... (the grid's y extent is capped)
    for (int64_t j0 = (int64_t)blockIdx.y * kRT; j0 < p.n; j0 += (int64_t)gridDim.y * kRT) {
        float s[4][4], c[4][4];  // [column][row]
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u) s[q][u] = c[q][u] = 0.f;
        for (int64_t l0 = 0; l0 < p.d; l0 += kRL) {
            for (int idx = tid; idx < kRT * kRL; idx += 256) {
                // Y(r0 + a, l0 + b): rows fastest; T(l0 + a2, j0 + b2): bases fastest (both coalesced)
                const int a = idx % kRT, b = idx / kRT;
                const int a2 = idx % kRL, b2 = idx / kRL;
                double y = 0.0, t = 0.0;
                if (r0 + a < p.m && l0 + b < p.d) y = p.Y[(l0 + b) * p.ldy + r0 + a];
                if (l0 + a2 < p.d && j0 + b2 < p.n) t = p.T[(j0 + b2) * p.ldt + l0 + a2];
                // integer splits: FP64 arithmetic here would cost as much as the products below
                float hi, lo;
                split_f64_fast(y, hi, lo);
                yh[b][a] = hi;
                yl[b][a] = lo;
                split_f64_fast(t, hi, lo);
                th[b2][a2] = hi;
                tl[b2][a2] = lo;
            }
            __syncthreads();
            const int lc = (int)min((int64_t)kRL, p.d - l0);
            for (int l = 0; l < lc; ++l) {
                const float4 ah = *reinterpret_cast<const float4*>(&yh[l][4 * tx]);
                const float4 al = *reinterpret_cast<const float4*>(&yl[l][4 * tx]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float bh = th[4 * ty + q][l], bl = tl[4 * ty + q][l];
                    ff_mac2(s[q][0], c[q][0], ah.x, al.x, bh, bl);
                    ff_mac2(s[q][1], c[q][1], ah.y, al.y, bh, bl);
                    ff_mac2(s[q][2], c[q][2], ah.z, al.z, bh, bl);
                    ff_mac2(s[q][3], c[q][3], ah.w, al.w, bh, bl);
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t j = j0 + 4 * ty + q;
            if (j >= p.n) continue;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t r = r0 + 4 * tx + u;
                if (r < p.m) p.Xr[j * p.ldxr + r] = ff_to_double(s[q][u], c[q][u]);
            }
        }
    }
}

cudaError_t launch_reconstruct(const double* Y, int64_t m, int64_t d, int64_t ldy, const double* T, int64_t n,
                               int64_t ldt, double* Xr, int64_t ldxr, cudaStream_t st) {
    ReconParams p{Y, m, d, ldy, T, n, ldt, Xr, ldxr};
    dim3 grid((unsigned)ceil_div(m, (int64_t)kRT), (unsigned)std::min<int64_t>(ceil_div(n, (int64_t)kRT), 65535));
    reconstruct_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace rbd
