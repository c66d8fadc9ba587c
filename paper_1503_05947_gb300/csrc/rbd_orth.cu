// rbd_orth.cu -- step 2.1-2.2 of Algorithm 1: orthogonalise the pivot column v = X(:, i)
// against xi_0..xi_{k-1} twice (one re-orthogonalisation sweep) and measure ||v||.
//
// The paper applies modified Gram-Schmidt, a sequence of k dependent dot products.  On a GPU
// each dependent dot product needs a grid-wide reduction, so the two sweeps are organised as
// classical Gram-Schmidt applied twice ("twice is enough", Giraud, Langou and Rozloznik 2005),
// which is mathematically the same projection and agrees with two MGS sweeps to rounding:
//   A1 (row-parallel):    v1 = x_i - Y t        t = T(0:k, i) = Y' x_i, already computed by the
//                                                earlier fused passes (T(l, :) = xi_l' X)
//   A2 (column-parallel): h  = Y' v1             the re-orthogonalisation coefficients
//   C  (row-parallel):    v2 = v1 - Y h,  nu = ||v2||  (FP64), then the stop decisions:
//                         nu is also the exact residual of the column that maximised the
//                         indicator in the previous step, i.e. that step's E_cur (2.3), so
//                         step 2.4 of the previous step and the break test of step 2.2 are both
//                         taken here.  One extra A1/A2/C after the last basis certifies the last
//                         indicator.
// The normalisation xi_k = v2 / nu is folded into the fused pass (it scales the dot products
// by 1 / nu and writes Y(:, k)).
//
// The GEMVs run in float-float arithmetic on a split FP32 copy of Y (relative error ~2^-47,
// below FP64 rounding of length-m dot products for m >= 128); the vectors v1, v2 and nu are
// FP64.  Partial sums are combined in a fixed order by the last CTA to arrive at a counter,
// so results are bitwise reproducible and no CTA ever waits for another.
#include <algorithm>

#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

struct GemvNParams {
    int mode;                 // 0: A1, 1: C
    const void* X;            // A1: pivot column source (storage type xt)
    int xt;
    int64_t ldx;
    const double* T;          // A1: coefficients T(0:k, pivot)
    int64_t ldt;
    const double* h;          // C: coefficients h(0:k)
    const double* vin;        // C: v1
    const float* yh;
    const float* yl;
    double* vpart;            // LC x ldp partial sums
    uint32_t* rb_cnt;
    double* vout;             // v1 (A1) or v2 (C)
    float* vouth;
    float* voutl;
    double* nu2part;          // C: per row-block partial ||v2||^2
    int64_t* pivots;          // C: outputs of step k
    double* nu_out;
    double* err;              // C: err[k-1], the certified indicator of the previous step
    const double* xn2;
    uint32_t* progress;       // C: host-mapped {steps finished, stop} (may be null)
    int64_t m, ldp, k, LC, LCH, RB;
    int64_t MT;               // C: tile rows of the tile-interleaved split output (v2s)
    Ctl* ctl;
};

__device__ __forceinline__ double load_x(const void* X, int xt, int64_t idx) {
    if (xt == 0) return ((const double*)X)[idx];
    if (xt == 1) return (double)((const float*)X)[idx];
    return (double)__bfloat162float(((const __nv_bfloat16*)X)[idx]);
}

// grid (RB, LC), 256 threads: 32 row-quads (128 rows) x 8 coefficient sub-lanes.
__global__ void __launch_bounds__(256) orth_gemv_n_kernel(GemvNParams p) {
    Ctl* ctl = p.ctl;
    if (ctl->stop != 0 || ctl->status != 0) return;
    if (ctl->d != p.k) {
        if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) raise_status(ctl, ST_EINVAL);
        return;
    }
    const int64_t piv = ctl->pivot;
    const int tid = threadIdx.x;
    const int q = tid & 31, ls = tid >> 5;
    const int64_t rb = blockIdx.x, lc = blockIdx.y;
    const int64_t r = rb * kGemvRows + 4 * q;
    const int64_t lbeg = lc * p.LCH;
    const int64_t lend = min(p.k, lbeg + p.LCH);

    extern __shared__ __align__(16) unsigned char smem[];
    float* ch = (float*)smem;              // LCH
    float* cl = ch + p.LCH;                // LCH
    double* red = (double*)(smem + round_up(8 * p.LCH, 16));  // 8 x 128
    __shared__ int s_last;

    // coefficients of this chunk, split to float-float
    for (int64_t l = lbeg + tid; l < lend; l += 256) {
        const double cval = (p.mode == 0) ? p.T[piv * p.ldt + l] : p.h[l];
        float hi, lo;
        split_double(cval, hi, lo);
        ch[l - lbeg] = hi;
        cl[l - lbeg] = lo;
    }
    __syncthreads();

    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    // batches of kU coefficients: all loads of a batch are issued before its arithmetic
    constexpr int kU = 4;
    for (int64_t l0 = lbeg + ls; l0 < lend; l0 += 8 * kU) {
        float4 a[kU], b[kU];
        float th[kU], tl[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t l = l0 + 8 * u;
            if (l < lend) {
                a[u] = *(const float4*)(p.yh + l * p.ldp + r);
                b[u] = *(const float4*)(p.yl + l * p.ldp + r);
                th[u] = ch[l - lbeg];
                tl[u] = cl[l - lbeg];
            } else {
                a[u] = b[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                th[u] = tl[u] = 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            ff_mac2(s[0], c[0], a[u].x, b[u].x, th[u], tl[u]);
            ff_mac2(s[1], c[1], a[u].y, b[u].y, th[u], tl[u]);
            ff_mac2(s[2], c[2], a[u].z, b[u].z, th[u], tl[u]);
            ff_mac2(s[3], c[3], a[u].w, b[u].w, th[u], tl[u]);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) red[ls * kGemvRows + 4 * q + e] = ff_to_double(s[e], c[e]);
    __syncthreads();
    if (tid < kGemvRows) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) acc += red[w * kGemvRows + tid];
        p.vpart[lc * p.ldp + rb * kGemvRows + tid] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.rb_cnt[rb], 1u) == (uint32_t)(p.LC - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // last CTA of this row block: combine the chunks in order and finish the rows
    double v = 0.0;
    const int64_t row = rb * kGemvRows + tid;
    if (tid < kGemvRows) {
        double acc = 0.0;
        for (int64_t cc = 0; cc < p.LC; ++cc) acc += __ldcg(&p.vpart[cc * p.ldp + row]);
        if (row < p.m) {
            const double base = (p.mode == 0) ? load_x(p.X, p.xt, piv * p.ldx + row) : p.vin[row];
            v = base - acc;
        }
        p.vout[row] = v;
        float hi, lo;
        split_double(v, hi, lo);
        if (p.mode == 0) {
            p.vouth[row] = hi;
            p.voutl[row] = lo;
        } else {
            // tile-interleaved for the fused pass: tile t = [hi(rows_t) | lo(rows_t)]
            const int64_t t = row / p.MT;
            const int64_t rt = min(p.MT, p.ldp - t * p.MT);
            const int64_t off = t * 2 * p.MT + (row - t * p.MT);
            p.vouth[off] = hi;
            p.vouth[off + rt] = lo;
        }
    }
    if (tid == 0) p.rb_cnt[rb] = 0;
    if (p.mode == 0) return;

    // C: ||v2||^2 of this row block (fixed-order tree), then the grid-level last arriver
    __syncthreads();
    double* sq = red;
    if (tid < kGemvRows) sq[tid] = v * v;
    __syncthreads();
    for (int o = kGemvRows / 2; o > 0; o >>= 1) {
        if (tid < o) sq[tid] += sq[tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        p.nu2part[rb] = sq[0];
        __threadfence();
        s_last = (atomicAdd(&ctl->c_arrive, 1u) == (uint32_t)(p.RB - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < 32) {
        // fixed order: lane l sums a contiguous range of row blocks, then a fixed shuffle tree
        const int64_t b0 = (p.RB * tid) / 32, b1 = (p.RB * (tid + 1)) / 32;
        double acc = 0.0;
        for (int64_t b = b0; b < b1; ++b) acc += __ldcg(&p.nu2part[b]);
        acc = warp_sum_double(acc);
        if (tid == 0) {
            const double nu = sqrt(acc);
            const double xin = sqrt(p.xn2[piv]);
            const int64_t k = p.k;
            ctl->c_arrive = 0;
            int32_t stop = STOP_NONE;
            if (k > 0) {
                // nu is the FP64 residual of the column that maximised the indicator after k
                // bases: the certified E_cur of step 2.3, free of the cancellation in
                // ||x||^2 - ||c||^2.  Step 2.4 of the previous iteration is decided on it.
                p.err[k - 1] = nu;
                ctl->err_last = nu;
                if (ctl->mode == MODE_FRO_REL) {
                    if (ctl->fro_last <= ctl->fro_tol) stop = STOP_TOL;
                } else if (nu <= ctl->eps_r) {
                    stop = STOP_TOL;
                }
            }
            if (stop == STOP_NONE && k >= ctl->d_max) stop = STOP_DMAX;
            // step 2.2: break if ||v|| < eps_R, or below the numerical-rank floor
            if (stop == STOP_NONE && (nu < ctl->eps_r22 || !(nu > rank_floor_of(ctl->mode) * xin))) stop = STOP_BREAK;
            if (stop != STOP_NONE) {
                ctl->stop = stop;
                if (p.progress) {
                    volatile uint32_t* pr = p.progress;
                    pr[1] = (uint32_t)stop;
                    __threadfence_system();
                }
            } else {
                ctl->nu = nu;
                ctl->inv_nu = 1.0 / nu;
                p.pivots[k] = piv;
                if (p.nu_out) p.nu_out[k] = nu;
            }
        }
    }
}

struct GemvTParams {
    const float* yh;
    const float* yl;
    const float* vh;
    const float* vl;
    double* hpart;            // NRC x d_max
    uint32_t* lb_cnt;
    double* h;
    int64_t ldp, k, d_max, RCH, NRC;
    Ctl* ctl;
};

// grid (ceil(k / 8), NRC), 256 threads: warp w handles coefficient l = 8 * blockIdx.x + w over
// the rows [blockIdx.y * RCH, ...); the last CTA of each coefficient block sums the row chunks.
__global__ void __launch_bounds__(256) orth_gemv_t_kernel(GemvTParams p) {
    Ctl* ctl = p.ctl;
    if (ctl->stop != 0 || ctl->status != 0) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t lb = blockIdx.x, rc = blockIdx.y;
    const int64_t l = lb * 8 + warp;
    const int64_t r0 = rc * p.RCH, r1 = min(p.ldp, r0 + p.RCH);
    __shared__ int s_last;
    if (l < p.k) {
        float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
        constexpr int kU = 4;
        for (int64_t rr = r0 + 4 * lane; rr < r1; rr += 128 * kU) {
            float4 a[kU], b[kU], x[kU], y[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int64_t r = rr + 128 * u;
                if (r < r1) {
                    a[u] = *(const float4*)(p.yh + l * p.ldp + r);
                    b[u] = *(const float4*)(p.yl + l * p.ldp + r);
                    x[u] = *(const float4*)(p.vh + r);
                    y[u] = *(const float4*)(p.vl + r);
                } else {
                    a[u] = b[u] = x[u] = y[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                ff_mac2(s[0], c[0], a[u].x, b[u].x, x[u].x, y[u].x);
                ff_mac2(s[1], c[1], a[u].y, b[u].y, x[u].y, y[u].y);
                ff_mac2(s[2], c[2], a[u].z, b[u].z, x[u].z, y[u].z);
                ff_mac2(s[3], c[3], a[u].w, b[u].w, x[u].w, y[u].w);
            }
        }
        double t = ff_to_double(s[0], c[0]) + ff_to_double(s[1], c[1]) + ff_to_double(s[2], c[2]) +
                   ff_to_double(s[3], c[3]);
        t = warp_sum_double(t);
        if (lane == 0) p.hpart[rc * p.d_max + l] = t;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&p.lb_cnt[lb], 1u) == (uint32_t)(p.NRC - 1));
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < 8) {
        const int64_t ll = lb * 8 + tid;
        if (ll < p.k) {
            double acc = 0.0;
            for (int64_t cc = 0; cc < p.NRC; ++cc) acc += __ldcg(&p.hpart[cc * p.d_max + ll]);
            p.h[ll] = acc;
        }
    }
    if (tid == 0) p.lb_cnt[lb] = 0;
}

static void gemv_n_geometry(const Work& w, int64_t k, int64_t& LC, int64_t& LCH) {
    if (k <= 0) {
        LC = 1;
        LCH = 0;
        return;
    }
    int64_t lc = ceil_div(kGemvTargetCtas, w.RB);
    lc = std::min<int64_t>(lc, ceil_div(k, 8));
    lc = std::max<int64_t>(lc, 1);
    lc = std::min<int64_t>(lc, w.LC_MAX);
    LCH = ceil_div(k, lc);
    LC = ceil_div(k, LCH);
}

static cudaError_t launch_gemv_n(const Work& w, GemvNParams& p, int64_t k, cudaStream_t st) {
    int64_t LC, LCH;
    gemv_n_geometry(w, k, LC, LCH);
    p.k = k;
    p.LC = LC;
    p.LCH = LCH;
    p.RB = w.RB;
    p.m = w.m;
    p.ldp = w.ldp;
    p.yh = w.yh;
    p.yl = w.yl;
    p.vpart = w.vpart;
    p.rb_cnt = w.rb_cnt;
    p.xn2 = w.xn2;
    p.ctl = w.ctl;
    const size_t smem = (size_t)round_up(8 * LCH, 16) + 8 * kGemvRows * 8;
    dim3 grid((unsigned)w.RB, (unsigned)LC);
    orth_gemv_n_kernel<<<grid, 256, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_orth_a1(const Work& w, const void* X, const double* T, int64_t ldt, int64_t k,
                           cudaStream_t st) {
    GemvNParams p = {};
    p.mode = 0;
    p.X = X;
    p.xt = w.xt;
    p.ldx = w.ldx;
    p.T = T;
    p.ldt = ldt;
    p.vout = w.v1;
    p.vouth = w.v1h;
    p.voutl = w.v1l;
    return launch_gemv_n(w, p, k, st);
}

cudaError_t launch_orth_c(const Work& w, int64_t k, int64_t* pivots, double* nu_out, double* err,
                          uint32_t* progress, cudaStream_t st) {
    GemvNParams p = {};
    p.mode = 1;
    p.err = err;
    p.progress = progress;
    p.h = w.h;
    p.vin = w.v1;
    p.vout = w.v2;
    p.vouth = w.v2s;
    p.voutl = nullptr;
    p.MT = w.MT;
    p.nu2part = w.nu2part;
    p.pivots = pivots;
    p.nu_out = nu_out;
    return launch_gemv_n(w, p, k, st);
}

cudaError_t launch_orth_a2(const Work& w, int64_t k, cudaStream_t st) {
    if (k <= 0) return cudaSuccess;
    GemvTParams p;
    p.yh = w.yh;
    p.yl = w.yl;
    p.vh = w.v1h;
    p.vl = w.v1l;
    p.hpart = w.hpart;
    p.lb_cnt = w.lb_cnt;
    p.h = w.h;
    p.ldp = w.ldp;
    p.k = k;
    p.d_max = w.d_max;
    p.ctl = w.ctl;
    const int64_t LB = ceil_div(k, 8);
    int64_t nrc = ceil_div(kGemvTargetCtas, LB);
    nrc = std::max<int64_t>(1, std::min<int64_t>(nrc, w.RC_MAX));
    int64_t rch = round_up(ceil_div(w.ldp, nrc), 128);
    nrc = ceil_div(w.ldp, rch);
    p.RCH = rch;
    p.NRC = nrc;
    dim3 grid((unsigned)LB, (unsigned)nrc);
    orth_gemv_t_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace rbd
