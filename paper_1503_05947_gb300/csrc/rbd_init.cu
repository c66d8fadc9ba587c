// rbd_init.cu -- the initial pass over X (Section 3.3, "pre-computation of diag(X'AX)"):
// e_j = ||X(:, j)||_A^2 for every column (A = I, or A = diag(w) in the A-norm form, where the
// Euclidean ||X(:, j)||^2 is kept as well for the numerical-rank floor), ||X||_F and
// max_j ||X(:, j)|| in the same norm for the tolerance modes, and the one-time re-layout of X
// into the tile-major plane format the fused pass streams with bulk copies (rbd_work.h).
#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

struct InitParams {
    const void* X;
    int64_t ldx, m, n, ldp;
    int64_t ncols_pad;        // ngroups * C: columns of the plane layout
    int C, MT;
    int64_t group_stride, tile_stride;
    void* planes;
    double* e;
    double* xn2;
    const double* wts;        // A = diag(wts), or nullptr for A = I
    Ctl* ctl;
    double tol;
    int mode;
    int64_t start;
    int64_t d_max;
};

// One warp per column of the plane layout; lane l handles rows 4l..4l+3 of every 128-row chunk.
template <int XT>
__global__ void __launch_bounds__(256) init_kernel(InitParams p) {
    constexpr int P = (XT == 0) ? 2 : 1;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int bad = ST_OK;
    for (int64_t j = gw; j < p.ncols_pad; j += nw) {
        const int64_t g = j / p.C;
        const int c = (int)(j % p.C);
        const bool live = j < p.n;
        float s = 0.f, cc = 0.f, sa = 0.f, ca = 0.f;
        if (p.wts && j == 0) {
            // the weights of A = diag(w) must be finite and positive
            for (int64_t r = lane; r < p.m; r += 32) {
                const double wr = p.wts[r];
                if (!(isfinite(wr) && wr > 0.0)) bad = ST_EINVAL;
            }
        }
        for (int64_t r0 = 4 * lane; r0 < p.ldp; r0 += 128) {
            const int64_t t = r0 / p.MT;
            const int64_t rt = min((int64_t)p.MT, p.ldp - t * p.MT);
            const int64_t base = g * p.group_stride + t * p.tile_stride + (int64_t)c * P * rt + (r0 - t * p.MT);
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t r = r0 + q;
                x[q] = 0.0;
                if (live && r < p.m) {
                    if (XT == 0) x[q] = ((const double*)p.X)[j * p.ldx + r];
                    else if (XT == 1) x[q] = (double)((const float*)p.X)[j * p.ldx + r];
                    else x[q] = (double)__bfloat162float(((const __nv_bfloat16*)p.X)[j * p.ldx + r]);
                }
                // exponent field all ones: Inf or NaN (an integer test: FP64 comparisons are slow here)
                if ((((unsigned long long)__double_as_longlong(x[q]) >> 52) & 0x7ffu) == 0x7ffu) {
                    bad = ST_ENONFINITE;
                    x[q] = 0.0;
                }
            }
            if (p.wts) {
                // w_r x_r^2 as (w_r x_r) * x_r: the FP64 product split, times the split x_r
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t r = r0 + q;
                    const double wx = (live && r < p.m) ? p.wts[r] * x[q] : 0.0;
                    float xh, xl, wh, wl;
                    split_double(x[q], xh, xl);
                    split_double(wx, wh, wl);
                    ff_mac2(sa, ca, xh, xl, wh, wl);
                }
            }
            if (XT == 0) {
                float hi[4], lo[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // |x| >= 2^127 (biased exponent >= 1023 + 127): outside the split's FP32 range
                    if ((((unsigned long long)__double_as_longlong(x[q]) >> 52) & 0x7ffu) >= 1150u)
                        bad = (bad == ST_OK) ? ST_EUNSUPPORTED : bad;
                    split_f64_fast(x[q], hi[q], lo[q]);
                    ff_mac2(s, cc, hi[q], lo[q], hi[q], lo[q]);
                }
                float* ph = (float*)p.planes + base;
                *reinterpret_cast<float4*>(ph) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<float4*>(ph + rt) = make_float4(lo[0], lo[1], lo[2], lo[3]);
            } else if (XT == 1) {
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = (float)x[q];
                    ff_mac1(s, cc, v[q], v[q], 0.f);
                }
                *reinterpret_cast<float4*>((float*)p.planes + base) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
                __nv_bfloat16 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = __float2bfloat16((float)x[q]);  // exact: the value came from bf16
                    const float f = (float)x[q];
                    ff_mac1(s, cc, f, f, 0.f);
                }
                __nv_bfloat162* pb = reinterpret_cast<__nv_bfloat162*>((__nv_bfloat16*)p.planes + base);
                pb[0] = __halves2bfloat162(v[0], v[1]);
                pb[1] = __halves2bfloat162(v[2], v[3]);
            }
        }
        const double tsum = warp_sum_double(ff_to_double(s, cc));
        const double asum = p.wts ? warp_sum_double(ff_to_double(sa, ca)) : tsum;
        if (live && lane == 0) {
            p.e[j] = asum;
            p.xn2[j] = tsum;
        }
    }
    if (bad != ST_OK) raise_status(p.ctl, bad);

    // Last CTA to finish: column-norm statistics in a fixed order, and the tolerances.
    __shared__ int s_last;
    __shared__ double s_sum[256], s_max[256];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&p.ctl->init_arrive, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int64_t t = threadIdx.x, nt = blockDim.x;
    const int64_t j0 = (p.n * t) / nt, j1 = (p.n * (t + 1)) / nt;
    double sum = 0.0, mx = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double v = __ldcg(p.wts ? &p.e[j] : &p.xn2[j]);
        sum += v;
        mx = fmax(mx, v);
    }
    s_sum[t] = sum;
    s_max[t] = mx;
    __syncthreads();
    for (int o = (int)nt / 2; o > 0; o >>= 1) {
        if (t < o) {
            s_sum[t] += s_sum[t + o];
            s_max[t] = fmax(s_max[t], s_max[t + o]);
        }
        __syncthreads();
    }
    if (t == 0) {
        Ctl* ctl = p.ctl;
        const double fro = sqrt(s_sum[0]);
        const double maxcol = sqrt(s_max[0]);
        ctl->x_fro = fro;
        ctl->x_maxcol = maxcol;
        ctl->tol = p.tol;
        ctl->mode = p.mode;
        ctl->d_max = p.d_max;
        if (p.mode == MODE_FRO_REL) {
            ctl->fro_tol = p.tol * fro;  // compared with sqrt(sum of e_j)
            ctl->eps_r = -1.0;
            ctl->eps_r22 = p.tol * fro / sqrt((double)p.n);
        } else if (p.mode == MODE_NONE) {
            // no tolerance: exactly d_max bases (a measurement mode)
            ctl->fro_tol = -1.0;
            ctl->eps_r = -1.0;
            ctl->eps_r22 = -1.0;
        } else {
            const double eps = (p.mode == MODE_MAXCOL_REL) ? p.tol * maxcol : p.tol;
            ctl->fro_tol = -1.0;
            ctl->eps_r = eps;
            ctl->eps_r22 = eps;
        }
        ctl->d = 0;
        ctl->pivot = p.start;
        ctl->err_last = 0.0;
        ctl->fro_last = fro;
        ctl->stop = (ctl->status != ST_OK) ? STOP_BREAK : STOP_NONE;
        ctl->init_arrive = 0;
    }
}

cudaError_t launch_init(const Work& w, const void* X, double tol, int mode, int64_t start,
                        cudaStream_t st) {
    InitParams p;
    p.X = X;
    p.ldx = w.ldx;
    p.m = w.m;
    p.n = w.n;
    p.ldp = w.ldp;
    p.ncols_pad = w.ngroups * w.C;
    p.C = w.C;
    p.MT = w.MT;
    p.group_stride = w.group_stride;
    p.tile_stride = w.tile_stride;
    p.planes = w.planes;
    p.e = w.e;
    p.xn2 = w.xn2;
    p.wts = w.wts;
    p.ctl = w.ctl;
    p.tol = tol;
    p.mode = mode;
    p.start = start;
    p.d_max = w.d_max;
    int blocks = (int)ceil_div(p.ncols_pad, 8);
    const int cap = w.num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    switch (w.xt) {
        case 0: init_kernel<0><<<blocks, 256, 0, st>>>(p); break;
        case 1: init_kernel<1><<<blocks, 256, 0, st>>>(p); break;
        default: init_kernel<2><<<blocks, 256, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}

}  // namespace rbd
