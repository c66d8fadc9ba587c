// rbd_resume.cu -- restoring the loop state of Algorithm 1 after d0 bases, so that a compression
// can be continued to a larger d_max (rbd_compress_resume).
//
// The state the greedy loop carries from one basis to the next is rebuilt from the caller's
// outputs (Y(:, 0:d0), T(0:d0, :), pivots) with the same floating-point operations, in the same
// order, as the loop produced it:
//   resume_state_kernel     e_j = ||x_j||^2 downdated by T(l, j)^2 for l = 0..d0-1 (Eq. (evalerr),
//                           A = I; the pivot column of step l is set to 0 there), and the
//                           per-group sums of e_j for the Frobenius residual
//                           (and, for the two-barrier loop kernel, T(0:d0, :) in FP32 in the
//                           group-blocked layout its flush corrections stream)
//   resume_y_kernel         the split FP32 copy of Y the Gram-Schmidt GEMVs stream
//   resume_finalize_kernel  the Frobenius residual (the order of the path that continues), the
//                           next pivot and d in the control block
#include <algorithm>

#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

struct ResumeParams {
    const double* T;
    int64_t ldt;
    const int64_t* piv;
    int64_t k0;
    const double* Y;
    int64_t ldy;
    int64_t m, n, ldp, ngroups;
    int C;
    double* e;
    const double* xn2;
    double* gsum;         // the group sums the continuing path reads first (a parity copy on the
                          // two-barrier path)
    float* tf;            // two-barrier path: T(0:d0, :) in FP32, group-blocked; else nullptr
    int use_loop;
    float* ysb;   // persistent kernel: [G][2][d_max][RS]
    int R, RS, G_loop;
    float *yh, *yl;  // stepwise path: ldp x d_max each
    int64_t d_max;
    Ctl* ctl;
    int64_t next_pivot;
};

// one warp per column group; lane c replays the downdates of column g C + c
__global__ void __launch_bounds__(256) resume_state_kernel(ResumeParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = gw; g < p.ngroups; g += nw) {
        const int64_t j = g * p.C + lane;
        double e = 0.0;
        if (lane < p.C && j < p.n) {
            e = p.xn2[j];
            for (int64_t l = 0; l < p.k0; ++l) {
                const double c = p.T[j * p.ldt + l];
                e = (j == p.piv[l]) ? 0.0 : fmax(e - c * c, 0.0);
                if (p.tf) p.tf[(g * p.d_max + l) * p.C + lane] = __double2float_rn(c);
            }
            p.e[j] = e;
        }
        // the group's sum of e_j in the order of the path that continues: columns in order, or
        // (two-barrier loop kernel) the fixed tree over the group's 16 lanes
        const int ncols = (int)min((int64_t)p.C, p.n - g * p.C);
        double s = 0.0;
        if (p.tf) {
            s = (lane < ncols) ? e : 0.0;
            for (int o = p.C / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        } else {
            for (int cw = 0; cw < ncols; ++cw) s += __shfl_sync(0xffffffffu, e, cw);
        }
        if (lane == 0) p.gsum[g] = s;
    }
}

__global__ void __launch_bounds__(256) resume_y_kernel(ResumeParams p) {
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    if (p.use_loop) {
        const int64_t total = (int64_t)p.G_loop * p.R * p.k0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += nthreads) {
            const int64_t r = i % p.R, rest = i / p.R;
            const int64_t l = rest % p.k0, b = rest / p.k0;
            const int64_t row = b * p.R + r;
            const double y = (row < p.m) ? p.Y[row + l * p.ldy] : 0.0;
            float hi, lo;
            split_double(y, hi, lo);
            p.ysb[(b * 2 + 0) * p.d_max * p.RS + l * p.RS + r] = hi;
            p.ysb[(b * 2 + 1) * p.d_max * p.RS + l * p.RS + r] = lo;
        }
    } else {
        const int64_t total = p.ldp * p.k0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += nthreads) {
            const int64_t r = i % p.ldp, l = i / p.ldp;
            const double y = (r < p.m) ? p.Y[r + l * p.ldy] : 0.0;
            float hi, lo;
            split_double(y, hi, lo);
            p.yh[r + l * p.ldp] = hi;
            p.yl[r + l * p.ldp] = lo;
        }
    }
}

// one warp: the Frobenius residual in the order of the path that continues the loop
__global__ void resume_finalize_kernel(ResumeParams p) {
    const int lane = threadIdx.x & 31;
    double fs = 0.0;
    if (p.use_loop) {
        for (int64_t gg = lane; gg < p.ngroups; gg += 32) fs += p.gsum[gg];
    } else {
        const int64_t g0 = (p.ngroups * lane) / 32, g1 = (p.ngroups * (lane + 1)) / 32;
        for (int64_t g = g0; g < g1; ++g) fs += p.gsum[g];
    }
    fs = warp_sum_double(fs);
    if (lane == 0) {
        p.ctl->fro_last = sqrt(fmax(fs, 0.0));
        p.ctl->pivot = p.next_pivot;
        p.ctl->d = p.k0;
    }
}

cudaError_t launch_resume(const Work& w, const double* Y, int64_t ldy, const double* T, int64_t ldt,
                          const int64_t* pivots, int64_t k0, int64_t next_pivot, cudaStream_t st) {
    ResumeParams p;
    p.T = T;
    p.ldt = ldt;
    p.piv = pivots;
    p.k0 = k0;
    p.Y = Y;
    p.ldy = ldy;
    p.m = w.m;
    p.n = w.n;
    p.ldp = w.ldp;
    p.ngroups = w.ngroups;
    p.C = w.C;
    p.e = w.e;
    p.xn2 = w.xn2;
    // the two-barrier kernel's service warps read the sums of basis k0 - 1 from copy (k0 - 1) & 1
    p.gsum = w.use_defer ? w.gsum + ((k0 - 1) & 1) * w.ngroups : w.gsum;
    p.tf = w.use_defer ? w.tf : nullptr;
    p.use_loop = w.use_loop;
    p.ysb = w.ysb;
    p.R = w.R;
    p.RS = w.RS;
    p.G_loop = w.G_loop;
    p.yh = w.yh;
    p.yl = w.yl;
    p.d_max = w.d_max;
    p.ctl = w.ctl;
    p.next_pivot = next_pivot;
    const int sblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(w.ngroups, (int64_t)8), 4096));
    resume_state_kernel<<<sblocks, 256, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int64_t total = w.use_loop ? (int64_t)w.G_loop * w.R * k0 : w.ldp * k0;
        const int yblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, (int64_t)256), 8192));
        resume_y_kernel<<<yblocks, 256, 0, st>>>(p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        resume_finalize_kernel<<<1, 32, 0, st>>>(p);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace rbd
