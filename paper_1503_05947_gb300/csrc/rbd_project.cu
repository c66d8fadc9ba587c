// rbd_project.cu -- the out-of-sample map of Section 3.1, v_C = Y' v (Section 3.3 "Online":
// cost m d per vector), for a block of k vectors: C = Y' V.
//
// Each CTA owns a 32 x 32 tile of C and walks the m rows in 32-row chunks staged in shared
// memory, split into float-float form on load; each thread accumulates 4 outputs over all m
// rows in order (deterministic), FP64-grade accuracy on the FP32 pipes.
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

// grid (ceil(d/32), ceil(k/32)), 256 threads; thread (ty = tid / 8, tx = tid % 8) computes
// C(l0 + ty, c0 + tx + 8 q), q = 0..3.
__global__ void __launch_bounds__(256) project_kernel(ProjParams p) {
    __shared__ float yh[kPT][kPT + 1], yl[kPT][kPT + 1];   // [row][basis]
    __shared__ float vh[kPT][kPT + 1], vl[kPT][kPT + 1];   // [row][vector]
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;
    const int64_t l0 = (int64_t)blockIdx.x * kPT, c0 = (int64_t)blockIdx.y * kPT;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t r0 = 0; r0 < p.m; r0 += kPT) {
        // stage a 32-row chunk of Y(:, l0:l0+32) and V(:, c0:c0+32); element (row, col) is
        // loaded by thread (col * 32 + row) % 256 four times over.
        for (int idx = tid; idx < kPT * kPT; idx += 256) {
            const int row = idx % kPT, col = idx / kPT;
            const int64_t r = r0 + row;
            double y = 0.0, v = 0.0;
            if (r < p.m) {
                if (l0 + col < p.d) y = p.Y[(l0 + col) * p.ldy + r];
                if (c0 + col < p.k) v = load_v(p.V, p.vt, (c0 + col) * p.ldv + r);
            }
            float a, b;
            split_double(y, a, b);
            yh[row][col] = a;
            yl[row][col] = b;
            split_double(v, a, b);
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
            if (col < p.k) p.C[col * p.ldc + l] = ff_to_double(s[q], c[q]);
        }
    }
}

cudaError_t launch_project(const double* Y, int64_t m, int64_t d, int64_t ldy, const void* V, int vt,
                           int64_t k, int64_t ldv, double* C, int64_t ldc, cudaStream_t st) {
    ProjParams p{Y, m, d, ldy, V, vt, k, ldv, C, ldc};
    dim3 grid((unsigned)ceil_div(d, kPT), (unsigned)ceil_div(k, kPT));
    project_kernel<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace rbd
