// rbd_rows.cu -- the row-space form (Section 3.1: each column, "or row if we are compressing the
// row space", of the data matrix is one entry): rbd_compress_rows compresses the rows of a
// column-major X by running the path on X' (n x m, column-major), which this tiled transpose
// writes into a stream-ordered scratch buffer.  A pure copy: the values are moved, not computed.
#include <stdint.h>

#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

// Xt(j, i) = X(i, j): X is m x n column-major (ldx), Xt is n x m column-major (ld = n).  One 32 x 32
// tile per iteration of a grid-stride loop over tiles, staged in shared memory (one padding column
// against bank conflicts) so that both the reads of X and the writes of Xt are coalesced.
template <typename E>
__global__ void __launch_bounds__(256) transpose_kernel(const E* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                                                        E* __restrict__ Xt) {
    __shared__ E tile[32][33];
    const int64_t ti = (m + 31) / 32, tj = (n + 31) / 32, ntiles = ti * tj;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t i0 = (t % ti) * 32, j0 = (t / ti) * 32;
        for (int jj = threadIdx.y; jj < 32; jj += 8) {
            const int64_t i = i0 + threadIdx.x, j = j0 + jj;
            if (i < m && j < n) tile[jj][threadIdx.x] = X[j * ldx + i];
        }
        __syncthreads();
        for (int ii = threadIdx.y; ii < 32; ii += 8) {
            const int64_t j = j0 + threadIdx.x, i = i0 + ii;
            if (i < m && j < n) Xt[i * n + j] = tile[threadIdx.x][ii];
        }
        __syncthreads();
    }
}

cudaError_t launch_transpose(const void* X, int esize, int64_t m, int64_t n, int64_t ldx, void* Xt, int num_sms,
                             cudaStream_t st) {
    const int64_t tiles = ceil_div(m, 32) * ceil_div(n, 32);
    const int64_t cap = (int64_t)(num_sms > 0 ? num_sms : 152) * 8;
    const unsigned blocks = (unsigned)(tiles < cap ? tiles : cap);
    const dim3 thr(32, 8);
    if (esize == 8)
        transpose_kernel<uint64_t><<<blocks, thr, 0, st>>>((const uint64_t*)X, m, n, ldx, (uint64_t*)Xt);
    else if (esize == 4)
        transpose_kernel<uint32_t><<<blocks, thr, 0, st>>>((const uint32_t*)X, m, n, ldx, (uint32_t*)Xt);
    else
        transpose_kernel<uint16_t><<<blocks, thr, 0, st>>>((const uint16_t*)X, m, n, ldx, (uint16_t*)Xt);
    return cudaGetLastError();
}

}  // namespace rbd
