// rbd_loop.cuh -- pieces shared by the two persistent loop kernels (rbd_loop.cu: four grid
// barriers per basis, every form; rbd_defer.cu: two grid barriers per basis, A = I): the bounded
// grid-wide barrier of a cooperative launch, the abort protocol, and the geometry of the Y-slice
// chunks streamed through the pass ring.
#pragma once

#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

constexpr uint64_t kBarrierLimitNs = 2000000000ull;

// Ring stages per Y-chunk buffer: a chunk of a tall row block spans several stages, so that it
// still holds about 32 columns of both planes (at most half the ring, so that two chunks are in
// flight).
template <class Cfg>
__host__ __device__ inline int loop_ybuf_stages(int R) {
    constexpr int S = Cfg::S, STAGE = Cfg::STAGE_FLOATS;
    int spb = (int)((32 * 2 * (int64_t)R + STAGE - 1) / STAGE);
    if (spb > S / 2) spb = S / 2;
    if (spb < 1) spb = 1;
    return spb;
}

// Y columns per chunk: both planes of LC x R floats fill one Y-chunk buffer.
template <class Cfg>
__host__ __device__ inline int loop_chunk_cols(int R) {
    int lc = (loop_ybuf_stages<Cfg>(R) * Cfg::STAGE_FLOATS / 2) / R;
    lc &= ~3;
    if (lc > 256) lc = 256;
    return lc;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bit 31 of the grid-barrier word: set by a CTA that raised an error, so that every other CTA
// leaves at its next barrier without a separate read of the status word (the arrival count stays
// far below 2^31: G * 4 barriers per basis).
constexpr uint32_t kAbortBit = 0x80000000u;

__device__ __forceinline__ void loop_abort(Ctl* ctl, uint32_t* bar, int32_t st) {
    raise_status(ctl, st);
    atomicOr(bar, kAbortBit);
}

// Thread 0's wait for a grid barrier: its arrival counter reaching target.  1 when passed, 0 when
// the abort bit appeared or limit_ns elapsed (the latter raises the abort).
__device__ __forceinline__ int grid_poll(uint32_t* bar, uint32_t target, Ctl* ctl, uint64_t limit_ns) {
    uint32_t v = ld_acquire_u32(bar);
    if (!(v & kAbortBit) && v < target) {
        const uint64_t t0 = globaltimer_ns();
        while (true) {
            v = ld_acquire_u32(bar);
            if ((v & kAbortBit) || v >= target) break;
            if (globaltimer_ns() - t0 > limit_ns) {
                loop_abort(ctl, bar, ST_ETIMEOUT);
                v = kAbortBit;
                break;
            }
        }
    }
    return (v & kAbortBit) ? 0 : 1;
}

// Grid-wide barrier for a cooperative launch; called by every thread of every CTA.  The arrival
// counter only grows: the barrier with index gen (1, 2, ...) is passed once it reaches
// nblocks * gen, so no CTA has to reset it and the last arrival needs no extra release step.
// Returns false in all threads of a CTA whose wait ran out (RBD_ETIMEOUT) or that saw the abort
// bit (the caller then leaves the loop).
__device__ __forceinline__ bool grid_sync(uint32_t* bar, uint32_t nblocks, uint32_t& gen, int* s_ok, Ctl* ctl,
                                          uint64_t limit_ns = kBarrierLimitNs) {
    __syncthreads();
    ++gen;  // in every thread: any thread may poll the next barrier
    if (threadIdx.x == 0) {
        // arrival without a returned value (no round trip before the first poll); the first poll
        // of the same word already sees it
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        *s_ok = grid_poll(bar, nblocks * gen, ctl, limit_ns);
    }
    __syncthreads();
    return *s_ok != 0;
}

// One lane's share of a sum over the CTAs: v[b * stride] for b = lane, lane + 32, ... (< G),
// added in that order.  Every load is issued before the first addition: in a loop whose trip
// count the compiler cannot see, each round trip to L2 would wait for the one before.
__device__ __forceinline__ double lane_sum_ctas(const double* v, int64_t stride, int64_t G, int lane) {
    constexpr int SL = kLoopMaxCtas / 32;
    double x[SL];
#pragma unroll
    for (int i = 0; i < SL; ++i) x[i] = (lane + 32 * i < G) ? __ldcg(v + (int64_t)(lane + 32 * i) * stride) : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < SL; ++i)
        if (lane + 32 * i < G) acc += x[i];
    return acc;
}

// The arrival half of grid_sync, so that a CTA can work between publishing its writes and waiting
// for everyone else's: ONE thread, after a barrier among the threads whose writes it publishes (the
// release is cumulative over them).  The wait is grid_poll (target nblocks * gen, gen counted in
// every thread) followed by a CTA barrier that broadcasts its result.
__device__ __forceinline__ void grid_arrive(uint32_t* bar) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}

}  // namespace rbd
