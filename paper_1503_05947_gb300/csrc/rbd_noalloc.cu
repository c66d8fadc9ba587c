// rbd_noalloc.cu -- rbd_compress_noalloc: Algorithm 1 with its workspace in a fixed, statically
// sized device array instead of memory obtained from an allocator.
//
// Some callers must not allocate while they compress: a serving loop that forbids allocator
// calls on its hot path (cudaMalloc can synchronise the whole device, and a stream-ordered
// pool may have to grow), a process whose HBM is already held by another caching allocator,
// or code that runs under a hard memory cap where any new allocation may fail.  For them this
// entry point takes its scratch from g_noalloc_scratch, a __device__ array that exists as soon
// as this translation unit's module is loaded on a device, and calls no allocating routine:
// no cudaMalloc / cudaMallocAsync / cudaFree, no host-pinned or mapped buffer, no CUDA events.
//
// Setup: the first call on a device (with that device current) sets the kernel attributes (the
// same per-device setup as rbd_compress, device_state in rbd_abi.cu) and looks up the array's
// device address with cudaGetSymbolAddress; later calls on that device reuse what was recorded.
// The argument rules and the choice of path are rbd_compress's own (validate, plan_work), so the
// two entry points cannot drift apart.  Because the array is one per device and per process, calls that
// overlap on the same device -- from several host threads, or on several streams -- race on
// it and corrupt each other's results: callers serialise them.
#include <cstring>
#include <mutex>

#include "../../include/rbd.h"
#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

// The workspace of one call (control block, re-laid-out X, split Y and the O(m + n + d_max)
// vectors); its size is RBD_NOALLOC_SCRATCH_BYTES.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RBD_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_na_mu;
void* g_na_scratch[64];

// The device address of g_noalloc_scratch on the current device (looked up once per device;
// in host code the array's name is only a host-side stand-in for it).
cudaError_t noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (p == nullptr || ((uintptr_t)p & 255u) != 0) return cudaErrorInvalidSymbol;
        g_na_scratch[dev] = p;
    }
    *out = g_na_scratch[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace rbd

using namespace rbd;

extern "C" rbd_status rbd_compress_noalloc(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                                           double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                                           double* Y, int64_t ldy, double* T, int64_t ldt, int64_t* pivots,
                                           double* err, double* nu, void* stream, rbd_result* result) {
    rbd_status v = validate(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    DeviceState ds;
    void* scratch = nullptr;
    cudaError_t ce = device_state(ds);
    if (ce == cudaSuccess) ce = noalloc_scratch(&scratch);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(ce);
    }
    const bool acc32 = xt == RBD_F32_ACC32;
    xt = (rbd_dtype)storage_of((int)xt);
    Work w;
    if (!plan_work(w, m, n, ldx, d_max, (int)xt, ds.num_sms, ds.pass_ctas_per_sm[(int)xt], ds.loop_max_smem, 0,
                   mode != RBD_TOL_NONE))
        return RBD_EUNSUPPORTED;
    if (xt == RBD_BF16 && !w.use_loop) return RBD_EUNSUPPORTED;
    if (acc32 && !w.use_defer) return RBD_EUNSUPPORTED;
    w.acc32 = acc32 ? 1 : 0;
    // the problem's workspace must fit the fixed array
    if (w.total_bytes > (size_t)RBD_NOALLOC_SCRATCH_BYTES) return RBD_ENOMEM;
    carve_work(w, scratch);
    cudaStream_t st = (cudaStream_t)stream;

    // the control block and the last-arriver counters start at zero
    int32_t launches = 0;
    ce = cudaMemsetAsync(scratch, 0, w.zero_bytes, st);
    if (ce == cudaSuccess) {
        ce = launch_init(w, X, tol, (int)mode, start, st);
        ++launches;
    }
    if (w.use_loop) {
        if (ce == cudaSuccess) {
            ce = w.use_defer ? launch_defer(w, X, Y, ldy, T, ldt, pivots, err, nu, 0, st)
                             : launch_loop(w, X, Y, ldy, T, ldt, pivots, err, nu, 0, st);
            ++launches;
        }
    } else {
        // stepwise: every step is enqueued; kernels launched after the device stopped return at
        // entry (no host-mapped progress word, which would need a pinned host allocation)
        for (int64_t k = 0; k <= d_max && ce == cudaSuccess; ++k) {
            ce = launch_orth_a1(w, X, T, ldt, k, st);
            ++launches;
            if (ce == cudaSuccess && k > 0) {
                ce = launch_orth_a2(w, k, st);
                ++launches;
            }
            if (ce == cudaSuccess) {
                ce = launch_orth_c(w, k, pivots, nu, err, nullptr, st);
                ++launches;
            }
            if (k == d_max) break;
            if (ce == cudaSuccess) {
                ce = launch_pass(w, Y, ldy, T, ldt, k, nullptr, st);
                ++launches;
            }
        }
    }

    Ctl hctl;
    memset(&hctl, 0, sizeof(hctl));
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(ce);
    }
    rbd_status rs = (hctl.status != ST_OK) ? (rbd_status)hctl.status : RBD_OK;
    if (result) {
        result->d = hctl.d;
        result->next_pivot = hctl.pivot;
        result->stop_reason = hctl.stop;
        result->launches = launches;
        result->err_last = hctl.d > 0 ? hctl.err_last : 0.0;
        result->fro_last = hctl.fro_last;
        result->x_fro = hctl.x_fro;
        result->x_maxcol = hctl.x_maxcol;
    }
    return rs;
}
