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
// Setup: the first call on a device (with that device current) sets the kernel attributes and
// looks up the array's device address with cudaGetSymbolAddress; later calls on that device
// reuse what was recorded.  Because the array is one per device and per process, calls that
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

struct NoallocDevice {
    bool ready = false;
    int num_sms = 0;
    int pass_ctas_per_sm[3] = {1, 1, 1};
    int loop_max_smem = 0;
    void* scratch = nullptr;
};

std::mutex g_na_mu;
NoallocDevice g_na_dev[64];

bool stepwise_forced() {
    const char* v = getenv("RBD_STEPWISE");
    return v && v[0] && v[0] != '0';
}

// One-time setup of the current device: SM count, kernel attributes, scratch address.
cudaError_t noalloc_device(NoallocDevice& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    NoallocDevice& s = g_na_dev[dev];
    if (!s.ready) {
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = pass_kernel_setup(s.pass_ctas_per_sm);
        if (e != cudaSuccess) return e;
        int coop = 0, optin = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        s.loop_max_smem = 0;
        if (coop && optin > 0) {
            if (loop_kernel_setup(optin) == cudaSuccess)
                s.loop_max_smem = optin;
            else
                cudaGetLastError();
        }
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (p == nullptr || ((uintptr_t)p & 255u) != 0) return cudaErrorInvalidSymbol;
        s.scratch = p;
        s.ready = true;
    }
    out = s;
    if (stepwise_forced()) out.loop_max_smem = 0;
    return cudaSuccess;
}

rbd_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return RBD_OK;
    if (e == cudaErrorMemoryAllocation) return RBD_ENOMEM;
    return RBD_ECUDA;
}

// The argument rules of rbd_compress.
rbd_status check_args(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                      rbd_tol_mode mode, int64_t d_max, int64_t start, const double* Y, int64_t ldy,
                      const double* T, int64_t ldt, const int64_t* pivots, const double* err) {
    if (!X || !Y || !T || !pivots || !err) return RBD_EINVAL;
    if (xt != RBD_F64 && xt != RBD_F32 && xt != RBD_BF16) return RBD_EINVAL;
    if (m < 1 || n < 1 || ldx < m || ldy < m || d_max < 1 || ldt < d_max) return RBD_EINVAL;
    if (d_max > m || d_max > n) return RBD_EINVAL;
    if (start < 0 || start >= n) return RBD_EINVAL;
    if (!(tol >= 0.0) || tol == __builtin_inf()) return RBD_EINVAL;
    if (mode != RBD_TOL_MAXCOL_ABS && mode != RBD_TOL_MAXCOL_REL && mode != RBD_TOL_FRO_REL) return RBD_EINVAL;
    if (m > (int64_t(1) << 40) || n > (int64_t(1) << 40)) return RBD_EUNSUPPORTED;
    return RBD_OK;
}

}  // namespace
}  // namespace rbd

using namespace rbd;

extern "C" rbd_status rbd_compress_noalloc(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                                           double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                                           double* Y, int64_t ldy, double* T, int64_t ldt, int64_t* pivots,
                                           double* err, double* nu, void* stream, rbd_result* result) {
    rbd_status v = check_args(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    NoallocDevice ds;
    cudaError_t ce = noalloc_device(ds);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return map_err(ce);
    }
    Work w;
    if (!plan_work(w, m, n, ldx, d_max, (int)xt, ds.num_sms, ds.pass_ctas_per_sm[(int)xt], ds.loop_max_smem))
        return RBD_EUNSUPPORTED;
    if (xt == RBD_BF16 && !w.use_loop) return RBD_EUNSUPPORTED;
    // the problem's workspace must fit the fixed array
    if (w.total_bytes > (size_t)RBD_NOALLOC_SCRATCH_BYTES) return RBD_ENOMEM;
    carve_work(w, ds.scratch);
    cudaStream_t st = (cudaStream_t)stream;

    // the control block and the last-arriver counters start at zero
    int32_t launches = 0;
    ce = cudaMemsetAsync(ds.scratch, 0, w.zero_bytes, st);
    if (ce == cudaSuccess) {
        ce = launch_init(w, X, tol, (int)mode, start, st);
        ++launches;
    }
    if (w.use_loop) {
        if (ce == cudaSuccess) {
            ce = launch_loop(w, X, Y, ldy, T, ldt, pivots, err, nu, 0, st);
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
        return map_err(ce);
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
