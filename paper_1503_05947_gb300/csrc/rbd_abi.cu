// rbd_abi.cu -- the extern "C" entry points declared in include/rbd.h.
//
// rbd_compress drives Algorithm 1 on one CUDA stream: the initial pass, then per basis the
// three orthogonalisation kernels and the fused pass.  The loop is enqueued without host
// round trips; the last kernel of each step publishes (steps finished, stop reason) to a
// small host-mapped buffer, and the host never runs more than kLookahead steps ahead of the
// device, so an early stop wastes at most a few empty launches.  Kernels launched after the
// device decided to stop return at entry.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/rbd.h"
#include "rbd_device.cuh"
#include "rbd_work.h"

namespace rbd {

static const int kLookahead = 4;

// ---------------------------------------------------------------------------------------
// Workspace planning
// ---------------------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// RBD_LOOP_CLASSIC=1 keeps the four-barrier loop kernel for A = I (for comparisons).
static bool classic_loop_forced() {
    const char* v = getenv("RBD_LOOP_CLASSIC");
    return v && v[0] && v[0] != '0';
}


bool plan_work(Work& w, int64_t m, int64_t n, int64_t ldx, int64_t d_max, int xt, int num_sms,
               int pass_ctas_per_sm, int loop_max_smem, int wt, bool allow_defer) {
    w = Work{};
    w.wt = wt;
    w.m = m;
    w.n = n;
    w.ldx = ldx;
    w.d_max = d_max;
    w.xt = xt;
    w.num_sms = num_sms;
    w.ldp = round_up(m, 128);
    w.planes_n = (xt == RBD_F64) ? 2 : 1;
    w.esize = (xt == RBD_BF16) ? 2 : 4;
    if (xt == RBD_BF16) {
        w.C = PassCfgBf16::C;
        w.MT = PassCfgBf16::MT;
    } else if (xt == RBD_F64) {
        w.C = PassCfg<2>::C;
        w.MT = PassCfg<2>::MT;
    } else {
        w.C = PassCfg<1>::C;
        w.MT = PassCfg<1>::MT;
    }
    w.NT = ceil_div(w.ldp, w.MT);
    w.ngroups = ceil_div(n, w.C);
    w.W = w.NT * w.ngroups;
    w.group_stride = (int64_t)w.C * w.planes_n * w.ldp;
    w.tile_stride = (int64_t)w.C * w.planes_n * w.MT;
    w.G = (int)std::min<int64_t>((int64_t)num_sms * std::max(1, pass_ctas_per_sm), w.W);
    // The persistent loop kernel: one CTA per SM at most, each owning a block of R rows of Y.
    w.use_loop = 0;
    if (loop_max_smem > 0) {
        const int64_t gl = std::min<int64_t>(std::min<int64_t>(num_sms, kLoopMaxCtas),
                                             std::max<int64_t>(w.W, ceil_div(w.ldp, kLoopMaxRows)));
        const int64_t R = round_up(ceil_div(w.ldp, gl), 4);
        if (R <= kLoopMaxRows) {
            const int64_t RS = (R % 8 == 4) ? R : R + 4;
            const int LC = loop_chunk_cols_for(xt, wt, (int)RS);
            const size_t smem = loop_smem_bytes(xt, wt, (int)R, LC);
            if (LC >= 4 && smem > 0 && smem <= (size_t)loop_max_smem) {
                w.use_loop = 1;
                w.G_loop = (int)gl;
                w.R = (int)R;
                w.RS = (int)RS;
                w.LC = LC;
                w.loop_smem = smem;
            }
            // A = I: the two-barrier kernel, when its shared memory (the T block grows with d_max) fits
            const int KC = (int)round_up(d_max, 4);
            const int LCd = defer_chunk_cols(xt, (int)RS);
            const size_t smd = defer_smem_bytes(xt, (int)R, KC);
            if (w.use_loop && !wt && allow_defer && !classic_loop_forced() && LCd >= 4 && smd > 0 &&
                smd <= (size_t)loop_max_smem) {
                w.use_defer = 1;
                w.KC = KC;
                w.LC = LCd;
                w.loop_smem = smd;
            }
        }
    }
    // Largest number of CTAs sharing one column group.
    int64_t kmax = 1;
    const int64_t G = w.use_loop ? w.G_loop : w.G, W = w.W;
    for (int64_t g = 0; g < w.ngroups; ++g) {
        const int64_t u0 = g * w.NT, u1 = g * w.NT + w.NT - 1;
        const int64_t b0 = ((u0 + 1) * G + W - 1) / W - 1;
        const int64_t b1 = ((u1 + 1) * G + W - 1) / W - 1;
        kmax = std::max<int64_t>(kmax, b1 - b0 + 1);
    }
    w.KMAX = (int)kmax;
    w.RB = w.ldp / kGemvRows;
    w.LC_MAX = std::max<int64_t>(1, ceil_div(kGemvTargetCtas, w.RB));
    w.RC_MAX = std::max<int64_t>(1, w.ldp / 128);
    const double xbytes = (double)w.ldp * (double)n * w.planes_n * w.esize;
    w.evict_first = xbytes > 48.0 * 1024 * 1024 ? 1 : 0;

    // sizes
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t ldp = (size_t)w.ldp;
    size_t o_ctl = take(sizeof(Ctl));
    size_t o_rb = take((size_t)w.RB * 4);
    size_t o_lb = take((size_t)ceil_div(d_max, 8) * 4);
    size_t o_gc = take((size_t)w.ngroups * 4);
    w.zero_bytes = off;
    const bool lp = w.use_loop != 0;
    const size_t gp = (size_t)(lp ? w.G_loop : w.G);
    size_t o_planes = take((size_t)w.ngroups * (size_t)w.group_stride * w.esize);
    size_t o_yh = take(lp ? 0 : ldp * (size_t)d_max * 4);
    size_t o_yl = take(lp ? 0 : ldp * (size_t)d_max * 4);
    size_t o_ysb = take(lp ? (size_t)w.G_loop * 2 * (size_t)d_max * (size_t)w.RS * 4 : 0);
    size_t o_v1 = take(lp ? 0 : ldp * 8), o_v2 = take(lp ? 0 : ldp * 8);
    size_t o_v1h = take(lp ? 0 : ldp * 4), o_v1l = take(lp ? 0 : ldp * 4);
    size_t o_v2s = take((size_t)w.NT * 2 * w.MT * 4);
    size_t o_zs = take(lp ? (size_t)w.NT * 2 * w.MT * 4 : 0);
    size_t o_e = take((size_t)n * 8), o_xn2 = take((size_t)n * 8);
    size_t o_vpart = take(lp ? 0 : (size_t)w.LC_MAX * ldp * 8);
    size_t o_hpart = take((size_t)(lp ? w.G_loop : w.RC_MAX) * (size_t)d_max * 8);
    size_t o_h = take((size_t)d_max * 8);
    size_t o_nu2 = take((size_t)std::max<int64_t>(w.RB, lp ? 2 * (int64_t)w.G_loop : 0) * 8);
    size_t o_gslot = take((size_t)(lp ? 2 : 1) * (size_t)w.ngroups * (size_t)w.KMAX * (size_t)w.C * 8);
    size_t o_gsum = take((size_t)(w.use_defer ? 2 : 1) * (size_t)w.ngroups * 8);
    size_t o_tf = take(w.use_defer ? (size_t)w.ngroups * (size_t)d_max * (size_t)w.C * 4 : 0);
    size_t o_pbe = take(gp * 8), o_pbj = take(gp * 8);
    w.total_bytes = off;
    // stash offsets in the pointer fields (carve_work rebases them)
    w.ctl = (Ctl*)o_ctl;
    w.rb_cnt = (uint32_t*)o_rb;
    w.lb_cnt = (uint32_t*)o_lb;
    w.gcnt = (uint32_t*)o_gc;
    w.planes = (void*)o_planes;
    w.yh = (float*)o_yh;
    w.yl = (float*)o_yl;
    w.ysb = (float*)o_ysb;
    w.v1 = (double*)o_v1;
    w.v2 = (double*)o_v2;
    w.v1h = (float*)o_v1h;
    w.v1l = (float*)o_v1l;
    w.v2s = (float*)o_v2s;
    w.zs = (float*)o_zs;
    w.e = (double*)o_e;
    w.xn2 = (double*)o_xn2;
    w.vpart = (double*)o_vpart;
    w.hpart = (double*)o_hpart;
    w.h = (double*)o_h;
    w.nu2part = (double*)o_nu2;
    w.gslot = (double*)o_gslot;
    w.gsum = (double*)o_gsum;
    w.tf = (float*)o_tf;
    w.pbest_e = (double*)o_pbe;
    w.pbest_j = (int64_t*)o_pbj;
    return true;
}

void carve_work(Work& w, void* base) {
    unsigned char* b = (unsigned char*)base;
    w.base = b;
#define RB_REBASE(f) w.f = (decltype(w.f))(b + (size_t)w.f)
    RB_REBASE(ctl);
    RB_REBASE(rb_cnt);
    RB_REBASE(lb_cnt);
    RB_REBASE(gcnt);
    RB_REBASE(planes);
    RB_REBASE(yh);
    RB_REBASE(yl);
    RB_REBASE(ysb);
    RB_REBASE(v1);
    RB_REBASE(v2);
    RB_REBASE(v1h);
    RB_REBASE(v1l);
    RB_REBASE(v2s);
    RB_REBASE(zs);
    RB_REBASE(e);
    RB_REBASE(xn2);
    RB_REBASE(vpart);
    RB_REBASE(hpart);
    RB_REBASE(h);
    RB_REBASE(nu2part);
    RB_REBASE(gslot);
    RB_REBASE(gsum);
    RB_REBASE(tf);
    RB_REBASE(pbest_e);
    RB_REBASE(pbest_j);
#undef RB_REBASE
}

// ---------------------------------------------------------------------------------------
// Per-device state: SM count and one-time kernel attribute setup
// ---------------------------------------------------------------------------------------
static std::mutex g_dev_mu;
static DeviceState g_dev[64];

// The stepwise path (one launch per kernel per basis) can be forced with RBD_STEPWISE=1; the
// default is the persistent loop kernel whenever the device supports cooperative launches.
static bool stepwise_forced() {
    const char* v = getenv("RBD_STEPWISE");
    return v && v[0] && v[0] != '0';
}

cudaError_t device_state(DeviceState& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceState& s = g_dev[dev];
    if (!s.ready) {
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = pass_kernel_setup(s.pass_ctas_per_sm);
        if (e != cudaSuccess) return e;
        int coop = 0, optin = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (coop && optin > 0) {
            if (loop_kernel_setup(optin) == cudaSuccess && defer_kernel_setup(optin) == cudaSuccess)
                s.loop_max_smem = optin;
            else
                cudaGetLastError();
        }
        s.ready = true;
    }
    out = s;
    if (stepwise_forced()) out.loop_max_smem = 0;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------------
// Host-mapped progress slots: {steps finished, stop reason}, written by the device
// ---------------------------------------------------------------------------------------
static const int kProgressSlots = 256;
static std::mutex g_prog_mu;
static uint32_t* g_prog_host = nullptr;
static bool g_prog_failed = false;
static std::atomic<bool> g_prog_used[kProgressSlots];

static int progress_acquire(uint32_t** host, uint32_t** dev) {
    {
        std::lock_guard<std::mutex> lk(g_prog_mu);
        if (!g_prog_host && !g_prog_failed) {
            void* p = nullptr;
            if (cudaHostAlloc(&p, kProgressSlots * 16, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
                cudaGetLastError();
                g_prog_failed = true;
            } else {
                g_prog_host = (uint32_t*)p;
                for (int i = 0; i < kProgressSlots; ++i) g_prog_used[i].store(false);
            }
        }
        if (!g_prog_host) return -1;
    }
    for (int i = 0; i < kProgressSlots; ++i) {
        bool expect = false;
        if (g_prog_used[i].compare_exchange_strong(expect, true)) {
            uint32_t* h = g_prog_host + 4 * i;
            void* d = nullptr;
            if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
                cudaGetLastError();
                g_prog_used[i].store(false);
                return -1;
            }
            h[0] = 0;
            h[1] = 0;
            *host = h;
            *dev = (uint32_t*)d;
            return i;
        }
    }
    return -1;
}

static void progress_release(int slot) {
    if (slot >= 0) g_prog_used[slot].store(false);
}

// ---------------------------------------------------------------------------------------
// Profiling (CUDA events around launches, per host thread)
// ---------------------------------------------------------------------------------------
static std::atomic<int> g_profiling{0};
static std::atomic<uint64_t> g_wait_ns{0};

uint64_t wait_limit_ns(uint64_t dflt) {
    const uint64_t v = g_wait_ns.load();
    return v ? v : dflt;
}
static thread_local rbd_profile t_profile = {};

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_ready[64] = {};
}  // namespace

cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pool_ready[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&g_pool[dev], &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = kPoolKeepBytes;
            e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(g_pool[dev]);
                return e;
            }
            g_pool_ready[dev] = true;
        }
        pool = g_pool[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

rbd_status map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RBD_OK;
    if (e == cudaErrorMemoryAllocation) return RBD_ENOMEM;
    return RBD_ECUDA;
}

static bool valid_dtype(int t) { return t == RBD_F64 || t == RBD_F32 || t == RBD_BF16 || t == RBD_F32_ACC32; }


// ---------------------------------------------------------------------------------------
// The greedy loop on device buffers
// ---------------------------------------------------------------------------------------
// k0 > 0 continues a compression after k0 bases (Y, T, pivots hold them; next_pivot is the
// column the next basis uses); k0 = 0 starts from `start`.
static rbd_status compress_device(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                                  rbd_tol_mode mode, int64_t d_max, int64_t start, double* Y, int64_t ldy,
                                  double* T, int64_t ldt, int64_t* pivots, double* err, double* nu,
                                  void* workspace, size_t workspace_bytes, cudaStream_t st,
                                  rbd_result* result, int64_t k0 = 0, int64_t next_pivot = 0,
                                  const double* wts = nullptr) {
    DeviceState ds;
    cudaError_t ce = device_state(ds);
    if (ce != cudaSuccess) return map_cuda(ce);
    const bool acc32 = xt == RBD_F32_ACC32;
    xt = (rbd_dtype)storage_of((int)xt);
    Work w;
    if (!plan_work(w, m, n, ldx, d_max, (int)xt, ds.num_sms, ds.pass_ctas_per_sm[(int)xt], ds.loop_max_smem,
                   wts ? 1 : 0, mode != RBD_TOL_NONE))
        return RBD_EUNSUPPORTED;
    if (xt == RBD_BF16 && !w.use_loop) return RBD_EUNSUPPORTED;  // BF16 runs in the persistent kernel only
    if (acc32 && (!w.use_defer || wts)) return RBD_EUNSUPPORTED;  // FP32 accumulation: the two-barrier kernel
    w.acc32 = acc32 ? 1 : 0;
    if (wts && (!w.use_loop || k0 > 0)) return RBD_EUNSUPPORTED;  // the A-norm form: loop kernel, fresh runs
    w.wts = wts;

    bool own = false;
    void* ws = workspace;
    if (ws == nullptr) {
        ce = lib_malloc_async(&ws, w.total_bytes, st);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return RBD_ENOMEM;
        }
        own = true;
    } else {
        if (workspace_bytes < w.total_bytes) return RBD_ENOMEM;
        if (((uintptr_t)ws & 255u) != 0) return RBD_EINVAL;
    }
    carve_work(w, ws);

    const bool prof = g_profiling.load() != 0;
    std::vector<cudaEvent_t> evs;
    auto new_event = [&]() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return (cudaEvent_t) nullptr;
        }
        evs.push_back(e);
        return e;
    };
    cudaEvent_t ev_init0 = nullptr, ev_init1 = nullptr;
    std::vector<cudaEvent_t> ev_o0, ev_o1, ev_p1;
    if (prof) {
        ev_init0 = new_event();
        ev_init1 = new_event();
    }

    uint32_t *prog_h = nullptr, *prog_d = nullptr;
    const int slot = progress_acquire(&prog_h, &prog_d);

    int32_t launches = 0;
    rbd_status rs = RBD_OK;
    ce = cudaMemsetAsync(ws, 0, w.zero_bytes, st);
    if (ce == cudaSuccess && prof) cudaEventRecord(ev_init0, st);
    if (ce == cudaSuccess) {
        ce = launch_init(w, X, tol, (int)mode, start, st);
        ++launches;
    }
    if (ce == cudaSuccess && k0 > 0) {
        ce = launch_resume(w, Y, ldy, T, ldt, pivots, k0, next_pivot, st);
        launches += 3;
    }
    if (ce == cudaSuccess && prof) cudaEventRecord(ev_init1, st);

    cudaEvent_t ev_loop0 = nullptr, ev_loop1 = nullptr;
    if (w.use_loop && ce == cudaSuccess) {
        // the whole greedy loop in one cooperative launch
        if (prof) {
            ev_loop0 = new_event();
            ev_loop1 = new_event();
            cudaEventRecord(ev_loop0, st);
        }
        ce = w.use_defer ? launch_defer(w, X, Y, ldy, T, ldt, pivots, err, nu, k0, st)
                         : launch_loop(w, X, Y, ldy, T, ldt, pivots, err, nu, k0, st);
        ++launches;
        if (prof) cudaEventRecord(ev_loop1, st);
    }
    // stepwise path: orthogonalisation steps k = 0..d_max (the last one only certifies E_cur of
    // basis d_max - 1 and takes the final stop decision); passes k = 0..d_max-1
    if (prog_h) prog_h[0] = (uint32_t)k0;
    for (int64_t k = k0; !w.use_loop && k <= d_max && ce == cudaSuccess; ++k) {
        if (prog_h && k >= kLookahead) {
            // stay at most kLookahead steps ahead of the device; stop launching once it stopped
            volatile uint32_t* pr = prog_h;
            auto t0 = std::chrono::steady_clock::now();
            uint64_t spins = 0;
            bool stopped = false;
            while (true) {
                if (pr[1] != 0) {
                    stopped = true;
                    break;
                }
                if ((int64_t)pr[0] >= k - kLookahead + 1) break;
                if ((++spins & 1023) == 0) {
                    const cudaError_t q = cudaStreamQuery(st);
                    if (q == cudaSuccess) {
                        // everything enqueued has finished without publishing progress:
                        // the device stopped (or failed) inside a step
                        if (pr[1] != 0 || (int64_t)pr[0] < k - kLookahead + 1) stopped = true;
                        break;
                    }
                    if (q != cudaErrorNotReady) {
                        ce = q;
                        break;
                    }
                    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(120)) {
                        rs = RBD_ETIMEOUT;
                        stopped = true;
                        break;
                    }
                    std::this_thread::yield();
                }
            }
            if (ce != cudaSuccess || stopped) break;
        }
        if (prof) {
            ev_o0.push_back(new_event());
            cudaEventRecord(ev_o0.back(), st);
        }
        ce = launch_orth_a1(w, X, T, ldt, k, st);
        ++launches;
        if (ce == cudaSuccess && k > 0) {
            ce = launch_orth_a2(w, k, st);
            ++launches;
        }
        if (ce == cudaSuccess) {
            ce = launch_orth_c(w, k, pivots, nu, err, prog_d, st);
            ++launches;
        }
        if (prof) {
            ev_o1.push_back(new_event());
            cudaEventRecord(ev_o1.back(), st);
        }
        if (k == d_max) break;
        if (ce == cudaSuccess) {
            ce = launch_pass(w, Y, ldy, T, ldt, k, prog_d, st);
            ++launches;
        }
        if (prof) {
            ev_p1.push_back(new_event());
            cudaEventRecord(ev_p1.back(), st);
        }
    }

    Ctl hctl;
    memset(&hctl, 0, sizeof(hctl));
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (own) {
        cudaError_t fe = cudaFreeAsync(ws, st);
        if (ce == cudaSuccess) ce = fe;
    }
    cudaError_t se = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = se;
    progress_release(slot);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        for (auto e : evs) cudaEventDestroy(e);
        return map_cuda(ce);
    }
    if (rs == RBD_OK && hctl.status != ST_OK) rs = (rbd_status)hctl.status;

    if (prof) {
        rbd_profile pf = {};
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev_init0, ev_init1) == cudaSuccess) pf.init_ms = ms;
        const int64_t dd = hctl.d;
        for (size_t k = 0; k < ev_o1.size(); ++k) {
            if ((int64_t)k <= dd && cudaEventElapsedTime(&ms, ev_o0[k], ev_o1[k]) == cudaSuccess) {
                pf.orth_ms += ms;
                pf.orth_launches += (k > 0) ? 3 : 2;
            }
            const bool ran_pass = (int64_t)k < dd && k < ev_p1.size();
            if (ran_pass && cudaEventElapsedTime(&ms, ev_o1[k], ev_p1[k]) == cudaSuccess) {
                pf.pass_ms += ms;
                pf.pass_launches += 1;
            }
        }
        if (ev_loop0 && cudaEventElapsedTime(&ms, ev_loop0, ev_loop1) == cudaSuccess) {
            pf.loop_ms = ms;
            pf.loop_launches = 1;
            pf.pass_launches = dd;  // fused passes executed inside the loop kernel
        }
        pf.pass_bytes = pf.pass_launches * m * n * elem_bytes((int)xt);
        pf.loop_kernel = w.use_loop;
        cudaGetLastError();
        t_profile = pf;
    }
    for (auto e : evs) cudaEventDestroy(e);

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

rbd_status validate(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol, rbd_tol_mode mode,
                    int64_t d_max, int64_t start, const double* Y, int64_t ldy, const double* T, int64_t ldt,
                    const int64_t* pivots, const double* err) {
    if (!X || !Y || !T || !pivots || !err) return RBD_EINVAL;
    if (!valid_dtype((int)xt)) return RBD_EINVAL;
    if (m < 1 || n < 1 || ldx < m || ldy < m || d_max < 1 || ldt < d_max) return RBD_EINVAL;
    if (d_max > m || d_max > n) return RBD_EINVAL;
    if (start < 0 || start >= n) return RBD_EINVAL;
    if (!(tol >= 0.0) || tol == __builtin_inf()) return RBD_EINVAL;
    if (mode != RBD_TOL_MAXCOL_ABS && mode != RBD_TOL_MAXCOL_REL && mode != RBD_TOL_FRO_REL && mode != RBD_TOL_NONE)
        return RBD_EINVAL;
    if (m > (int64_t(1) << 40) || n > (int64_t(1) << 40)) return RBD_EUNSUPPORTED;
    return RBD_OK;
}

}  // namespace rbd

using namespace rbd;

extern "C" {

size_t rbd_compress_workspace_bytes(int64_t m, int64_t n, int64_t d_max, rbd_dtype xt) {
    if (m < 1 || n < 1 || d_max < 1 || d_max > m || d_max > n || !valid_dtype((int)xt)) return 0;
    xt = (rbd_dtype)storage_of((int)xt);
    DeviceState ds;
    if (device_state(ds) != cudaSuccess) {
        // no device: the larger of the two paths' needs, planned for a 160-SM part
        cudaGetLastError();
        Work a, b;
        if (!plan_work(a, m, n, m, d_max, (int)xt, 160, RBD_PASS_MINB, 232448)) return 0;
        if (!plan_work(b, m, n, m, d_max, (int)xt, 160, RBD_PASS_MINB, 0)) return 0;
        return std::max(a.total_bytes, b.total_bytes);
    }
    Work w;
    if (!plan_work(w, m, n, m, d_max, (int)xt, ds.num_sms, ds.pass_ctas_per_sm[(int)xt], ds.loop_max_smem)) return 0;
    return w.total_bytes;
}

rbd_status rbd_compress(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                        rbd_tol_mode mode, int64_t d_max, int64_t start, double* Y, int64_t ldy, double* T,
                        int64_t ldt, int64_t* pivots, double* err, double* nu, void* workspace,
                        size_t workspace_bytes, void* stream, rbd_result* result) {
    rbd_status v = validate(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    return compress_device(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err, nu,
                           workspace, workspace_bytes, (cudaStream_t)stream, result);
}

rbd_status rbd_compress_weighted(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, const double* w,
                                 double tol, rbd_tol_mode mode, int64_t d_max, int64_t start, double* Y, int64_t ldy,
                                 double* T, int64_t ldt, int64_t* pivots, double* err, double* nu, void* workspace,
                                 size_t workspace_bytes, void* stream, rbd_result* result) {
    rbd_status v = validate(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    if (!w || ((uintptr_t)w & 7u) != 0) return RBD_EINVAL;
    return compress_device(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err, nu,
                           workspace, workspace_bytes, (cudaStream_t)stream, result, 0, 0, w);
}

rbd_status rbd_compress_resume(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                               rbd_tol_mode mode, int64_t d0, int64_t next_pivot, int64_t d_max, double* Y,
                               int64_t ldy, double* T, int64_t ldt, int64_t* pivots, double* err, double* nu,
                               void* workspace, size_t workspace_bytes, void* stream, rbd_result* result) {
    rbd_status v = validate(X, xt, m, n, ldx, tol, mode, d_max, 0, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    if (d0 < 1 || d0 > d_max || next_pivot < 0 || next_pivot >= n) return RBD_EINVAL;
    return compress_device(X, xt, m, n, ldx, tol, mode, d_max, next_pivot, Y, ldy, T, ldt, pivots, err, nu,
                           workspace, workspace_bytes, (cudaStream_t)stream, result, d0, next_pivot);
}

rbd_status rbd_compress_rows(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                             rbd_tol_mode mode, int64_t d_max, int64_t start, double* Y, int64_t ldy, double* T,
                             int64_t ldt, int64_t* pivots, double* err, double* nu, void* stream,
                             rbd_result* result) {
    // the problem on X' (n x m): its columns are the rows of X
    if (!X || m < 1 || n < 1 || ldx < m) return RBD_EINVAL;
    rbd_status v = validate(X, xt, n, m, n, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    DeviceState ds;
    cudaError_t ce = device_state(ds);
    if (ce != cudaSuccess) return map_cuda(ce);
    cudaStream_t st = (cudaStream_t)stream;
    const int es = elem_bytes((int)xt);
    void* Xt = nullptr;
    ce = lib_malloc_async(&Xt, (size_t)m * (size_t)n * es, st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return RBD_ENOMEM;
    }
    rbd_status rs = RBD_OK;
    ce = launch_transpose(X, es, m, n, ldx, Xt, ds.num_sms, st);
    if (ce == cudaSuccess)
        rs = compress_device(Xt, xt, n, m, n, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err, nu, nullptr, 0,
                             st, result);
    cudaError_t fe = cudaFreeAsync(Xt, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(ce);
    }
    if (result && rs == RBD_OK) result->launches += 1;
    return rs;
}

rbd_status rbd_compress_host(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol,
                             rbd_tol_mode mode, int64_t d_max, int64_t start, double* Y, int64_t ldy,
                             double* T, int64_t ldt, int64_t* pivots, double* err, double* nu, void* stream,
                             rbd_result* result) {
    rbd_status v = validate(X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err);
    if (v != RBD_OK) return v;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = (size_t)elem_bytes((int)xt);
    // device copies: X with its leading dimension m, outputs with compact leading dimensions
    void *dX = nullptr, *dY = nullptr, *dT = nullptr, *dP = nullptr, *dE = nullptr, *dN = nullptr;
    cudaError_t ce = lib_malloc_async(&dX, (size_t)m * n * es, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dY, (size_t)m * d_max * 8, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dT, (size_t)d_max * n * 8, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dP, (size_t)d_max * 8, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dE, (size_t)d_max * 8, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dN, (size_t)d_max * 8, st);
    rbd_status rs = RBD_OK;
    rbd_result res = {};
    if (ce == cudaSuccess)
        ce = cudaMemcpy2DAsync(dX, (size_t)m * es, X, (size_t)ldx * es, (size_t)m * es, (size_t)n,
                               cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) {
        rs = compress_device(dX, xt, m, n, m, tol, mode, d_max, start, (double*)dY, m, (double*)dT, d_max,
                             (int64_t*)dP, (double*)dE, (double*)dN, nullptr, 0, st, &res);
        if (rs == RBD_OK && res.d > 0) {
            const int64_t d = res.d;
            ce = cudaMemcpy2DAsync(Y, (size_t)ldy * 8, dY, (size_t)m * 8, (size_t)m * 8, (size_t)d,
                                   cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpy2DAsync(T, (size_t)ldt * 8, dT, (size_t)d_max * 8, (size_t)d * 8, (size_t)n,
                                       cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(pivots, dP, (size_t)d * 8, cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(err, dE, (size_t)d * 8, cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess && nu) ce = cudaMemcpyAsync(nu, dN, (size_t)d * 8, cudaMemcpyDeviceToHost, st);
        }
    }
    void* bufs[6] = {dX, dY, dT, dP, dE, dN};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return map_cuda(ce);
    }
    if (result) *result = res;
    return rs;
}

rbd_status rbd_project(const double* Y, int64_t m, int64_t d, int64_t ldy, const void* V, rbd_dtype vt, int64_t k,
                       int64_t ldv, double* C, int64_t ldc, void* stream) {
    if (m < 1 || d < 0 || k < 0 || !valid_dtype((int)vt)) return RBD_EINVAL;
    if (d == 0 || k == 0) return RBD_OK;
    if (!Y || !V || !C || ldy < m || ldv < m || ldc < d) return RBD_EINVAL;
    if (d > (int64_t(1) << 30) || k > (int64_t(1) << 30)) return RBD_EUNSUPPORTED;
    cudaError_t ce = launch_project(Y, m, d, ldy, V, (int)vt, k, ldv, C, ldc, (cudaStream_t)stream);
    return map_cuda(ce);
}

rbd_status rbd_reconstruct(const double* Y, int64_t m, int64_t d, int64_t ldy, const double* T, int64_t n,
                           int64_t ldt, double* Xr, int64_t ldxr, void* stream) {
    if (m < 1 || d < 0 || n < 0) return RBD_EINVAL;
    if (n == 0) return RBD_OK;
    if (!Xr || ldxr < m) return RBD_EINVAL;
    if (d > 0 && (!Y || !T || ldy < m || ldt < d)) return RBD_EINVAL;
    if (m > (int64_t(1) << 40) || n > (int64_t(1) << 31) || d > (int64_t(1) << 30)) return RBD_EUNSUPPORTED;
    if (ceil_div(m, (int64_t)64) > (int64_t(1) << 31) - 1) return RBD_EUNSUPPORTED;
    return map_cuda(launch_reconstruct(Y, m, d, ldy, T, n, ldt, Xr, ldxr, (cudaStream_t)stream));
}

void rbd_set_profiling(int enabled) { g_profiling.store(enabled ? 1 : 0); }

uint64_t rbd_set_wait_limit(uint64_t ns) { return g_wait_ns.exchange(ns); }

rbd_status rbd_get_profile(rbd_profile* out) {
    if (!out) return RBD_EINVAL;
    *out = t_profile;
    return RBD_OK;
}

const char* rbd_status_string(rbd_status s) {
    switch (s) {
        case RBD_OK: return "ok";
        case RBD_EINVAL: return "invalid argument";
        case RBD_ENOMEM: return "out of memory or workspace too small";
        case RBD_ECUDA: return "CUDA runtime error";
        case RBD_ENONFINITE: return "input holds NaN or Inf";
        case RBD_ETIMEOUT: return "a bounded device wait ran out";
        case RBD_EUNSUPPORTED: return "unsupported value or shape";
    }
    return "unknown status";
}

int rbd_version(void) { return 100; }

}  // extern "C"
