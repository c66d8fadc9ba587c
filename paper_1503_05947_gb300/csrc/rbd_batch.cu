// rbd_batch.cu -- the batched form: many independent matrices, each compressed by Algorithm 1,
// in one persistent cooperative launch.
//
// batch_init_kernel  the initial pass over every matrix (Section 3.3's pre-computation with
//                    A = I): e_j = ||x_j||^2 and the tile-major re-layout of X, one warp per
//                    column of the whole batch.
// batch_kernel       one CTA per SM.  The plan gives each matrix a TEAM of t CTAs (t = 1 for most;
//                    large matrices get up to 16 so that no single matrix outlasts the batch) and
//                    lays the matrices' member slots out in a queue ordered by decreasing size; a
//                    CTA claims the next slot and works as that member until the matrix stops:
//                      step 2.1-2.2  v1 = x_i - Y t (t = T(0:k, i)), h = Y' v1, v2 = v1 - Y h
//                                    (classical Gram-Schmidt twice, float-float) on the member's
//                                    block of rows; partial sums of h and ||v2||^2 and the rows of
//                                    v2 are exchanged through the matrix's team buffers; nu, stop
//                                    tests (identical in every member); xi = v2 / nu
//                      fused pass    the member's column groups: T(k, j) = xi' x_j,
//                                    e_j <- e_j - T(k, j)^2 (Eq. (evalerr), A = I), argmax, then
//                                    the team's argmax and Frobenius residual
//                    Three team barriers per basis (none when t = 1).  The members' row blocks of Y
//                    (split FP32 planes) and the X tiles stream through one ring of shared-memory
//                    stages with bulk (TMA) copies; xi stays in shared memory for the whole pass.
// The launch is cooperative (all CTAs resident), and slots are claimed in order, so a member only
// ever waits for members of its own team whose slots come before any later-claimed work: every team
// ahead of it is complete and finishes, freeing the CTAs that claim the remaining slots.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/rbd.h"
#include "rbd_device.cuh"
#include "rbd_tile.cuh"
#include "rbd_work.h"

namespace rbd {

namespace {

constexpr int kBNW = 8;                      // consumer warps
constexpr int kBNCONS = kBNW * 32;
constexpr int kBThreads = kBNCONS + 32;      // + producer warp
constexpr int kBMaxRows = 4096;              // padded rows per matrix
constexpr int kBMaxD = 512;
constexpr int kBQR = kBMaxRows / kBNCONS;    // rows per consumer thread
constexpr int kBRingBytes = 128 * 1024;
constexpr int kBMaxLC = 64;                  // Y columns per Gram-Schmidt chunk
constexpr int kBNB = 2;                      // Y chunk buffers (the ring in halves)

// Launch shape of the fused pass: CPW columns per consumer warp (a column group of C = 8 CPW
// columns) and MT rows per tile; both are chosen per plan (rbd_batch_config, the autotuner).
template <int P, int CPW, int MT>
struct BCfg {
    static constexpr int C = kBNW * CPW;
    static constexpr int STAGE_BYTES = C * P * MT * 4;
    static constexpr int SMAX = kBRingBytes / STAGE_BYTES;
    static_assert(MT % 128 == 0 && SMAX >= 2 && SMAX <= 32, "ring of 2..32 stages");
};

// Device descriptor of one matrix (built on the host, uploaded by plan_create).
struct BInst {
    const void* X;
    int64_t m, n, ldx, ldp, ngroups, NT;
    double tol;
    int32_t mode, team;   // team: CTAs working on this matrix
    int64_t d_max, start;
    double* Y;
    int64_t ldy;
    double* T;
    int64_t ldt;
    int64_t* piv;
    double* err;
    double* nu;
    float* planes;   // tile-major, as in rbd_work.h
    float* ys;       // split Y, one block of rb rows per member: [team][2][d_max][rb]
    int64_t rb;      // rows per member block (team * rb >= ldp)
    double* e;
    double* xn2;
    // team exchange (team > 1)
    uint32_t* bar;   // team barrier arrivals (zero before the run)
    double* hpart;   // [team][d_max]
    double* nrm;     // [team]
    float* vbuf;     // [2][ldp] rows of v2 (hi | lo)
    double* cand_e;  // [team]
    int64_t* cand_j; // [team]
    double* frop;    // [team]
};

struct BatchParams {
    const BInst* inst;
    int64_t count;
    int64_t nslots;
    const int32_t* slot_inst;    // claim slot -> matrix
    const int32_t* slot_member;  // claim slot -> member index in the matrix's team
    const int64_t* colstart;     // padded-column prefix sums (count + 1)
    uint32_t* queue;             // claim counter (zero before the run)
    int32_t* status;             // per matrix (zero before the run)
    rbd_batch_result* res;
    int S;                       // ring stages used by the pass (<= SMAX)
    int C, MT;                   // the plan's column-group width and tile rows (initial pass)
    uint64_t wait_ns;            // bound on a ring or Y-chunk wait (the exit drain keeps kWaitLimitNs)
    uint64_t team_ns;            // bound on a team barrier
};

constexpr uint64_t kTeamWaitNs = 10000000000ull;  // a member may wait for teams ahead to finish

__device__ __forceinline__ uint32_t ld_acquire_u32b(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------- initial pass
template <int P>
__global__ void __launch_bounds__(256) batch_init_kernel(BatchParams bp) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = bp.colstart[bp.count];
    for (int64_t q = gw; q < total; q += nw) {
        // matrix of padded column q: last i with colstart[i] <= q
        int64_t lo = 0, hi = bp.count - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (bp.colstart[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        // the fields this loop needs, in registers (the plane stores could alias the table)
        const BInst& Ig = bp.inst[lo];
        const void* IX = Ig.X;
        const int64_t Im = Ig.m, In = Ig.n, Ildx = Ig.ldx, Ildp = Ig.ldp;
        float* Iplanes = Ig.planes;
        double* Ie = Ig.e;
        double* Ixn2 = Ig.xn2;
        const int64_t j = q - bp.colstart[lo];
        const int64_t C = bp.C, MT = bp.MT;
        const int64_t g = j / C;
        const int c = (int)(j % C);
        const bool live = j < In;
        float s = 0.f, cc = 0.f;
        int bad = ST_OK;
        for (int64_t r0 = 4 * lane; r0 < Ildp; r0 += 128) {
            const int64_t t = r0 / MT;
            const int64_t rt = min(MT, Ildp - t * MT);
            const int64_t base = g * C * P * Ildp + t * C * P * MT + (int64_t)c * P * rt + (r0 - t * MT);
            float hv[4], lv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t r = r0 + u;
                // finiteness and range on the exponent bits (integer tests; the FP64 pipe is slow)
                if constexpr (P == 2) {
                    double x = (live && r < Im) ? ((const double*)IX)[j * Ildx + r] : 0.0;
                    const uint32_t ex = (uint32_t)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ffu);
                    if (ex == 0x7ffu) {
                        bad = ST_ENONFINITE;
                        x = 0.0;
                    } else if (ex >= 1150u && bad == ST_OK) {
                        bad = ST_EUNSUPPORTED;  // |x| >= 2^127
                    }
                    split_f64_fast(x, hv[u], lv[u]);
                    ff_mac2(s, cc, hv[u], lv[u], hv[u], lv[u]);
                } else {
                    float x = (live && r < Im) ? ((const float*)IX)[j * Ildx + r] : 0.f;
                    if ((__float_as_uint(x) & 0x7f800000u) == 0x7f800000u) {
                        bad = ST_ENONFINITE;
                        x = 0.f;
                    }
                    hv[u] = x;
                    lv[u] = 0.f;
                    ff_mac1(s, cc, x, x, 0.f);
                }
            }
            float* ph = Iplanes + base;
            *reinterpret_cast<float4*>(ph) = make_float4(hv[0], hv[1], hv[2], hv[3]);
            if (P == 2) *reinterpret_cast<float4*>(ph + rt) = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
        const double tsum = warp_sum_double(ff_to_double(s, cc));
        const int anybad = __reduce_max_sync(0xffffffffu, bad);
        if (lane == 0) {
            if (live) {
                Ie[j] = tsum;
                Ixn2[j] = tsum;
            }
            if (anybad != ST_OK) atomicCAS(&bp.status[lo], 0, anybad);
        }
    }
}

// ---------------------------------------------------------------- the per-matrix loop
template <int P, int CPW, int MT>
__global__ void __launch_bounds__(kBThreads, 1) batch_kernel(BatchParams bp) {
    using Cfg = BCfg<P, CPW, MT>;
    constexpr int C = Cfg::C;
    constexpr int SMAX = Cfg::SMAX;
    constexpr int STAGE_F = Cfg::STAGE_BYTES / 4;
    extern __shared__ __align__(128) unsigned char bsm[];
    float* ring = reinterpret_cast<float*>(bsm);                               // kBRingBytes
    uint64_t* full = reinterpret_cast<uint64_t*>(bsm + kBRingBytes);           // SMAX
    uint64_t* empty = full + SMAX;                                             // SMAX
    uint64_t* ybar = empty + SMAX;                                             // kBNB: chunk landed
    uint64_t* yempty = ybar + kBNB;                                            // kBNB: chunk consumed
    float* vh = reinterpret_cast<float*>(yempty + kBNB);                       // kBMaxRows
    float* vl = vh + kBMaxRows;                                                // kBMaxRows
    double* hacc = reinterpret_cast<double*>(vl + kBMaxRows);                  // kBMaxD
    float* cst_h = reinterpret_cast<float*>(hacc + kBMaxD);                    // kBMaxD: coefficients (hi)
    float* cst_l = cst_h + kBMaxD;                                             // kBMaxD: (lo)
    float* wps = cst_l + kBMaxD;                                               // kBNW x kBMaxD (ff hi)
    float* wpc = wps + kBNW * kBMaxD;                                          // (ff lo)
    double* red = reinterpret_cast<double*>(wpc + kBNW * kBMaxD);              // 4 kBNW + 16
    int64_t* redj = reinterpret_cast<int64_t*>(red + 2 * kBNW);
    double* bc = red + 4 * kBNW;                                               // broadcasts
    int* flag = reinterpret_cast<int*>(bc + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = bp.S;

    if (tid == 0) {
        for (int s = 0; s < SMAX; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kBNW);
        }
        for (int bq = 0; bq < kBNB; ++bq) {
            mbar_init(&ybar[bq], 1);
            mbar_init(&yempty[bq], kBNW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    bool ok = true;
    uint32_t ycount = 0;          // Y chunks streamed so far (buffer and parity of each)
    uint32_t yiss = 0, ywait = 0; // thread 0: chunks issued / waited (those in between are landing)
    uint32_t iss_par = 0, iss_mask = 0;  // producer: parity and presence of the last issue per stage
    int ps = 0, cs = 0;           // pass ring: producer / consumer stage and phase
    uint32_t pph = 0, cph = 0;
    bool preuse = false;
    const uint64_t pol_x = l2_policy_evict_first();
    const uint64_t pol_y = l2_policy_evict_normal();

    for (;;) {
        if (tid == 0) flag[0] = (int)atomicAdd(bp.queue, 1u);
        __syncthreads();
        const int64_t slot = flag[0];
        __syncthreads();
        if (slot >= bp.nslots) break;
        const int64_t idx = bp.slot_inst[slot];
        const int mb = bp.slot_member[slot];
        const BInst I = bp.inst[idx];
        const int tm = I.team;
        const int64_t m = I.m, n = I.n, ldp = I.ldp, dmax = I.d_max, NT = I.NT, rb = I.rb;
        const int64_t r_lo = (int64_t)mb * rb, r_hi = min(ldp, r_lo + rb);  // this member's rows
        const int64_t g_lo = (I.ngroups * mb) / tm, g_hi = (I.ngroups * (mb + 1)) / tm;  // its groups
        const int64_t W = (g_hi - g_lo) * NT;
        const float* ysb = I.ys + (int64_t)mb * 2 * dmax * rb;  // this member's block of Y
        uint32_t tepoch = 0;

        // team barrier: every thread of every member; false if the wait ran out
        auto team_sync = [&]() {
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const uint32_t target = (uint32_t)tm * (++tepoch);
                atomicAdd(I.bar, 1u);
                int good = 1;
                if (ld_acquire_u32b(I.bar) < target) {
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_acquire_u32b(I.bar) < target) {
                        if (globaltimer_ns() - t0 > bp.team_ns) {
                            good = 0;
                            break;
                        }
                    }
                }
                flag[2] = good;
            }
            __syncthreads();
            if (!flag[2]) ok = false;
        };

        // ---- statistics of the initial pass and the tolerances (fixed order; every member)
        if (warp == 0) {
            double sum = 0.0, mx = 0.0;
            for (int64_t j = lane; j < n; j += 32) {
                const double v = __ldcg(&I.xn2[j]);
                sum += v;
                mx = fmax(mx, v);
            }
            sum = warp_sum_double(sum);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
            if (lane == 0) {
                bc[0] = sqrt(sum);
                bc[1] = sqrt(mx);
            }
        }
        __syncthreads();
        const double x_fro = bc[0], x_maxcol = bc[1];
        const int st0 = __ldcg(&bp.status[idx]);
        double fro_tol = -1.0, eps_r, eps_r22;
        if (I.mode == MODE_FRO_REL) {
            fro_tol = I.tol * x_fro;
            eps_r = -1.0;
            eps_r22 = I.tol * x_fro / sqrt((double)n);
        } else {
            eps_r = (I.mode == MODE_MAXCOL_REL) ? I.tol * x_maxcol : I.tol;
            eps_r22 = eps_r;
        }
        int64_t piv = I.start;
        double fro_prev = x_fro, err_last = 0.0;
        int32_t stop = (st0 != ST_OK) ? STOP_BREAK : STOP_NONE;
        int64_t k = 0;
        // Y chunk geometry: the ring as kBNB buffers, both planes per chunk
        const int64_t buf_f = kBRingBytes / 4 / kBNB;  // floats per buffer
        const int LC = (int)max((int64_t)1, min((int64_t)kBMaxLC, buf_f / (2 * rb)));

        // streams columns [0, k) of this member's Y block in chunks through the ring buffers, up
        // to kBNB in flight (consumer threads); stage(l, hi, lo) gives the coefficient of column l
        // (all k staged once, before the first chunk), body(yh, yl, ch, cl, l0, lc) runs on the
        // chunk.  No barrier per chunk: each consumer warp marks a chunk consumed on the buffer's
        // yempty barrier, and thread 0 waits there (for the buffer's previous chunk) before it
        // refills a buffer.  Every consumer warp arrives whatever its waits returned.
        auto ystream = [&](auto&& stage, auto&& body) {
            const int64_t nch = ceil_div(k, (int64_t)LC);
            auto issue = [&](int64_t c) {
                const uint32_t gc = ycount + (uint32_t)c;
                const int bf = (int)(gc % (uint32_t)kBNB);
                if (gc >= (uint32_t)kBNB && ok && !mbar_wait(&yempty[bf], (gc / (uint32_t)kBNB - 1u) & 1u, bp.wait_ns))
                    ok = false;
                if (!ok) return;
                const int64_t l0 = c * LC;
                const int lc = (int)min((int64_t)LC, k - l0);
                const uint32_t bytes = (uint32_t)(lc * rb * 4);
                yiss = max(yiss, gc + 1u);
                mbar_arrive_expect_tx(&ybar[bf], 2u * bytes);
                bulk_g2s(ring + bf * buf_f, ysb + l0 * rb, bytes, &ybar[bf], pol_y);
                bulk_g2s(ring + bf * buf_f + (int64_t)LC * rb, ysb + (dmax + l0) * rb, bytes, &ybar[bf], pol_y);
            };
            if (tid == 0)
                for (int64_t c = 0; c < min(nch, (int64_t)kBNB); ++c) issue(c);
            for (int64_t l = tid; l < k; l += kBNCONS) stage(l, cst_h[l], cst_l[l]);
            named_bar(1, kBNCONS);  // coefficients visible
            for (int64_t c = 0; c < nch; ++c) {
                const int bf = (int)((ycount + (uint32_t)c) % (uint32_t)kBNB);
                const int64_t l0 = c * LC;
                const int lc = (int)min((int64_t)LC, k - l0);
                const uint32_t par = ((ycount + (uint32_t)c) / (uint32_t)kBNB) & 1u;
                if (ok) {
                    if (mbar_wait(&ybar[bf], par, bp.wait_ns)) ywait = max(ywait, ycount + (uint32_t)c + 1u);
                    else ok = false;
                }
                if (ok) body(ring + bf * buf_f, ring + bf * buf_f + (int64_t)LC * rb, cst_h + l0, cst_l + l0, l0, lc);
                __syncwarp();
                if (lane == 0) mbar_arrive(&yempty[bf]);  // this warp is done with chunk c
                if (tid == 0 && c + kBNB < nch) issue(c + kBNB);
            }
            ycount += (uint32_t)nch;
        };

        while (stop == STOP_NONE && ok) {
            if (warp < kBNW) {
                // ---- O1: v1 = x_i - Y t for this member's rows (tid + kBNCONS q)
                float as[kBQR], ac[kBQR];
#pragma unroll
                for (int q = 0; q < kBQR; ++q) as[q] = ac[q] = 0.f;
                const double* tcol = I.T + piv * I.ldt;
                if (k > 0)
                    ystream([&](int64_t l, float& hi, float& lo) { split_double(__ldcg(&tcol[l]), hi, lo); },
                            [&](const float* yh, const float* yl, const float* ch, const float* cl, int64_t, int lc) {
#pragma unroll
                                for (int q = 0; q < kBQR; ++q) {
                                    const int64_t rr = tid + (int64_t)kBNCONS * q;
                                    if (r_lo + rr >= r_hi) break;
                                    for (int l = 0; l < lc; ++l)
                                        ff_mac2(as[q], ac[q], yh[l * rb + rr], yl[l * rb + rr], ch[l], cl[l]);
                                }
                            });
#pragma unroll
                for (int q = 0; q < kBQR; ++q) {
                    const int64_t r = r_lo + tid + (int64_t)kBNCONS * q;
                    if (r >= r_hi) break;
                    // v1 = x - Y t in float-float on the FP32 pipes (the FP64 pipe runs at 1/64 rate)
                    float xh = 0.f, xl = 0.f;
                    if (r < m) {
                        if constexpr (P == 2)
                            split_f64_fast(((const double*)I.X)[piv * I.ldx + r], xh, xl);
                        else
                            xh = ((const float*)I.X)[piv * I.ldx + r];
                        ff_add_acc(xh, xl, -as[q], -ac[q]);
                    }
                    vh[r] = xh;
                    vl[r] = xl;
                }
                named_bar(1, kBNCONS);
                // ---- O1': h_l = Y(:, l)' v1 over this member's rows (per-warp float-float sums,
                //      warps in order)
                if (k > 0) {
                    ystream([&](int64_t, float& hi, float& lo) { hi = lo = 0.f; },
                            [&](const float* yh, const float* yl, const float*, const float*, int64_t l0, int lc) {
                                for (int l = 0; l < lc; ++l) {
                                    float s = 0.f, c = 0.f;
#pragma unroll
                                    for (int q = 0; q < kBQR; ++q) {
                                        const int64_t rr = tid + (int64_t)kBNCONS * q;
                                        if (r_lo + rr >= r_hi) break;
                                        ff_mac2(s, c, yh[l * rb + rr], yl[l * rb + rr], vh[r_lo + rr], vl[r_lo + rr]);
                                    }
                                    warp_sum_ff(s, c);
                                    if (lane == 0) {
                                        wps[warp * kBMaxD + l0 + l] = s;
                                        wpc[warp * kBMaxD + l0 + l] = c;
                                    }
                                }
                            });
                    named_bar(1, kBNCONS);  // every warp's partial sums are in
                    for (int64_t l = tid; l < k; l += kBNCONS) {
                        float s = wps[l], c = wpc[l];
                        for (int w = 1; w < kBNW; ++w) ff_add(s, c, wps[w * kBMaxD + l], wpc[w * kBMaxD + l]);
                        hacc[l] = ff_to_double(s, c);
                    }
                    named_bar(1, kBNCONS);  // h is complete before anything reads it
                }
            }
            if (tm > 1 && k > 0) {
                // the team's h: every member's partial sums, added in member order
                __syncthreads();
                if (warp < kBNW)
                    for (int64_t l = tid; l < k; l += kBNCONS) I.hpart[mb * dmax + l] = hacc[l];
                team_sync();
                if (warp < kBNW)
                    for (int64_t l = tid; l < k; l += kBNCONS) {
                        double acc = 0.0;
                        for (int b2 = 0; b2 < tm; ++b2) acc += __ldcg(&I.hpart[b2 * dmax + l]);
                        hacc[l] = acc;
                    }
                __syncthreads();
            }
            if (warp < kBNW) {
                // ---- O3: v2 = v1 - Y h on this member's rows, ||v2||^2
                float as[kBQR], ac[kBQR];
#pragma unroll
                for (int q = 0; q < kBQR; ++q) as[q] = ac[q] = 0.f;
                if (k > 0)
                    ystream([&](int64_t l, float& hi, float& lo) { split_double(hacc[l], hi, lo); },
                            [&](const float* yh, const float* yl, const float* ch, const float* cl, int64_t, int lc) {
#pragma unroll
                                for (int q = 0; q < kBQR; ++q) {
                                    const int64_t rr = tid + (int64_t)kBNCONS * q;
                                    if (r_lo + rr >= r_hi) break;
                                    for (int l = 0; l < lc; ++l)
                                        ff_mac2(as[q], ac[q], yh[l * rb + rr], yl[l * rb + rr], ch[l], cl[l]);
                                }
                            });
                // v2 = v1 - Y h and ||v2||^2 in float-float (v2 replaces v1: each thread owns its rows)
                float ns = 0.f, nc = 0.f;
#pragma unroll
                for (int q = 0; q < kBQR; ++q) {
                    const int64_t r = r_lo + tid + (int64_t)kBNCONS * q;
                    if (r >= r_hi) break;
                    float wh = 0.f, wl = 0.f;
                    if (r < m) {
                        wh = vh[r];
                        wl = vl[r];
                        ff_add_acc(wh, wl, -as[q], -ac[q]);
                    }
                    vh[r] = wh;
                    vl[r] = wl;
                    if (tm > 1) {
                        I.vbuf[r] = wh;
                        I.vbuf[ldp + r] = wl;
                    }
                    ff_mac2(ns, nc, wh, wl, wh, wl);
                }
                warp_sum_ff(ns, nc);
                if (lane == 0) red[warp] = ff_to_double(ns, nc);
            }
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            if (tid == 0) {
                double acc = 0.0;
                for (int w = 0; w < kBNW; ++w) acc += red[w];
                bc[2] = acc;
                if (tm > 1) I.nrm[mb] = acc;
            }
            if (tm > 1) {
                team_sync();  // every member's rows of v2 and ||v2||^2 are out
                if (tid == 0) {
                    double acc = 0.0;
                    for (int b2 = 0; b2 < tm; ++b2) acc += __ldcg(&I.nrm[b2]);
                    bc[2] = acc;
                }
                // the other members' rows of v2
                if (warp < kBNW)
                    for (int64_t r = tid; r < ldp; r += kBNCONS)
                        if (r < r_lo || r >= r_hi) {
                            vh[r] = __ldcg(&I.vbuf[r]);
                            vl[r] = __ldcg(&I.vbuf[ldp + r]);
                        }
            }
            __syncthreads();
            // ---- nu, certified E_cur of basis k-1, stop tests of steps 2.2 / 2.4 (identical in
            //      every member; member 0 writes the outputs)
            if (tid == 0) {
                const double nuv = sqrt(bc[2]);
                const double xin = sqrt(__ldcg(&I.xn2[piv]));
                int32_t st = STOP_NONE;
                if (k > 0) {
                    if (I.mode == MODE_FRO_REL) {
                        if (fro_prev <= fro_tol) st = STOP_TOL;
                    } else if (nuv <= eps_r) {
                        st = STOP_TOL;
                    }
                }
                if (st == STOP_NONE && k >= dmax) st = STOP_DMAX;
                if (st == STOP_NONE && (nuv < eps_r22 || nuv <= kRankFloor * xin)) st = STOP_BREAK;
                if (mb == 0) {
                    if (k > 0) I.err[k - 1] = nuv;
                    if (st == STOP_NONE) {
                        I.piv[k] = piv;
                        if (I.nu) I.nu[k] = nuv;
                    }
                }
                bc[3] = nuv;
                bc[7] = recip_pos(nuv);  // once, for every thread
                flag[1] = st;
            }
            __syncthreads();
            const double nuv = bc[3];
            if (k > 0) err_last = nuv;
            stop = flag[1];
            if (stop != STOP_NONE) break;

            // ---- xi = v2 / nu: the whole vector for the pass; this member's rows of Y(:, k)
            const double inv_nu = bc[7];
            if (warp < kBNW) {
                // (vh + vl) / nu in float-float (FP64 only for this member's rows of Y), unless
                // 1 / nu is outside the FP32 range: then in FP64
                const bool ffm = inv_nu < 1e38;
                float ih = 0.f, il = 0.f;
                if (ffm) split_f64_fast(inv_nu, ih, il);
                for (int64_t r = tid; r < ldp; r += kBNCONS) {
                    double y = 0.0;
                    if (ffm) {
                        const float a = vh[r], b = vl[r];
                        const float p0 = __fmul_rn(a, ih);
                        float pe = __fmaf_rn(a, ih, -p0);
                        pe = __fmaf_rn(a, il, pe);
                        pe = __fmaf_rn(b, ih, pe);
                        fast_two_sum(p0, pe, vh[r], vl[r]);
                    } else {
                        y = ((double)vh[r] + (double)vl[r]) * inv_nu;
                        split_double(y, vh[r], vl[r]);
                    }
                    if (r >= r_lo && r < r_hi) {
                        if (r < m) I.Y[r + k * I.ldy] = ffm ? (double)vh[r] + (double)vl[r] : y;
                        I.ys[((int64_t)mb * 2 * dmax + k) * rb + (r - r_lo)] = vh[r];
                        I.ys[((int64_t)mb * 2 * dmax + dmax + k) * rb + (r - r_lo)] = vl[r];
                    }
                }
                fence_proxy_async_global();  // Y's split copy is read by bulk copies later
            }
            __syncthreads();

            // ---- the fused pass over this member's column groups
            if (warp == kBNW) {
                if (lane == 0 && ok) {
                    int64_t g = g_lo, t = 0;
                    for (int64_t u = 0; u < W; ++u) {
                        if (preuse && !mbar_wait(&empty[ps], pph ^ 1u, bp.wait_ns)) {
                            ok = false;
                            break;
                        }
                        const uint32_t rows = (uint32_t)min((int64_t)MT, ldp - t * MT);
                        const uint32_t bytes = (uint32_t)(C * P) * rows * 4u;
                        mbar_arrive_expect_tx(&full[ps], bytes);
                        bulk_g2s(ring + (size_t)ps * STAGE_F, I.planes + g * C * P * ldp + t * C * P * MT, bytes,
                                 &full[ps], pol_x);
                        iss_mask |= 1u << ps;
                        iss_par = (iss_par & ~(1u << ps)) | (pph << ps);
                        if (++ps == S) {
                            ps = 0;
                            pph ^= 1u;
                            preuse = true;
                        }
                        if (++t == NT) {
                            t = 0;
                            ++g;
                        }
                    }
                }
            } else {
                float acc_s[CPW][4], acc_c[CPW][4];
#pragma unroll
                for (int qq = 0; qq < CPW; ++qq)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc_s[qq][e] = acc_c[qq][e] = 0.f;
                // lanes 0 .. CPW-1 finalise one column each (their FP64 work runs side by side)
                double best_e = -1.0, esum = 0.0;
                int64_t best_j = INT64_MAX;
                double e_old = 0.0;
                int64_t g = g_lo, t = 0;
                for (int64_t u = 0; u < W; ++u) {
                    const int s = cs;
                    const uint32_t ph = cph;
                    if (++cs == S) {
                        cs = 0;
                        cph ^= 1u;
                    }
                    const int64_t c0 = g * C;
                    const int ncols = (int)min((int64_t)C, n - c0);
                    if (t == 0 && lane < CPW) {
                        const int cw = warp * CPW + lane;
                        e_old = (cw < ncols) ? __ldcg(&I.e[c0 + cw]) : 0.0;
                    }
                    if (ok && !mbar_wait(&full[s], ph, bp.wait_ns)) ok = false;
                    const int rows = (int)min((int64_t)MT, ldp - t * MT);
                    if (ok) {
                        const float* st = ring + (size_t)s * STAGE_F;
                        if (rows == MT)
                            consume_tile_xi<P, CPW, MT, true>(st, vh + t * MT, vl + t * MT, MT, warp, lane,
                                                                  acc_s, acc_c);
                        else
                            consume_tile_xi<P, CPW, MT, false>(st, vh + t * MT, vl + t * MT, rows, warp, lane,
                                                                   acc_s, acc_c);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    if (++t < NT) continue;
                    t = 0;
                    // end of column group g: T(k, j), e_j, the running argmax
                    // each column's total (valid in lane 0), then lane qq takes column qq
                    float my_s = 0.f, my_c = 0.f;
#pragma unroll
                    for (int qq = 0; qq < CPW; ++qq) {
                        float sq = acc_s[qq][0], cq = acc_c[qq][0];
#pragma unroll
                        for (int e = 1; e < 4; ++e) ff_add(sq, cq, acc_s[qq][e], acc_c[qq][e]);
                        warp_sum_ff(sq, cq);
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc_s[qq][e] = acc_c[qq][e] = 0.f;
                        sq = __shfl_sync(0xffffffffu, sq, 0);
                        cq = __shfl_sync(0xffffffffu, cq, 0);
                        if (lane == qq) {
                            my_s = sq;
                            my_c = cq;
                        }
                    }
                    if (lane < CPW) {
                        const int cw = warp * CPW + lane;
                        if (cw < ncols) {
                            const int64_t j = c0 + cw;
                            const double cj = ff_to_double(my_s, my_c);
                            I.T[j * I.ldt + k] = cj;
                            const double en = (j == piv) ? 0.0 : fmax(e_old - cj * cj, 0.0);
                            I.e[j] = en;
                            esum += en;
                            // en >= 0 and best_e >= 0 or -1: the order of the values is that of their
                            // bit patterns as signed integers (integer compares: the FP64 pipe is slow)
                            const long long eb = __double_as_longlong(en), bb = __double_as_longlong(best_e);
                            if (eb > bb || (eb == bb && j < best_j)) {
                                best_e = en;
                                best_j = j;
                            }
                        }
                    }
                    ++g;
                }
                {
                    // the finalising lanes' candidates and sums (a fixed tree over lanes 0 .. CPW-1)
#pragma unroll
                    for (int o = 1; o < CPW; o <<= 1) {
                        const double be1 = __shfl_xor_sync(0xffffffffu, best_e, o);
                        const int64_t bj1 = __shfl_xor_sync(0xffffffffu, best_j, o);
                        const double es1 = __shfl_xor_sync(0xffffffffu, esum, o);
                        if (better(be1, bj1, best_e, best_j)) {
                            best_e = be1;
                            best_j = bj1;
                        }
                        esum += es1;
                    }
                    if (lane == 0) {
                        red[warp] = best_e;
                        redj[warp] = best_j;
                        red[kBNW + warp] = esum;
                    }
                }
            }
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            // ---- argmax over the warps (and the team's members), Frobenius residual (fixed order)
            if (tid == 0) {
                double be = -1.0, fs = 0.0;
                int64_t bj = INT64_MAX;
                for (int w = 0; w < kBNW; ++w) {
                    if (better(red[w], redj[w], be, bj)) {
                        be = red[w];
                        bj = redj[w];
                    }
                    fs += red[kBNW + w];
                }
                bc[4] = be;
                bc[5] = fs;
                redj[kBNW] = bj;
                if (tm > 1) {
                    I.cand_e[mb] = be;
                    I.cand_j[mb] = bj;
                    I.frop[mb] = fs;
                }
            }
            if (tm > 1) {
                team_sync();
                if (tid == 0) {
                    double be = -1.0, fs = 0.0;
                    int64_t bj = INT64_MAX;
                    for (int b2 = 0; b2 < tm; ++b2) {
                        const double ce = __ldcg(&I.cand_e[b2]);
                        const int64_t cj = __ldcg(reinterpret_cast<const long long*>(&I.cand_j[b2]));
                        if (better(ce, cj, be, bj)) {
                            be = ce;
                            bj = cj;
                        }
                        fs += __ldcg(&I.frop[b2]);
                    }
                    bc[5] = fs;
                    redj[kBNW] = bj;
                }
            }
            if (tid == 0) {
                const int64_t bj = redj[kBNW];
                bc[6] = sqrt(fmax(bc[5], 0.0));
                redj[kBNW] = (bj >= 0 && bj < n) ? bj : piv;
            }
            __syncthreads();
            fro_prev = bc[6];
            piv = redj[kBNW];
            ++k;
            ok = __syncthreads_and(ok) != 0;
        }
        // ---- result of this matrix (member 0)
        if (tid == 0 && mb == 0) {
            rbd_batch_result rr;
            rr.d = k;
            rr.next_pivot = piv;
            rr.stop_reason = ok ? stop : STOP_BREAK;
            rr.status = ok ? st0 : ST_ETIMEOUT;
            rr.err_last = (k > 0) ? err_last : 0.0;
            rr.fro_last = fro_prev;
            rr.x_fro = x_fro;
            rr.x_maxcol = x_maxcol;
            bp.res[idx] = rr;
        }
        __syncthreads();
        if (!ok) break;
    }
    // No bulk copy may still be writing this CTA's shared memory when it exits (a wait that gave
    // up leaves copies in flight): these waits keep the default bound.
    if (warp == kBNW && lane == 0)
        for (int s = 0; s < SMAX; ++s)
            if ((iss_mask >> s) & 1u) mbar_wait(&full[s], (iss_par >> s) & 1u);
    if (tid == 0)
        for (uint32_t gc = ywait; gc < yiss; ++gc) mbar_wait(&ybar[gc % (uint32_t)kBNB], (gc / (uint32_t)kBNB) & 1u);
}

template <int P, int CPW, int MT>
size_t batch_smem() {
    return (size_t)kBRingBytes + (size_t)(2 * BCfg<P, CPW, MT>::SMAX + 2 * kBNB) * 8 + (size_t)2 * kBMaxRows * 4 +
           (size_t)kBMaxD * 8 + (size_t)2 * kBMaxD * 4 + (size_t)2 * kBNW * kBMaxD * 4 + (size_t)(4 * kBNW + 16) * 8;
}

}  // namespace
}  // namespace rbd

// ==================================================================== host: plans
struct rbd_batch_plan_s {
    int xt = 0;
    int64_t count = 0;
    int64_t nslots = 0;
    int S = 0;
    int cols = 16, tile_rows = 256, team_pct = 150;  // launch shape (rbd_batch_config)
    std::vector<rbd_instance> inst;                  // the caller's descriptors (re-layout)
    unsigned char* ws = nullptr;
    size_t ws_bytes = 0;
    int num_sms = 0;
    size_t smem = 0;
    int init_blocks = 0;
    rbd::BInst* d_inst = nullptr;
    int32_t* d_slot_inst = nullptr;
    int32_t* d_slot_member = nullptr;
    int64_t* d_colstart = nullptr;
    uint32_t* d_queue = nullptr;
    int32_t* d_status = nullptr;
    size_t zero_bytes = 0;  // queue, statuses and team barrier counters
};

using namespace rbd;

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

rbd_status check_inst(const rbd_instance& I, rbd_dtype xt) {
    if (!I.X || !I.Y || !I.T || !I.pivots || !I.err) return RBD_EINVAL;
    if (I.m < 1 || I.n < 1 || I.ldx < I.m || I.ldy < I.m || I.d_max < 1 || I.ldt < I.d_max) return RBD_EINVAL;
    if (I.d_max > I.m || I.d_max > I.n) return RBD_EINVAL;
    if (I.start < 0 || I.start >= I.n) return RBD_EINVAL;
    if (!(I.tol >= 0.0) || I.tol == __builtin_inf()) return RBD_EINVAL;
    if (I.mode != RBD_TOL_MAXCOL_ABS && I.mode != RBD_TOL_MAXCOL_REL && I.mode != RBD_TOL_FRO_REL) return RBD_EINVAL;
    if (xt != RBD_F64 && xt != RBD_F32) return RBD_EUNSUPPORTED;
    if (round_up(I.m, 128) > kBMaxRows || I.d_max > kBMaxD) return RBD_EUNSUPPORTED;
    if (I.n > ((int64_t)1 << 31)) return RBD_EUNSUPPORTED;
    return RBD_OK;
}

// Team sizes: a matrix whose estimated work (passes over X for its expected number of bases -- the
// caller's hint, else d_max -- plus the Gram-Schmidt streams) is large against a CTA's fair share
// of the batch gets ceil(team_pct / 100 * work / share) members (team_pct 150 by default), at most
// 16, one column group and 128 rows per member.
struct Plan {
    std::vector<int32_t> team;
    std::vector<int64_t> rb;
    std::vector<double> cost;
    std::vector<int32_t> order;  // matrices by decreasing cost
    int64_t nslots = 0;
};

Plan make_plan(const rbd_instance* inst, int64_t count, int P, int ctas, int C, int team_pct) {
    Plan pl;
    pl.team.resize(count);
    pl.rb.resize(count);
    pl.cost.resize(count);
    double total = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t dh = inst[i].d_hint > 0 ? std::min<int64_t>(inst[i].d_hint, inst[i].d_max) : inst[i].d_max;
        const double ldp = (double)round_up(inst[i].m, 128), n = (double)inst[i].n, d = (double)dh;
        pl.cost[i] = ldp * n * P * d + 3.0 * ldp * d * d;
        total += pl.cost[i];
    }
    const double share = total / std::max(1, ctas);
    for (int64_t i = 0; i < count; ++i) {
        const int64_t ldp = round_up(inst[i].m, 128);
        const int64_t ng = ceil_div(inst[i].n, (int64_t)C);
        const int64_t tmax = std::max<int64_t>(1, std::min<int64_t>({16, ng, ldp / 128}));
        int64_t t = (int64_t)std::ceil(0.01 * team_pct * pl.cost[i] / share);
        t = std::max<int64_t>(1, std::min(t, tmax));
        pl.team[i] = (int32_t)t;
        pl.rb[i] = round_up(ceil_div(ldp, t), 32);
        pl.nslots += t;
    }
    pl.order.resize(count);
    std::iota(pl.order.begin(), pl.order.end(), 0);
    std::stable_sort(pl.order.begin(), pl.order.end(), [&](int32_t a, int32_t b) { return pl.cost[a] > pl.cost[b]; });
    return pl;
}

struct Layout {
    size_t queue, status, bars, per_begin, inst, slot_inst, slot_member, colstart, total;
    std::vector<size_t> planes, ys, e, xn2, hpart, nrm, vbuf, cand_e, cand_j, frop;
};

bool make_layout(const rbd_instance* inst, int64_t count, rbd_dtype xt, const Plan& pl, int C, Layout& L) {
    const int P = (xt == RBD_F64) ? 2 : 1;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = al256(off + b);
        return o;
    };
    L.queue = take(4);
    L.status = take((size_t)count * 4);
    L.bars = take((size_t)count * 4);
    L.per_begin = off;
    L.inst = take((size_t)count * sizeof(BInst));
    L.slot_inst = take((size_t)pl.nslots * 4);
    L.slot_member = take((size_t)pl.nslots * 4);
    L.colstart = take((size_t)(count + 1) * 8);
    for (auto* v : {&L.planes, &L.ys, &L.e, &L.xn2, &L.hpart, &L.nrm, &L.vbuf, &L.cand_e, &L.cand_j, &L.frop})
        v->assign(count, 0);
    for (int64_t i = 0; i < count; ++i) {
        if (check_inst(inst[i], xt) != RBD_OK) return false;
        const int64_t ldp = round_up(inst[i].m, 128);
        const int64_t ng = ceil_div(inst[i].n, (int64_t)C);
        const int64_t t = pl.team[i];
        L.planes[i] = take((size_t)ng * C * P * ldp * 4);
        L.ys[i] = take((size_t)t * 2 * inst[i].d_max * pl.rb[i] * 4);
        L.e[i] = take((size_t)inst[i].n * 8);
        L.xn2[i] = take((size_t)inst[i].n * 8);
        if (t > 1) {
            L.hpart[i] = take((size_t)t * inst[i].d_max * 8);
            L.nrm[i] = take((size_t)t * 8);
            L.vbuf[i] = take((size_t)2 * ldp * 4);
            L.cand_e[i] = take((size_t)t * 8);
            L.cand_j[i] = take((size_t)t * 8);
            L.frop[i] = take((size_t)t * 8);
        }
    }
    L.total = off;
    return true;
}

rbd_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RBD_OK;
    if (e == cudaErrorMemoryAllocation) return RBD_ENOMEM;
    return RBD_ECUDA;
}

// The kernel instances: storage (P = 2: FP64 as two planes, 1: FP32) x columns per warp (2, 4) x
// tile rows (128, 256).
struct BKernel {
    const void* fn;
    size_t smem;
    int smax;
};

template <int P, int CPW, int MT>
BKernel bkernel() {
    return BKernel{(const void*)batch_kernel<P, CPW, MT>, batch_smem<P, CPW, MT>(), BCfg<P, CPW, MT>::SMAX};
}

BKernel kernel_for(int P, int cols, int tile_rows) {
    const int i = (P == 2 ? 4 : 0) + (cols == 32 ? 2 : 0) + (tile_rows == 128 ? 1 : 0);
    switch (i) {
        case 0: return bkernel<1, 2, 256>();
        case 1: return bkernel<1, 2, 128>();
        case 2: return bkernel<1, 4, 256>();
        case 3: return bkernel<1, 4, 128>();
        case 4: return bkernel<2, 2, 256>();
        case 5: return bkernel<2, 2, 128>();
        case 6: return bkernel<2, 4, 256>();
        default: return bkernel<2, 4, 128>();
    }
}

constexpr int kColsOpt[2] = {16, 32};
constexpr int kRowsOpt[2] = {256, 128};
constexpr int kTeamOpt[3] = {150, 75, 300};

bool valid_config(int cols, int tile_rows, int team_pct) {
    return (cols == 16 || cols == 32) && (tile_rows == 128 || tile_rows == 256) &&
           (team_pct == 75 || team_pct == 150 || team_pct == 300);
}

std::mutex g_battr_mu;
bool g_battr_done[64] = {};

cudaError_t batch_setup(int dev) {
    std::lock_guard<std::mutex> lk(g_battr_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_battr_done[dev]) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int P = 1; P <= 2 && e == cudaSuccess; ++P)
        for (int cols : kColsOpt)
            for (int rows : kRowsOpt) {
                const BKernel k = kernel_for(P, cols, rows);
                if (e == cudaSuccess) e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
            }
    if (e == cudaSuccess) g_battr_done[dev] = true;
    return e;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}

rbd_status run_with(rbd_batch_plan p, rbd_batch_result* results, cudaStream_t st, int S) {
    BatchParams bp;
    bp.inst = p->d_inst;
    bp.count = p->count;
    bp.nslots = p->nslots;
    bp.slot_inst = p->d_slot_inst;
    bp.slot_member = p->d_slot_member;
    bp.colstart = p->d_colstart;
    bp.queue = p->d_queue;
    bp.status = p->d_status;
    bp.res = results;
    bp.S = S;
    bp.C = p->cols;
    bp.MT = p->tile_rows;
    bp.wait_ns = wait_limit_ns(kWaitLimitNs);
    bp.team_ns = wait_limit_ns(kTeamWaitNs);
    cudaError_t e = cudaMemsetAsync(p->d_queue, 0, p->zero_bytes, st);
    if (e != cudaSuccess) return cuda_status(e);
    void* args[] = {&bp};
    const int P = (p->xt == RBD_F64) ? 2 : 1;
    const BKernel k = kernel_for(P, p->cols, p->tile_rows);
    if (P == 2)
        batch_init_kernel<2><<<p->init_blocks, 256, 0, st>>>(bp);
    else
        batch_init_kernel<1><<<p->init_blocks, 256, 0, st>>>(bp);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(k.fn, dim3((unsigned)p->num_sms), dim3(kBThreads), args, k.smem, st);
    return cuda_status(e);
}

// Workspace of the layout every launch shape needs (the largest: the group width pads columns,
// the team size sizes the member blocks and exchange buffers).
size_t workspace_for_all(const rbd_instance* inst, int64_t count, rbd_dtype xt, int sms) {
    const int P = (xt == RBD_F64) ? 2 : 1;
    size_t most = 0;
    for (int cols : kColsOpt)
        for (int team : kTeamOpt) {
            const Plan pl = make_plan(inst, count, P, sms, cols, team);
            Layout L;
            if (!make_layout(inst, count, xt, pl, cols, L)) return 0;
            most = std::max(most, L.total);
        }
    return most;
}

// Lay the plan's workspace out for a launch shape and upload the descriptor table (synchronises
// the stream: the host vectors go out of scope).
rbd_status plan_apply(rbd_batch_plan p, int cols, int tile_rows, int team_pct, int stages, cudaStream_t st) {
    const rbd_dtype xt = (rbd_dtype)p->xt;
    const int P = (xt == RBD_F64) ? 2 : 1;
    const int64_t count = p->count;
    const rbd_instance* inst = p->inst.data();
    const Plan pl = make_plan(inst, count, P, p->num_sms, cols, team_pct);
    Layout L;
    if (!make_layout(inst, count, xt, pl, cols, L)) return RBD_EINVAL;
    if (L.total > p->ws_bytes) return RBD_ENOMEM;
    const BKernel k = kernel_for(P, cols, tile_rows);
    if (stages < 0 || stages == 1 || stages > k.smax) return RBD_EINVAL;
    unsigned char* base = p->ws;
    std::vector<BInst> hi(count);
    std::vector<int64_t> colstart(count + 1, 0);
    for (int64_t i = 0; i < count; ++i) {
        const rbd_instance& s = inst[i];
        BInst& b = hi[i];
        std::memset(&b, 0, sizeof(b));
        b.X = s.X;
        b.m = s.m;
        b.n = s.n;
        b.ldx = s.ldx;
        b.ldp = round_up(s.m, 128);
        b.ngroups = ceil_div(s.n, (int64_t)cols);
        b.NT = ceil_div(b.ldp, (int64_t)tile_rows);
        b.tol = s.tol;
        b.mode = s.mode;
        b.team = pl.team[i];
        b.d_max = s.d_max;
        b.start = s.start;
        b.Y = s.Y;
        b.ldy = s.ldy;
        b.T = s.T;
        b.ldt = s.ldt;
        b.piv = s.pivots;
        b.err = s.err;
        b.nu = s.nu;
        b.planes = (float*)(base + L.planes[i]);
        b.ys = (float*)(base + L.ys[i]);
        b.rb = pl.rb[i];
        b.e = (double*)(base + L.e[i]);
        b.xn2 = (double*)(base + L.xn2[i]);
        b.bar = (uint32_t*)(base + L.bars) + i;
        if (pl.team[i] > 1) {
            b.hpart = (double*)(base + L.hpart[i]);
            b.nrm = (double*)(base + L.nrm[i]);
            b.vbuf = (float*)(base + L.vbuf[i]);
            b.cand_e = (double*)(base + L.cand_e[i]);
            b.cand_j = (int64_t*)(base + L.cand_j[i]);
            b.frop = (double*)(base + L.frop[i]);
        }
        colstart[i + 1] = colstart[i] + b.ngroups * cols;
    }
    std::vector<int32_t> slot_inst, slot_member;
    slot_inst.reserve(pl.nslots);
    slot_member.reserve(pl.nslots);
    for (int32_t i : pl.order)
        for (int32_t b = 0; b < pl.team[i]; ++b) {
            slot_inst.push_back(i);
            slot_member.push_back(b);
        }
    cudaError_t ce = cudaMemcpyAsync(base + L.inst, hi.data(), (size_t)count * sizeof(BInst), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + L.slot_inst, slot_inst.data(), (size_t)pl.nslots * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + L.slot_member, slot_member.data(), (size_t)pl.nslots * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(base + L.colstart, colstart.data(), (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(ce);
    }
    p->nslots = pl.nslots;
    p->cols = cols;
    p->tile_rows = tile_rows;
    p->team_pct = team_pct;
    p->S = stages ? stages : k.smax;
    p->smem = k.smem;
    p->init_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(colstart[count], 8), (int64_t)p->num_sms * 8));
    p->d_inst = (BInst*)(base + L.inst);
    p->d_slot_inst = (int32_t*)(base + L.slot_inst);
    p->d_slot_member = (int32_t*)(base + L.slot_member);
    p->d_colstart = (int64_t*)(base + L.colstart);
    p->d_queue = (uint32_t*)(base + L.queue);
    p->d_status = (int32_t*)(base + L.status);
    p->zero_bytes = L.per_begin;
    return RBD_OK;
}

}  // namespace

extern "C" {

size_t rbd_batch_workspace_bytes(const rbd_instance* inst, int64_t count, rbd_dtype xt) {
    if (!inst || count < 1) return 0;
    for (int64_t i = 0; i < count; ++i)
        if (check_inst(inst[i], xt) != RBD_OK) return 0;
    int sms = device_sms();
    if (sms <= 0) sms = 160;  // no device: plan for a 160-SM part
    return workspace_for_all(inst, count, xt, sms);
}

rbd_status rbd_batch_plan_create(rbd_batch_plan* plan, const rbd_instance* inst, int64_t count, rbd_dtype xt,
                                 void* workspace, size_t workspace_bytes, void* stream) {
    if (!plan || !inst || count < 1 || count > ((int64_t)1 << 30)) return RBD_EINVAL;
    *plan = nullptr;
    for (int64_t i = 0; i < count; ++i) {
        const rbd_status s = check_inst(inst[i], xt);
        if (s != RBD_OK) return s;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_status(ce);
    int sms = 0, coop = 0;
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (ce == cudaSuccess) ce = batch_setup(dev);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(ce);
    }
    if (!coop) return RBD_EUNSUPPORTED;
    const size_t need = workspace_for_all(inst, count, xt, sms);
    if (need == 0) return RBD_EINVAL;
    if (!workspace || ((uintptr_t)workspace & 255u) != 0) return RBD_EINVAL;
    if (workspace_bytes < need) return RBD_ENOMEM;
    rbd_batch_plan p = new (std::nothrow) rbd_batch_plan_s();
    if (!p) return RBD_ENOMEM;
    p->xt = (int)xt;
    p->count = count;
    p->num_sms = sms;
    p->inst.assign(inst, inst + count);
    p->ws = (unsigned char*)workspace;
    p->ws_bytes = workspace_bytes;
    const rbd_status rs = plan_apply(p, 16, 256, 150, 0, (cudaStream_t)stream);
    if (rs != RBD_OK) {
        delete p;
        return rs;
    }
    *plan = p;
    return RBD_OK;
}

rbd_status rbd_batch_run(rbd_batch_plan plan, rbd_batch_result* results, void* stream) {
    if (!plan || !results) return RBD_EINVAL;
    return run_with(plan, results, (cudaStream_t)stream, plan->S);
}

rbd_status rbd_batch_tune(rbd_batch_plan plan, rbd_batch_result* results, void* stream, rbd_batch_config* chosen) {
    if (!plan || !results) return RBD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return RBD_ECUDA;
    }
    const int P = (plan->xt == RBD_F64) ? 2 : 1;
    // one run (the first of a shape warms it up), timed
    auto timed = [&](int S, float& ms) -> rbd_status {
        rbd_status rs = run_with(plan, results, st, S);
        if (rs != RBD_OK) return rs;
        cudaEventRecord(e0, st);
        rs = run_with(plan, results, st, S);
        cudaEventRecord(e1, st);
        if (rs != RBD_OK) return rs;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return RBD_ECUDA;
        return RBD_OK;
    };
    rbd_status rs = RBD_OK;
    float best = 1e30f;
    int bc = plan->cols, br = plan->tile_rows, bt = plan->team_pct;
    // every launch shape at its deepest ring
    for (int cols : kColsOpt)
        for (int rows : kRowsOpt)
            for (int team : kTeamOpt) {
                if (rs != RBD_OK) break;
                rs = plan_apply(plan, cols, rows, team, 0, st);
                float ms = 0.f;
                if (rs == RBD_OK) rs = timed(plan->S, ms);
                if (rs == RBD_OK && ms < best) {
                    best = ms;
                    bc = cols;
                    br = rows;
                    bt = team;
                }
            }
    // the ring depths of the fastest shape
    int bs = 0;
    if (rs == RBD_OK) rs = plan_apply(plan, bc, br, bt, 0, st);
    if (rs == RBD_OK) {
        const int smax = kernel_for(P, bc, br).smax;
        float best_s = best;
        for (int s = 2; s < smax && rs == RBD_OK; s = (s < 4) ? s + 1 : 2 * s) {
            float ms = 0.f;
            rs = timed(s, ms);
            if (rs == RBD_OK && ms < best_s) {
                best_s = ms;
                bs = s;
            }
        }
    }
    if (rs == RBD_OK) {
        plan->S = bs ? bs : kernel_for(P, bc, br).smax;
        if (chosen) {
            chosen->cols = bc;
            chosen->tile_rows = br;
            chosen->team_pct = bt;
            chosen->stages = plan->S;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return rs;
}

rbd_status rbd_batch_plan_config(rbd_batch_plan plan, rbd_batch_config* cfg) {
    if (!plan || !cfg) return RBD_EINVAL;
    cfg->cols = plan->cols;
    cfg->tile_rows = plan->tile_rows;
    cfg->team_pct = plan->team_pct;
    cfg->stages = plan->S;
    return RBD_OK;
}

rbd_status rbd_batch_plan_set_config(rbd_batch_plan plan, const rbd_batch_config* cfg, void* stream) {
    if (!plan || !cfg || !valid_config(cfg->cols, cfg->tile_rows, cfg->team_pct)) return RBD_EINVAL;
    return plan_apply(plan, cfg->cols, cfg->tile_rows, cfg->team_pct, cfg->stages, (cudaStream_t)stream);
}

rbd_status rbd_batch_plan_destroy(rbd_batch_plan plan) {
    delete plan;
    return RBD_OK;
}

rbd_status rbd_compress_batched(const rbd_instance* inst, int64_t count, rbd_dtype xt, rbd_batch_result* results,
                                void* stream) {
    if (!inst || !results || count < 1) return RBD_EINVAL;
    const size_t ws_bytes = rbd_batch_workspace_bytes(inst, count, xt);
    if (ws_bytes == 0) {
        for (int64_t i = 0; i < count; ++i) {
            const rbd_status s = check_inst(inst[i], xt);
            if (s != RBD_OK) return s;
        }
        return RBD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void* ws = nullptr;
    void* dres = nullptr;
    cudaError_t ce = lib_malloc_async(&ws, ws_bytes, st);
    if (ce == cudaSuccess) ce = lib_malloc_async(&dres, (size_t)count * sizeof(rbd_batch_result), st);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        if (ws) cudaFreeAsync(ws, st);
        return RBD_ENOMEM;
    }
    rbd_batch_plan plan = nullptr;
    rbd_status rs = rbd_batch_plan_create(&plan, inst, count, xt, ws, ws_bytes, stream);
    if (rs == RBD_OK) rs = rbd_batch_run(plan, (rbd_batch_result*)dres, stream);
    if (rs == RBD_OK) {
        ce = cudaMemcpyAsync(results, dres, (size_t)count * sizeof(rbd_batch_result), cudaMemcpyDeviceToHost, st);
        if (ce != cudaSuccess) rs = cuda_status(ce);
    }
    cudaFreeAsync(dres, st);
    cudaFreeAsync(ws, st);
    ce = cudaStreamSynchronize(st);
    if (rs == RBD_OK && ce != cudaSuccess) rs = cuda_status(ce);
    if (plan) rbd_batch_plan_destroy(plan);
    cudaGetLastError();
    return rs;
}

}  // extern "C"
