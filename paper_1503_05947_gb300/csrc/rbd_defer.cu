// rbd_defer.cu -- the greedy loop of Algorithm 1 (A = I) in ONE persistent cooperative kernel with
// two grid barriers per basis.
//
// Basis k applies classical Gram-Schmidt twice to the pivot column x_i (Section 3.1, step 2.2, with
// one re-orthogonalisation):
//     v1 = x_i - Y t,   t = Y' x_i = T(0:k, i)        (the first sweep's coefficients are in T)
//     h  = Y' v1,       v2 = v1 - Y h,   nu = ||v2||,   xi_k = v2 / nu.
// The fused pass (T(k, :) of step 2.2, the indicator of step 2.3) needs c_j = xi_k' x_j for every
// column.  Because Y' x_j = T(0:k, j) and Y'Y = I,
//     c_j = (v1' x_j - h' T(0:k, j)) / nu,        nu^2 = ||v1||^2 - ||h||^2,
// so X can be streamed as soon as v1 is known.  The grid-wide reduction of the second sweep (h, nu
// and the stop tests of steps 2.2 and 2.4) runs in a service warp while the pass streams X, and a
// column's dot product v1' x_j is corrected when its column group is finalised.  v2 and xi_k are
// formed at the start of the next basis, in the same stream over Y as that basis's first sweep.
//
// Per basis k, every CTA (one per SM: 8 consumer warps, a producer warp and a service warp):
//   F    Y_b(:, 0:k-1) (this CTA's rows, split FP32, row-block-major) streamed once for two row
//        sums: a = Y h_{k-1} gives v2 = v1_{k-1} - a and xi_{k-1} = v2 / nu_{k-1} = Y(:, k-1);
//        b = Y t gives v1_k = x_i - b - xi_{k-1} T(k-1, i)
//   O1'  hpart[b] = Y_b(:, 0:k)' v1_k (the new column from shared memory), the partial ||v1_k||^2,
//        and v1_k split into the pivot-vector tiles of the pass
//   ---- grid barrier 1
//   P    the pass with v1_k: the producer's bulk copies into a ring of stages, float-float dot
//        products in the consumers (rbd_tile.cuh).  Meanwhile the service warp sums k / G
//        coefficients of h over the CTAs, waits on a counter for the other CTAs' shares (the
//        consumers keep streaming), and forms nu and the stop decision.  A group's finaliser
//        subtracts h' T(0:k, j) and divides by nu.  The term is ||h|| / nu relative to the
//        column's norm (~4e-12 on the image workload): in FP32 from a group-blocked FP32 copy of
//        T streamed into shared memory while ||h|| / nu <= 2^-29, else in float-float from T
//        itself (ill-conditioned steps: T(:, i) is the first sweep of later bases, and an error
//        there returns amplified by ||x_i|| / nu).
//   ---- grid barrier 2
//   A    argmax over the CTAs' candidates (every CTA)
// A basis that step 2.2 or 2.4 rejects is known once the service warp is done; its pass stops at
// the next finalised group and writes nothing.  Every wait is bounded (kWaitLimitNs,
// kBarrierLimitNs); a wait that runs out raises RBD_ETIMEOUT and the abort bit of the barrier
// word, and the CTAs leave at their next grid barrier after their copies in flight have landed.
#include <algorithm>
#include <climits>

#include "rbd_device.cuh"
#include "rbd_loop.cuh"
#include "rbd_tile.cuh"
#include "rbd_work.h"

namespace rbd {

struct DeferParams {
    int64_t m, n, ldp, ldx, ldt, ldy, d_max;
    int64_t k0;           // first basis index of this launch (0, or d0 when resuming)
    int xt;
    const unsigned char* planes;
    int64_t group_stride, tile_stride, NT, ngroups, W;
    int KMAX;
    int evict_first;
    const void* X;
    double* Y;
    double* T;
    int64_t* pivots;
    double* err;
    double* nu_out;
    Ctl* ctl;
    uint32_t* bar;        // grid barrier word (monotonic arrivals, abort bit)
    uint32_t* hcnt;       // shares of h published (monotonic, G per basis)
    uint32_t* hdone;      // CTAs whose partial Y' v1 and ||v1||^2 are published (monotonic, G per basis)
    double* e;
    const double* xn2;
    float* ysb;           // [G][2][d_max][RS] split Y, row-block-major
    float* vs;            // tile-interleaved split v1 (pivot-vector tiles of the pass)
    float* tf;            // [ngroups][d_max][C] T in FP32, group-blocked (the flush corrections)
    double* hpart;        // [G][d_max] float-float pairs (hi, lo) of the partial second-sweep sums
    double* h;            // [d_max]
    double* nu2part;      // [G] float-float pairs: each block's ||v1||^2
    double* pbest_e;      // [G]
    int64_t* pbest_j;     // [G]
    uint32_t* gcnt;
    double* gslot;
    double* gsum;         // [2][ngroups]: per-group sums of e_j, by parity of the basis
    int R, RS, LC, KC;
    uint64_t wait_ns;     // bound on every wait of the loop (the exit drains keep kWaitLimitNs)
};

struct DeferSmem {
    size_t bars, v1s, xis, v1hl, part, coef, tfb, corr, scratch, total;
};

// Shared-memory layout (host and device agree through this function).  KC = d_max rounded up to 4.
template <class Cfg>
__host__ __device__ inline DeferSmem defer_smem_layout(int R, int KC) {
    constexpr int NCONS = Cfg::NW * 32;
    DeferSmem s;
    size_t o = (size_t)Cfg::S * Cfg::STAGE_FLOATS * 4;  // the ring: pass stages / Y chunks
    s.bars = o;
    o += (size_t)(3 * Cfg::S + 2) * 8;              // full, empty, ybar; tfull, svc
    o = (o + 15) & ~size_t(15);
    s.v1s = o;
    o += (size_t)R * 8;                            // v1 (FP64), kept into the next basis
    s.xis = o;
    o += (size_t)2 * R * 4;                        // xi_{k-1} split: hi, lo
    s.v1hl = o;
    o += (size_t)2 * R * 4;                        // v1 split: hi, lo
    s.part = o;
    o += (size_t)2 * NCONS * 8;                    // partial sums of the slice GEMVs
    s.coef = o;
    o += (size_t)4 * KC * 4;                       // [h hi | h lo | t hi | t lo]
    s.tfb = o;
    // T(0:k, group) in FP32 during the pass; the row-sum partials of F (4 NCONS float pairs) before it
    const size_t tfb_bytes = (size_t)KC * Cfg::C * 4, fp_bytes = (size_t)4 * NCONS * 8;
    o += (tfb_bytes > fp_bytes) ? tfb_bytes : fp_bytes;
    s.corr = o;
    o += (size_t)Cfg::NW * Cfg::C * 4;             // flush corrections, per warp
    s.scratch = o;
    o += (size_t)(2 * Cfg::NW + 2 * Cfg::C + 8) * 8 + 16 * 4;
    s.total = (o + 127) & ~size_t(127);
    return s;
}

// Spin on the h counter until it reaches target (all lanes of the warp read the same word);
// false if the abort bit appeared or kBarrierLimitNs elapsed.
__device__ __forceinline__ bool wait_counter(const uint32_t* cnt, const uint32_t* bar, uint32_t target,
                                             uint64_t limit_ns) {
    if (ld_acquire_u32(cnt) >= target) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire_u32(cnt) >= target) return true;
        if ((it & 63u) == 63u) {
            if (*(volatile const uint32_t*)bar & kAbortBit) return false;
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
}

template <int XT>
__global__ void __launch_bounds__(TileCfg<XT>::THREADS + 32, 1) defer_kernel(DeferParams p) {
    using Cfg = TileCfg<XT>;
    constexpr int UB = Cfg::PL * Cfg::ESIZE;  // X bytes per element and column of a unit
    constexpr int NW = Cfg::NW, CPW = Cfg::CPW, C = Cfg::C, MT = Cfg::MT, S = Cfg::S;
    constexpr int XI = Cfg::XI_FLOATS, STAGE = Cfg::STAGE_FLOATS;
    constexpr int NCONS = NW * 32;
    constexpr int MAXRPT = kLoopMaxRows / NCONS;  // rows per consumer thread when R > NCONS
    constexpr int NLS = NCONS / C;                // row subsets of a flush correction
    constexpr int PROD = NW, SVC = NW + 1;        // producer and service warps

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int R = p.R, RS = p.RS, LC = p.LC, KC = p.KC;
    const DeferSmem L = defer_smem_layout<Cfg>(R, KC);
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bars);
    uint64_t* empty = full + S;
    uint64_t* ybar = empty + S;
    uint64_t* tfull = ybar + S;
    uint64_t* svcb = tfull + 1;
    double* v1s = reinterpret_cast<double*>(smem_raw + L.v1s);
    float* xih = reinterpret_cast<float*>(smem_raw + L.xis);
    float* xil = xih + R;
    float* v1h = reinterpret_cast<float*>(smem_raw + L.v1hl);
    float* v1l = v1h + R;
    double* part = reinterpret_cast<double*>(smem_raw + L.part);
    float* cah = reinterpret_cast<float*>(smem_raw + L.coef);
    float* cal = cah + KC;
    float* cbh = cal + KC;
    float* cbl = cbh + KC;
    float* tfb = reinterpret_cast<float*>(smem_raw + L.tfb);
    float* corr = reinterpret_cast<float*>(smem_raw + L.corr);
    double* red_e = reinterpret_cast<double*>(smem_raw + L.scratch);  // NW
    int64_t* red_j = reinterpret_cast<int64_t*>(red_e + NW);          // NW
    double* grp_e = reinterpret_cast<double*>(red_j + NW);           // 2 C
    double* bcast = grp_e + 2 * C;                                   // 8: nu, 1/nu, ||h||^2
    int* sfl = reinterpret_cast<int*>(bcast + 8);
    // sfl: [0] grid-barrier result  [1] stop decision (service warp)  [2] last-arriver flag of a
    //      flush  [3] units the producer issued in a cut pass  [4] basis tag of [3]  [5] the
    //      decision as the consumers read it (one reader, then a barrier: a uniform value)
    //      [6] float-float flush corrections this basis (service warp)
    volatile int* vfl = sfl;

    Ctl* ctl = p.ctl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t r0 = b * (int64_t)R;
    const int Rb = (int)max((int64_t)0, min((int64_t)R, p.ldp - r0));  // rows of this block within ldp
    const int NQ = Rb / 4;
    const int64_t W = p.W, NT = p.NT;
    const int64_t L0 = (W * b) / G, L1 = (W * (b + 1)) / G;
    const int64_t nunits = L1 - L0;
    // Column groups of this CTA's range.  The T block of each group the CTA starts is streamed into
    // shared memory for the flush correction; a range that starts inside a group leaves that group
    // to the CTA before it (its last arriver in practice), and reads T from global memory in the
    // rare case that it finalises it.
    const int64_t gfirst = (nunits > 0) ? L0 / NT : 0, glast = (nunits > 0) ? (L1 - 1) / NT : -1;
    const int64_t gtf0 = (L0 % NT != 0) ? gfirst + 1 : gfirst;

    if (ctl->status != 0 || ctl->stop != 0) return;  // set by the initial pass, uniform

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 2);    // X part and pivot-vector part arrive separately
            mbar_init(&empty[s], NW);
            mbar_init(&ybar[s], 1);    // Y chunks streamed through the same buffers
        }
        mbar_init(tfull, 1);
        mbar_init(svcb, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Y-chunk geometry: NB buffers of spb ring stages, LC columns of both planes each.
    const int spb = loop_ybuf_stages<Cfg>(RS);
    const int NB = S / spb;
    const int ybuf = spb * STAGE;
    const int yplane = LC * RS;
    const float* ysrc = p.ysb + b * 2 * p.d_max * (int64_t)RS;
    // Y slices and the FP32 T blocks are re-read every basis: kept in L2 against the X stream
    const uint64_t pol_y = l2_policy_evict_last();
    const uint64_t pol_x = p.evict_first ? l2_policy_evict_first() : l2_policy_evict_normal();
    const uint64_t pol_v = l2_policy_evict_normal();
    const unsigned char* planes = p.planes;

    bool ok = true;
    uint32_t gen = 0, hround = 0;
    // producer (lane 0 of warp PROD)
    int ps = 0;
    uint32_t pph = 0;
    bool preuse = false;
    uint32_t iss_par = 0, iss_mask = 0;  // parity and presence of the last issue into each stage
    // consumers (identical copies in every consumer thread)
    int cs = 0;
    uint32_t cph = 0;
    uint32_t ypar = 0, ypend = 0;  // per Y buffer: parity of the next phase, chunk in flight
    int64_t ypre = 0;              // chunks of the coming F issued at the end of the last pass
    uint32_t tcnt = 0;             // T blocks streamed
    bool tf_pend = false;
    uint32_t dcount = 0;           // column-dot chunks (parity of their partial buffer)

    int64_t piv = ctl->pivot;
    const int mode = ctl->mode;
    const double eps_r = ctl->eps_r, eps_r22 = ctl->eps_r22, fro_tol = ctl->fro_tol;
    double inv_prev = 0.0;   // 1 / nu_{k-1}
    bool small_h = true;     // ||h_{k-1}|| <= 2^-36 nu_{k-1}: Y h_{k-1} in plain FP32 is exact enough

    int64_t k = p.k0;
    int32_t stop = STOP_NONE;
    for (;; ++k) {
        const bool deferred = k > p.k0;            // xi_{k-1} is formed in this basis
        const int64_t ncol = deferred ? k - 1 : k; // columns of Y streamed (complete in ysb)
        const int64_t nch = ceil_div(ncol, (int64_t)LC);
        const bool resident = nch <= NB;           // the slice stays in the ring for O1'
        const int64_t ytot = resident ? nch : 2 * nch;
        const bool run_pass = k < p.d_max;
        const uint32_t spar = (uint32_t)((k - p.k0) & 1);

        // Y chunk u of a basis with ncolv streamed columns (nchv chunks) into buffer u % NB
        auto y_issue = [&](int64_t u, int64_t ncolv, int64_t nchv) {
            const int bf = (int)(u % NB);
            if (tid == 0) {
                const int64_t l0 = (u % nchv) * LC;
                const int lc = (int)min((int64_t)LC, ncolv - l0);
                const uint32_t bytes = (uint32_t)lc * (uint32_t)RS * 4u;
                float* dst = stages + (size_t)bf * ybuf;
                mbar_arrive_expect_tx(&ybar[bf], 2u * bytes);
                bulk_g2s(dst, ysrc + l0 * RS, bytes, &ybar[bf], pol_y);
                bulk_g2s(dst + yplane, ysrc + (p.d_max + l0) * RS, bytes, &ybar[bf], pol_y);
            }
            ypend |= 1u << bf;
        };
        auto y_wait = [&](int bf) {
            if (ok && !mbar_wait(&ybar[bf], (ypar >> bf) & 1u, p.wait_ns)) {
                loop_abort(ctl, p.bar, ST_ETIMEOUT);
                ok = false;
            }
            ypar ^= 1u << bf;
            ypend &= ~(1u << bf);
        };

        // ---------------- F: xi_{k-1} and v1_k in one stream over Y ----------------
        if (warp < NW) {
            // the pivot column's rows of this block (row tid + i NCONS in thread tid), and the
            // first-sweep coefficients t = T(0:k, i), split with integer operations
            double xr[MAXRPT];
#pragma unroll
            for (int i = 0; i < MAXRPT; ++i) {
                const int r = tid + i * NCONS;
                xr[i] = (r < Rb && r0 + r < p.m) ? load_x_elem(p.X, p.xt, piv * p.ldx + r0 + r) : 0.0;
            }
            const double* tcol = p.T + piv * p.ldt;
            const double tlast = deferred ? __ldcg(&tcol[k - 1]) : 0.0;
            for (int64_t l = tid; l < ncol; l += 2 * NCONS) {
                // both loads in flight before the shared-memory stores
                const double t0 = __ldcg(&tcol[l]);
                const double t1 = (l + NCONS < ncol) ? __ldcg(&tcol[l + NCONS]) : 0.0;
                split_f64_fast(t0, cbh[l], cbl[l]);
                if (l + NCONS < ncol) split_f64_fast(t1, cbh[l + NCONS], cbl[l + NCONS]);
            }
            // Generic-proxy writes (this CTA's columns of ysb) are read by bulk copies (the async
            // proxy): the issuing thread orders them with a proxy fence after the barriers that made
            // them visible to it (here and before every batch of copies below).
            if (tid == 0 && ypre < min((int64_t)NB, ytot)) fence_proxy_async_global();
            for (int64_t u = ypre; u < min((int64_t)NB, ytot); ++u) y_issue(u, ncol, nch);
            ypre = 0;
            named_bar(1, NCONS);  // coefficients staged

            // Row sums: thread (pair pr, segment sg) sums rows 2 pr and 2 pr + 1 over the columns sg,
            // sg + NSG, ... of each chunk: four independent chains (two rows x B and A).  B = Y t in
            // float-float; A = Y h_{k-1} in plain FP32 while h is small, else float-float.
            const int NPR = R / 2;
            const int NSG = max(1, NCONS / NPR);
            const int pr = tid % NPR, sg = tid / NPR;
            const bool active = sg < NSG;
            const int rp = 2 * pr;
            float b0s = 0.f, b0c = 0.f, b1s = 0.f, b1c = 0.f, a0s = 0.f, a0c = 0.f, a1s = 0.f, a1c = 0.f;
            const int amode = deferred ? (small_h ? 1 : 2) : 0;
            for (int64_t u = 0; u < nch; ++u) {
                const int bf = (int)(u % NB);
                y_wait(bf);
                const float* yh = stages + (size_t)bf * ybuf;
                const float* yl = yh + yplane;
                const int64_t l0 = u * LC;
                const int lc = (int)min((int64_t)LC, ncol - l0);
                const float* ch = cbh + l0;
                const float* cl = cbl + l0;
                const float* hh = cah + l0;
                const float* hl = cal + l0;
                if (active && ok && rp < Rb) {
                    if (amode == 1) {
                        for (int l = sg; l < lc; l += NSG) {
                            const float2 y = *reinterpret_cast<const float2*>(yh + l * RS + rp);
                            const float2 z = *reinterpret_cast<const float2*>(yl + l * RS + rp);
                            const float th = ch[l], tl = cl[l], ha = hh[l];
                            ff_mac2(b0s, b0c, y.x, z.x, th, tl);
                            ff_mac2(b1s, b1c, y.y, z.y, th, tl);
                            a0s = __fmaf_rn(y.x, ha, a0s);
                            a1s = __fmaf_rn(y.y, ha, a1s);
                        }
                    } else if (amode == 2) {
                        for (int l = sg; l < lc; l += NSG) {
                            const float2 y = *reinterpret_cast<const float2*>(yh + l * RS + rp);
                            const float2 z = *reinterpret_cast<const float2*>(yl + l * RS + rp);
                            const float th = ch[l], tl = cl[l], ha = hh[l], hb = hl[l];
                            ff_mac2(b0s, b0c, y.x, z.x, th, tl);
                            ff_mac2(b1s, b1c, y.y, z.y, th, tl);
                            ff_mac2(a0s, a0c, y.x, z.x, ha, hb);
                            ff_mac2(a1s, a1c, y.y, z.y, ha, hb);
                        }
                    } else {
                        for (int l = sg; l < lc; l += NSG) {
                            const float2 y = *reinterpret_cast<const float2*>(yh + l * RS + rp);
                            const float2 z = *reinterpret_cast<const float2*>(yl + l * RS + rp);
                            const float th = ch[l], tl = cl[l];
                            ff_mac2(b0s, b0c, y.x, z.x, th, tl);
                            ff_mac2(b1s, b1c, y.y, z.y, th, tl);
                        }
                    }
                }
                if (!resident && u + NB < ytot) {
                    named_bar(1, NCONS);  // buffer bf consumed
                    y_issue(u + NB, ncol, nch);
                }
            }
            named_bar_arrive(2, NCONS + 32);  // F's loads are done: the producer may use HBM
            auto fin = [&](int r, int i, double A, double B) {
                const bool live = r < Rb && r0 + r < p.m;
                double xs = 0.0;  // xi_{k-1} as its split copy holds it (the value every stream sees)
                if (deferred) {
                    const double xi = live ? (v1s[r] - A) * inv_prev : 0.0;
                    if (live) p.Y[(r0 + r) + (k - 1) * p.ldy] = xi;
                    float hi, lo;
                    split_f64_fast(xi, hi, lo);
                    p.ysb[(b * 2 + 0) * p.d_max * RS + (k - 1) * RS + r] = hi;
                    p.ysb[(b * 2 + 1) * p.d_max * RS + (k - 1) * RS + r] = lo;
                    xih[r] = hi;
                    xil[r] = lo;
                    xs = (double)hi + (double)lo;
                }
                const double v = live ? (xr[i] - B) - xs * tlast : 0.0;
                v1s[r] = v;
                split_f64_fast(v, v1h[r], v1l[r]);
            };
            // The segments' partial sums of each row, added in segment order without loss: the high
            // parts through a chain of exact TwoSums, their rounding errors and the low parts into a
            // float-float accumulator some 2^-24 the size of the sum, so that the one rounding left
            // is the final conversion to FP64 (v1 = x - Y t cancels heavily when the pivot nearly
            // lies in span(Y); FP64 instructions are slow on this part).
            float2* fpart = reinterpret_cast<float2*>(tfb);  // [sg][pr][B0, B1, A0, A1]
            if (active) {
                float2* o = fpart + ((size_t)sg * NPR + pr) * 4;
                o[0] = make_float2(b0s, b0c);
                o[1] = make_float2(b1s, b1c);
                o[2] = make_float2(a0s, (amode == 1) ? 0.f : a0c);
                o[3] = make_float2(a1s, (amode == 1) ? 0.f : a1c);
            }
            named_bar(1, NCONS);
#pragma unroll
            for (int i = 0; i < MAXRPT; ++i) {
                const int r = tid + i * NCONS;
                if (r >= R) break;
                double A = 0.0, B = 0.0;
                if (r < Rb && ncol > 0) {
                    const float2* pin = fpart + (size_t)(r >> 1) * 4 + (r & 1);
                    float bs = pin[0].x, beh = pin[0].y, bel = 0.f;
                    float as = pin[2].x, aeh = pin[2].y, ael = 0.f;
                    for (int sgi = 1; sgi < NSG; ++sgi) {
                        const float2 pb = pin[(size_t)sgi * NPR * 4], pa = pin[(size_t)sgi * NPR * 4 + 2];
                        float e;
                        two_sum(bs, pb.x, bs, e);
                        ff_add(beh, bel, e, 0.f);
                        ff_add(beh, bel, pb.y, 0.f);
                        two_sum(as, pa.x, as, e);
                        ff_add(aeh, ael, e, 0.f);
                        ff_add(aeh, ael, pa.y, 0.f);
                    }
                    B = (double)bs + ((double)beh + (double)bel);
                    A = (double)as + ((double)aeh + (double)ael);
                }
                fin(r, i, A, B);
            }
            named_bar(1, NCONS);         // v1 and xi_{k-1} complete in shared memory

            // The split v1 tiles of the pass (tile t holds [hi(rows_t) | lo(rows_t)] at t * 2 * MT)
            // are all the pass needs from this CTA: they are published with the arrival at grid
            // barrier 1, and O1' runs while the other CTAs arrive.
            for (int r = tid; r < Rb; r += NCONS) {
                const int64_t row = r0 + r;
                const int64_t t = row / MT;
                const int64_t rt = min((int64_t)MT, p.ldp - t * MT);
                const int64_t off = t * 2 * MT + (row - t * MT);
                p.vs[off] = v1h[r];
                p.vs[off + rt] = v1l[r];
            }
            named_bar(1, NCONS);
            if (tid == 0) grid_arrive(p.bar);  // barrier 1: arrival

            // ---------------- O1': hpart[b] = Y_b(:, 0:k)' v1 ----------------
            // A streamed slice (too long to stay in the ring) goes chunk by chunk: one thread per
            // (column, row segment) of a chunk, four float-float chains over quads of rows, the
            // segments combined in order through shared memory.
            // Columns lc, lc + 1 of the last call (nx = 2, or 1 without a deferred column) are the new
            // column xi_{k-1} and v1 itself, both from shared memory: its hpart entry and this block's
            // ||v1||^2 come out of the same pass over the chunk's rows.
            auto dots_chunk = [&](const float* yh, const float* yl, int64_t l0, int lc, int nx) {
                const int lt = lc + nx;
                const int nseg = max(1, min(8, NCONS / lt));
                const int sq = (NQ + nseg - 1) / nseg;
                float* pf = reinterpret_cast<float*>(part) + ((dcount++ & 1u) ? 2 * NCONS : 0);
                if (tid < nseg * lt) {
                    const int l = tid % lt, sg = tid / lt;
                    const int q0 = sg * sq, q1 = min(NQ, q0 + sq);
                    const bool vcol = l >= lc && (l > lc || !deferred);  // the v1 column
                    const float* ch = (l < lc) ? yh + l * RS : vcol ? v1h : xih;
                    const float* cl = (l < lc) ? yl + l * RS : vcol ? v1l : xil;
                    float s4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (ok)
                        for (int qq = q0; qq < q1; ++qq) {
                            const float4 a = *reinterpret_cast<const float4*>(ch + 4 * qq);
                            const float4 al = *reinterpret_cast<const float4*>(cl + 4 * qq);
                            const float4 v = *reinterpret_cast<const float4*>(v1h + 4 * qq);
                            const float4 vl = *reinterpret_cast<const float4*>(v1l + 4 * qq);
                            ff_mac2(s4[0], c4[0], a.x, al.x, v.x, vl.x);
                            ff_mac2(s4[1], c4[1], a.y, al.y, v.y, vl.y);
                            ff_mac2(s4[2], c4[2], a.z, al.z, v.z, vl.z);
                            ff_mac2(s4[3], c4[3], a.w, al.w, v.w, vl.w);
                        }
                    ff_add_acc(s4[0], c4[0], s4[1], c4[1]);
                    ff_add_acc(s4[2], c4[2], s4[3], c4[3]);
                    ff_add_acc(s4[0], c4[0], s4[2], c4[2]);
                    pf[2 * (sg * lt + l)] = s4[0];
                    pf[2 * (sg * lt + l) + 1] = c4[0];
                }
                named_bar(1, NCONS);
                if (tid < lt) {
                    float s0 = pf[2 * tid], c0 = pf[2 * tid + 1];
                    for (int sg = 1; sg < nseg; ++sg)
                        ff_add_acc(s0, c0, pf[2 * (sg * lt + tid)], pf[2 * (sg * lt + tid) + 1]);
                    // float-float; the service warp converts (FP64 off the critical path)
                    const float2 r2 = make_float2(s0, c0);
                    if (tid < lc)
                        reinterpret_cast<float2*>(p.hpart)[b * p.d_max + l0 + tid] = r2;
                    else if (tid > lc || !deferred)
                        reinterpret_cast<float2*>(p.nu2part)[b] = r2;
                    else
                        reinterpret_cast<float2*>(p.hpart)[b * p.d_max + k - 1] = r2;
                }
            };
            const int nx = deferred ? 2 : 1;
            if (resident) {
                // Every column of the resident slice at once (column l < ncol in buffer l / LC, row
                // offset (l % LC) RS), then xi_{k-1} and v1: one thread per (column, row segment),
                // four float-float chains over quads of rows; segments only while the columns leave
                // threads idle, their partial sums combined in order through shared memory.
                const int lt = (int)ncol + nx;
                const int nseg = (2 * lt >= NCONS) ? 1 : max(1, min(8, NCONS / lt));
                const int sq = (NQ + nseg - 1) / nseg;
                float* pf = reinterpret_cast<float*>(part) + ((dcount++ & 1u) ? 2 * NCONS : 0);
                const int nh = (int)ncol + (deferred ? 1 : 0);  // columns with an hpart entry
                auto publish = [&](int l, float s0, float c0) {
                    const float2 r2 = make_float2(s0, c0);
                    if (l < nh)
                        reinterpret_cast<float2*>(p.hpart)[b * p.d_max + l] = r2;  // xi_{k-1}: index k - 1
                    else
                        reinterpret_cast<float2*>(p.nu2part)[b] = r2;
                };
                for (int task = tid; task < nseg * lt; task += NCONS) {
                    const int l = task % lt, sg = task / lt;
                    const float* ch;
                    const float* cl;
                    if (l < ncol) {
                        const int u = l / LC;
                        ch = stages + (size_t)u * ybuf + (size_t)(l - u * LC) * RS;
                        cl = ch + yplane;
                    } else {
                        const bool vcol = l > ncol || !deferred;
                        ch = vcol ? v1h : xih;
                        cl = vcol ? v1l : xil;
                    }
                    const int q0 = sg * sq, q1 = min(NQ, q0 + sq);
                    float s4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (ok)
                        for (int qq = q0; qq < q1; ++qq) {
                            const float4 a = *reinterpret_cast<const float4*>(ch + 4 * qq);
                            const float4 al = *reinterpret_cast<const float4*>(cl + 4 * qq);
                            const float4 v = *reinterpret_cast<const float4*>(v1h + 4 * qq);
                            const float4 vl = *reinterpret_cast<const float4*>(v1l + 4 * qq);
                            ff_mac2(s4[0], c4[0], a.x, al.x, v.x, vl.x);
                            ff_mac2(s4[1], c4[1], a.y, al.y, v.y, vl.y);
                            ff_mac2(s4[2], c4[2], a.z, al.z, v.z, vl.z);
                            ff_mac2(s4[3], c4[3], a.w, al.w, v.w, vl.w);
                        }
                    ff_add_acc(s4[0], c4[0], s4[1], c4[1]);
                    ff_add_acc(s4[2], c4[2], s4[3], c4[3]);
                    ff_add_acc(s4[0], c4[0], s4[2], c4[2]);
                    if (nseg == 1) {
                        publish(l, s4[0], c4[0]);
                    } else {
                        pf[2 * (sg * lt + l)] = s4[0];
                        pf[2 * (sg * lt + l) + 1] = c4[0];
                    }
                }
                if (nseg > 1) {
                    named_bar(1, NCONS);
                    if (tid < lt) {
                        float s0 = pf[2 * tid], c0 = pf[2 * tid + 1];
                        for (int sg = 1; sg < nseg; ++sg)
                            ff_add_acc(s0, c0, pf[2 * (sg * lt + tid)], pf[2 * (sg * lt + tid) + 1]);
                        publish(tid, s0, c0);
                    }
                }
            } else {
                for (int64_t u = nch; u < 2 * nch; ++u) {
                    const int bf = (int)(u % NB);
                    y_wait(bf);
                    const float* yh = stages + (size_t)bf * ybuf;
                    const int64_t l0 = (u - nch) * LC;
                    dots_chunk(yh, yh + yplane, l0, (int)min((int64_t)LC, ncol - l0), (u == 2 * nch - 1) ? nx : 0);
                    if (u + NB < ytot) y_issue(u + NB, ncol, nch);  // dots_chunk's barrier freed it
                }
            }
            // this CTA's partial Y' v1 and ||v1||^2 are published
            named_bar(1, NCONS);
            if (tid == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p.hdone) : "memory");
        } else if (warp == PROD) {
            named_bar(2, NCONS + 32);
            if (lane == 0 && run_pass) {
                // the first tiles of the pass into L2 while the orthogonalisation runs
                int64_t g = L0 / NT, t = L0 - (L0 / NT) * NT;
                const int64_t npf = min(nunits, (int64_t)S);
                for (int64_t i = 0; i < npf; ++i) {
                    const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                    bulk_prefetch_l2(planes + (g * p.group_stride + t * p.tile_stride) * Cfg::ESIZE,
                                     (uint32_t)(C * UB) * rows);
                    if (++t == NT) {
                        t = 0;
                        ++g;
                    }
                }
            }
            // barrier 1: this lane waits for the other CTAs' arrivals while the consumers run O1'
            if (lane == 0) sfl[0] = grid_poll(p.bar, (uint32_t)G * (gen + 1u), ctl, p.wait_ns);
        }
        // barrier 1 passed (uniform result), and every consumer is done with the ring
        __syncthreads();
        ++gen;
        if (!sfl[0]) break;

        int32_t dec = STOP_NONE;
        if (warp == SVC) {
            // ---------------- second sweep over the grid: h, nu, the stop tests ----------------
            double nu2 = 0.0, fs = 0.0, hh = 0.0;
            const double xn2p = (lane == 0) ? __ldg(&p.xn2[piv]) : 0.0;  // loads of this round first
            // every CTA's partial Y' v1 and ||v1||^2 (published after its arrival at barrier 1)
            if (!wait_counter(p.hdone, p.bar, (uint32_t)G * (uint32_t)(k - p.k0 + 1), p.wait_ns)) {
                if (lane == 0) loop_abort(ctl, p.bar, ST_ETIMEOUT);
                ok = false;
            }
#pragma unroll 4
            for (int64_t bb = lane; bb < G; bb += 32) {
                const float2 nv = __ldcg(reinterpret_cast<const float2*>(p.nu2part) + bb);
                nu2 += (double)nv.x + (double)nv.y;
            }
            if (k > 0) {
                const double* gs = p.gsum + ((k - 1) & 1) * p.ngroups;
#pragma unroll 8
                for (int64_t gg = lane; gg < p.ngroups; gg += 32) fs += __ldcg(&gs[gg]);
                // this CTA's share of h, k / G coefficients, summed over the CTAs in fixed order
                const int64_t lb0 = (k * b) / G, lb1 = (k * (b + 1)) / G;
                for (int64_t l = lb0; l < lb1; l += 4) {
                    double a4[4] = {0.0, 0.0, 0.0, 0.0};
                    for (int64_t bb = lane; bb < G; bb += 32)
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (l + j < lb1) {
                                const float2 hv = __ldcg(reinterpret_cast<const float2*>(p.hpart) + bb * p.d_max + l + j);
                                a4[j] += (double)hv.x + (double)hv.y;
                            }
#pragma unroll
                    for (int j = 0; j < 4; ++j) a4[j] = warp_sum_double(a4[j]);
                    if (lane == 0)
                        for (int j = 0; j < 4; ++j)
                            if (l + j < lb1) p.h[l + j] = a4[j];
                }
                __syncwarp();
                if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p.hcnt) : "memory");
                ++hround;
                if (!wait_counter(p.hcnt, p.bar, (uint32_t)G * hround, p.wait_ns)) {
                    if (lane == 0) loop_abort(ctl, p.bar, ST_ETIMEOUT);
                    ok = false;
                }
                // h (every CTA, same order): ||h||^2, and its split for the corrections of this pass
                // and the first stream of the next basis
                for (int64_t l0 = 0; l0 < k; l0 += 32 * 16) {
                    double hv[16];  // all loads in flight before the shared-memory stores
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t l = l0 + lane + 32 * j;
                        hv[j] = (ok && l < k) ? __ldcg(&p.h[l]) : 0.0;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t l = l0 + lane + 32 * j;
                        hh += hv[j] * hv[j];
                        if (l < k) split_f64_fast(hv[j], cah[l], cal[l]);
                    }
                }
                hh = warp_sum_double(hh);
            }
            nu2 = warp_sum_double(nu2);
            fs = warp_sum_double(fs);
            if (lane == 0) {
                // nu^2 = ||v1||^2 - ||h||^2 (accurate while ||h|| << ||v1||, which the numerical-rank
                // floor guarantees: past it both are rounding noise, and the no-tolerance mode that
                // runs there takes the four-barrier kernel)
                const double nuv = sqrt(fmax(nu2 - hh, 0.0));
                const double frol = sqrt(fmax(fs, 0.0));
                const double xin = sqrt(xn2p);
                int32_t st = STOP_NONE;
                if (k > 0) {
                    if (mode == MODE_FRO_REL) {
                        if (frol <= fro_tol) st = STOP_TOL;
                    } else if (nuv <= eps_r) {
                        st = STOP_TOL;
                    }
                }
                if (st == STOP_NONE && k >= p.d_max) st = STOP_DMAX;
                if (st == STOP_NONE && (nuv < eps_r22 || !(nuv > rank_floor_of(mode) * xin))) st = STOP_BREAK;
                bcast[0] = nuv;
                bcast[1] = recip_pos(nuv);
                bcast[2] = hh;
                vfl[6] = hh > ldexp(nuv * nuv, -58) ? 1 : 0;  // the flush corrections in float-float
                vfl[1] = st;
                if (b == 0) {
                    if (k > 0) {
                        p.err[k - 1] = nuv;
                        ctl->err_last = nuv;
                        ctl->fro_last = frol;
                    }
                    if (st == STOP_NONE) {
                        p.pivots[k] = piv;
                        if (p.nu_out) p.nu_out[k] = nuv;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(svcb);
            dec = vfl[1];
        } else if (warp == PROD) {
            if (lane == 0 && run_pass) {
                int64_t g = L0 / NT, t = L0 - (L0 / NT) * NT;
                int64_t issued = nunits;
                if (ok) {
                    fence_proxy_async_global();  // the v1 tiles every CTA wrote before barrier 1
                    // Every unit, X part and pivot-vector part; the first units' X tiles were
                    // prefetched into L2 during the orthogonalisation (issuing them into the ring
                    // before barrier 1 would load the memory system the barrier's atomics cross).
                    for (int64_t i = 0; i < nunits; ++i) {
                        if (mbar_test_wait(svcb, spar) && vfl[1] != STOP_NONE) {
                            issued = i;  // the basis was rejected: stop streaming
                            break;
                        }
                        if (preuse && !mbar_wait(&empty[ps], pph ^ 1u, p.wait_ns)) {
                            loop_abort(ctl, p.bar, ST_ETIMEOUT);
                            ok = false;
                            issued = i;
                            break;
                        }
                        const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                        const uint32_t xi_bytes = 2u * rows * 4u;
                        const uint32_t x_bytes = (uint32_t)(C * UB) * rows;
                        float* st = stages + (size_t)ps * STAGE;
                        mbar_arrive_expect_tx(&full[ps], x_bytes);
                        bulk_g2s(st + XI, planes + (g * p.group_stride + t * p.tile_stride) * Cfg::ESIZE, x_bytes,
                                 &full[ps], pol_x);
                        mbar_arrive_expect_tx(&full[ps], xi_bytes);
                        bulk_g2s(st, p.vs + t * 2 * MT, xi_bytes, &full[ps], pol_v);
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
                } else {
                    issued = 0;
                }
                vfl[3] = (int)issued;
                __threadfence_block();
                vfl[4] = (int)(k + 1);
            }
            __syncwarp();
            if (ok && !mbar_wait(svcb, spar, p.wait_ns)) {
                if (lane == 0) loop_abort(ctl, p.bar, ST_ETIMEOUT);
                ok = false;
            }
            dec = vfl[1];
        } else {
            // ---------------- consumers: the pass ----------------
            bool have_dec = false;
            auto get_dec = [&]() {  // uniform call sites; one reader, then a barrier
                if (have_dec) return;
                if (tid == 0) {
                    int d = STOP_NONE;
                    if (ok && !mbar_wait(svcb, spar, p.wait_ns)) {
                        loop_abort(ctl, p.bar, ST_ETIMEOUT);
                    } else {
                        d = vfl[1];
                    }
                    vfl[5] = d;
                }
                named_bar(1, NCONS);
                dec = vfl[5];
                have_dec = true;
            };
            if (run_pass) {
                if (k > 0 && gtf0 <= glast) {
                    if (tid == 0) {
                        fence_proxy_async_global();  // the T rows other CTAs wrote in earlier bases
                        const uint32_t bytes = (uint32_t)(k * C * 4);
                        mbar_arrive_expect_tx(tfull, bytes);
                        bulk_g2s(tfb, p.tf + gtf0 * p.d_max * C, bytes, tfull, pol_y);
                    }
                    tf_pend = true;
                }
                float acc_s[CPW][4], acc_c[CPW][4];
#pragma unroll
                for (int qq = 0; qq < CPW; ++qq)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc_s[qq][e] = acc_c[qq][e] = 0.f;
                long long best_k = LLONG_MIN;  // running argmax of this lane's columns (lanes < CPW)
                int64_t best_j = INT64_MAX;
                double e_old = 0.0;            // e_j of this lane's column of the current group
                int gbuf = 0;
                bool cut = false;
                double* gsum_k = p.gsum + (k & 1) * p.ngroups;
                int64_t g_next = L0 / NT, t_next = L0 - (L0 / NT) * NT;
                for (int64_t u = L0; u < L1; ++u) {
                    const int64_t g = g_next, t = t_next;
                    const int s = cs;
                    const uint32_t ph = cph;
                    if (++cs == S) {
                        cs = 0;
                        cph ^= 1u;
                    }
                    if (++t_next == NT) {
                        t_next = 0;
                        ++g_next;
                    }
                    // Wait for the unit, unless the producer stopped issuing before it (a basis the
                    // service warp rejected: the producer sees the decision before the consumers
                    // reach a finalised group).  Every consumer thread reaches the same verdict: the
                    // unit either arrives or is known never to be issued.
                    bool got = true;
                    if (ok && !mbar_try_wait(&full[s], ph)) {
                        const uint64_t t0 = globaltimer_ns();
                        while (true) {
                            if (mbar_try_wait(&full[s], ph)) break;
                            if (vfl[4] == (int)(k + 1) && (u - L0) >= (int64_t)vfl[3]) {
                                got = false;
                                break;
                            }
                            if (globaltimer_ns() - t0 > p.wait_ns) {
                                loop_abort(ctl, p.bar, ST_ETIMEOUT);
                                ok = false;
                                break;
                            }
                        }
                    }
                    if (!got) {
                        // nothing further is in flight; the stage sequence stays aligned with the
                        // producer's, which issued nothing from here
                        cs = s;
                        cph = ph;
                        break;
                    }
                    if (cut) {
                        // the basis was rejected: drain without arithmetic
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[s]);
                        continue;
                    }
                    const int64_t c0 = g * C;
                    const int ncols = (int)min((int64_t)C, p.n - c0);
                    if (lane < CPW && (t == 0 || u == L0) && warp * CPW + lane < ncols)
                        e_old = __ldcg(&p.e[c0 + warp * CPW + lane]);
                    const int rows = (int)min((int64_t)MT, p.ldp - t * MT);
                    if (ok) {
                        const float* st = stages + (size_t)s * STAGE;
                        if constexpr (XT == 2) {
                            if (rows == MT)
                                consume_tile_bf16<CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c);
                            else
                                consume_tile_bf16<CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c);
                        } else if constexpr (XT == 3) {
                            if (rows == MT)
                                consume_tile_f32acc<CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c);
                            else
                                consume_tile_f32acc<CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c);
                        } else {
                            if (rows == MT)
                                consume_tile<Cfg::PL, CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c);
                            else
                                consume_tile<Cfg::PL, CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[s]);
                    if (t != NT - 1 && u != L1 - 1) continue;

                    // ---------------- end of this CTA's share of column group g ----------------
                    // Each column's total over the warp (xor butterfly, a fixed order per lane); lane q
                    // then finalises the warp's column q, so that the FP64 steps of the two columns run
                    // side by side (dependent FP64 instructions are slow on this part).
                    float ts = 0.f, tc = 0.f;
#pragma unroll
                    for (int qq = 0; qq < CPW; ++qq) {
                        float sq = acc_s[qq][0], cq = acc_c[qq][0];
#pragma unroll
                        for (int e = 1; e < 4; ++e) ff_add(sq, cq, acc_s[qq][e], acc_c[qq][e]);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const float s2 = __shfl_xor_sync(0xffffffffu, sq, o);
                            const float c2 = __shfl_xor_sync(0xffffffffu, cq, o);
                            ff_add(sq, cq, s2, c2);
                        }
                        if (lane == qq) {
                            ts = sq;
                            tc = cq;
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc_s[qq][e] = acc_c[qq][e] = 0.f;
                    }
                    const int cwl = warp * CPW + lane;  // this lane's column of the group (lanes < CPW)
                    const bool colv = lane < CPW && cwl < ncols;
                    double tot = colv ? ff_to_double(ts, tc) : 0.0;
                    const bool tf_here = k > 0 && g >= gtf0;  // this group's T block was streamed
                    if (tf_here) {
                        if (ok && !mbar_wait(tfull, tcnt & 1u, p.wait_ns)) {
                            loop_abort(ctl, p.bar, ST_ETIMEOUT);
                            ok = false;
                        }
                        ++tcnt;
                        tf_pend = false;
                    }
                    const bool whole = (g * NT >= L0) && ((g + 1) * NT <= L1);
                    bool fin_here = true;
                    if (!whole) {
                        // a group split between CTAs: publish this share; the last to arrive sums
                        // the shares in CTA order
                        const int64_t bfirst = unit_owner(g * NT, W, G);
                        const int64_t blast = unit_owner(g * NT + NT - 1, W, G);
                        const uint32_t ncontrib = (uint32_t)(blast - bfirst + 1);
                        const int64_t slot = b - bfirst;
                        if (colv) {
                            p.gslot[(g * p.KMAX + slot) * C + cwl] = tot;
                            __threadfence();
                        }
                        named_bar(1, NCONS);
                        if (tid == 0) vfl[2] = (atomicAdd(&p.gcnt[g], 1u) == ncontrib - 1);
                        named_bar(1, NCONS);
                        fin_here = vfl[2] != 0;
                        if (fin_here) {
                            __threadfence();
                            if (colv) {
                                // the shares in CTA order, four loads in flight at a time
                                double acc = 0.0;
                                for (uint32_t s0 = 0; s0 < ncontrib; s0 += 4) {
                                    double sv[4];
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        sv[q] = (s0 + q < ncontrib) ? __ldcg(&p.gslot[(g * p.KMAX + s0 + q) * C + cwl]) : 0.0;
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        if (s0 + q < ncontrib) acc += sv[q];
                                }
                                tot = acc;
                            }
                            if (tid == 0) p.gcnt[g] = 0;
                        }
                    }
                    if (fin_here) {
                        get_dec();
                        if (dec != STOP_NONE) {
                            cut = true;
                            continue;
                        }
                        const double inv_nu = bcast[1];
                        // correction -h' T(0:k, j) of the columns' dot products
                        if (k > 0 && vfl[6]) {
                            // ||h|| / nu > 2^-29: FP32 would leave more than FP64 rounding in T(k, j),
                            // and T(:, i) is the next bases' first sweep.  Float-float products of the
                            // split h with T read in FP64, lanes 0-15 of a warp on its first column,
                            // 16-31 on its second, summed over the half-warp in a fixed tree.
                            static_assert(CPW == 2, "one half-warp per column");
                            const int cw = warp * CPW + (lane >> 4);
                            float s = 0.f, cc = 0.f;
                            if (cw < ncols) {
                                const double* tcolj = p.T + (c0 + cw) * p.ldt;
                                for (int64_t l = lane & 15; l < k; l += 16) {
                                    float th, tl;
                                    split_f64_fast(__ldcg(&tcolj[l]), th, tl);
                                    ff_mac2(s, cc, th, tl, cah[l], cal[l]);
                                }
                            }
#pragma unroll
                            for (int o = 8; o > 0; o >>= 1) {
                                const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
                                const float c2 = __shfl_xor_sync(0xffffffffu, cc, o);
                                ff_add(s, cc, s2, c2);
                            }
                            // lane 0 holds column 0's sum, lane 16 column 1's: to lanes 0 and 1
                            const float s1 = __shfl_sync(0xffffffffu, s, 16), c1 = __shfl_sync(0xffffffffu, cc, 16);
                            if (lane == 1) {
                                s = s1;
                                cc = c1;
                            }
                            if (colv) tot -= ff_to_double(s, cc);
                        } else if (k > 0) {
                            // FP32: the term is ||h|| / nu <= 2^-29 relative to the column's norm
                            const int c = tid % C, ls = tid / C;
                            float sacc = 0.f;
                            if (tf_here) {
                                for (int64_t l = ls; l < k; l += NLS) sacc = __fmaf_rn(cah[l], tfb[l * C + c], sacc);
                            } else {
                                const float* tg = p.tf + g * p.d_max * C;
                                for (int64_t l = ls; l < k; l += NLS) sacc = __fmaf_rn(cah[l], __ldcg(&tg[l * C + c]), sacc);
                            }
                            sacc = __fadd_rn(sacc, __shfl_xor_sync(0xffffffffu, sacc, 16));
                            if (lane < 16) corr[warp * C + lane] = sacc;
                            named_bar(1, NCONS);
                            if (colv) {
                                float cr = 0.f;
#pragma unroll
                                for (int w = 0; w < NW; ++w) cr = __fadd_rn(cr, corr[w * C + cwl]);
                                tot -= (double)cr;
                            }
                        }
                        if (colv) {
                            const int64_t j = c0 + cwl;
                            const double cj = tot * inv_nu;
                            p.T[j * p.ldt + k] = cj;
                            p.tf[(g * p.d_max + k) * C + cwl] = __double2float_rn(cj);
                            const double en = (j == piv) ? 0.0 : fmax(e_old - cj * cj, 0.0);
                            p.e[j] = en;
                            grp_e[gbuf * C + cwl] = en;
                            const long long ek = __double_as_longlong(en);  // e >= 0: ordered as integers
                            if (better_key(ek, j, best_k, best_j)) {
                                best_k = ek;
                                best_j = j;
                            }
                        }
                        named_bar(1, NCONS);
                        // the group's sum of e_j: warp 0, a fixed tree over the group's columns
                        if (warp == 0) {
                            double sv = (lane < ncols && lane < C) ? grp_e[gbuf * C + lane] : 0.0;
#pragma unroll
                            for (int o = C / 2; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
                            if (lane == 0) gsum_k[g] = sv;
                        }
                        gbuf ^= 1;
                    }
                    // the next group's T block (the buffer was read before the last barrier)
                    if (k > 0 && g >= gtf0 && g + 1 <= glast) {
                        if (tid == 0) {
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            const uint32_t bytes = (uint32_t)(k * C * 4);
                            mbar_arrive_expect_tx(tfull, bytes);
                            bulk_g2s(tfb, p.tf + (g + 1) * p.d_max * C, bytes, tfull, pol_y);
                        }
                        tf_pend = true;
                    }
                }
                get_dec();  // a CTA that finalised no group learns the decision here
                if (dec == STOP_NONE) {
#pragma unroll
                    for (int o = 1; o < CPW; o <<= 1) {
                        const long long ok2 = __shfl_xor_sync(0xffffffffu, best_k, o);
                        const int64_t oj2 = __shfl_xor_sync(0xffffffffu, best_j, o);
                        if (better_key(ok2, oj2, best_k, best_j)) {
                            best_k = ok2;
                            best_j = oj2;
                        }
                    }
                    if (lane == 0) {
                        red_e[warp] = __longlong_as_double(best_k);
                        red_j[warp] = best_j;
                    }
                    named_bar(1, NCONS);
                    if (tid == 0) {
                        long long bk = LLONG_MIN;
                        int64_t bj = INT64_MAX;
                        for (int w = 0; w < NW; ++w) {
                            const long long wk = __double_as_longlong(red_e[w]);
                            if (better_key(wk, red_j[w], bk, bj)) {
                                bk = wk;
                                bj = red_j[w];
                            }
                        }
                        p.pbest_e[b] = __longlong_as_double(bk);  // the key's bits (e_j itself, or none)
                        p.pbest_j[b] = bj;
                    }
                }
            } else {
                get_dec();
            }
            if (dec == STOP_NONE && ok) {
                // the Y chunks of the next basis's first stream (columns 0..k-1 are complete; column
                // k is formed there) into the ring, which every consumer has left
                const int64_t ncol2 = k, nch2 = ceil_div(ncol2, (int64_t)LC);
                const int64_t tot2 = (nch2 <= NB) ? nch2 : 2 * nch2;
                ypre = min((int64_t)NB, tot2);
                if (tid == 0 && ypre > 0) fence_proxy_async_global();
                for (int64_t u = 0; u < ypre; ++u) y_issue(u, ncol2, nch2);
            }
        }
        // every role leaves the loop together: the decision as the service warp wrote it, read by
        // all threads after one CTA barrier (a role's own copy can differ only after a timeout)
        __syncthreads();
        dec = vfl[1];
        if (dec != STOP_NONE) {
            stop = dec;
            break;
        }
        if (!grid_sync(p.bar, (uint32_t)G, gen, &sfl[0], ctl, p.wait_ns)) break;  // barrier 2 (uniform result)

        // ---------------- A: argmax over CTAs ----------------
        if (warp == 0) {
            // keys compared as integers: e_j >= 0, whose FP64 bit patterns order like the values
            // every candidate load in flight before the comparisons: in a loop whose trip count the
            // compiler cannot see, each round trip to L2 would wait for the one before
            constexpr int SL = kLoopMaxCtas / 32;
            long long ckv[SL];
            int64_t cjv[SL];
#pragma unroll
            for (int i = 0; i < SL; ++i) {
                const int64_t cb = lane + 32 * i;
                ckv[i] = (cb < G) ? __ldcg(reinterpret_cast<const long long*>(&p.pbest_e[cb])) : LLONG_MIN;
                cjv[i] = (cb < G) ? __ldcg(reinterpret_cast<const long long*>(&p.pbest_j[cb])) : INT64_MAX;
            }
            long long bk = LLONG_MIN;
            int64_t bj = INT64_MAX;
#pragma unroll
            for (int i = 0; i < SL; ++i)
                if (better_key(ckv[i], cjv[i], bk, bj)) {
                    bk = ckv[i];
                    bj = cjv[i];
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const long long ok2 = __shfl_down_sync(0xffffffffu, bk, o);
                const int64_t oj = __shfl_down_sync(0xffffffffu, bj, o);
                if (better_key(ok2, oj, bk, bj)) {
                    bk = ok2;
                    bj = oj;
                }
            }
            if (lane == 0) red_j[0] = (bj >= 0 && bj < p.n) ? bj : piv;
        }
        __syncthreads();
        piv = red_j[0];
        {
            const double nuv = bcast[0];
            inv_prev = bcast[1];
            small_h = bcast[2] <= ldexp(nuv * nuv, -72);
        }
        if (b == 0 && tid == 0) {
            ctl->d = k + 1;
            ctl->pivot = piv;
        }
        __syncthreads();
    }

    // ---------------- leave: no bulk copy may still be writing this CTA's shared memory ----------------
    if (warp == PROD && lane == 0) {
        for (int s = 0; s < S; ++s)
            if ((iss_mask >> s) & 1u)
                if (!mbar_wait(&full[s], (iss_par >> s) & 1u)) {
                    raise_status(ctl, ST_ETIMEOUT);
                    break;
                }
    }
    if (warp < NW && tid == 0) {
        for (int bf = 0; bf < NB; ++bf)
            if ((ypend >> bf) & 1u)
                if (!mbar_wait(&ybar[bf], (ypar >> bf) & 1u)) raise_status(ctl, ST_ETIMEOUT);
        if (tf_pend && !mbar_wait(tfull, tcnt & 1u)) raise_status(ctl, ST_ETIMEOUT);
    }
    if (b == 0 && tid == 0 && stop != STOP_NONE) {
        ctl->stop = stop;
        ctl->d = k;
        ctl->pivot = piv;
    }
}

size_t defer_smem_bytes(int xt, int R, int KC) {
    if (xt == 0) return defer_smem_layout<TileCfg<0>>(R, KC).total;
    if (xt == 1) return defer_smem_layout<TileCfg<1>>(R, KC).total;
    if (xt == 2) return defer_smem_layout<TileCfg<2>>(R, KC).total;
    return 0;
}

// Y columns per streamed chunk; at most 252 so that the last chunk's two extra columns (the new
// basis vector and v1) still give every column a thread in the column dots.
int defer_chunk_cols(int xt, int RS) {
    const int lc = (xt == 0) ? loop_chunk_cols<TileCfg<0>>(RS) : (xt == 1) ? loop_chunk_cols<TileCfg<1>>(RS)
                 : (xt == 2) ? loop_chunk_cols<TileCfg<2>>(RS) : 0;
    return lc < 252 ? lc : 252;
}

// xt 0..2: the storage type; 3: FP32 storage with FP32 accumulation in the pass
static const void* defer_fn(int xt) {
    return (xt == 0) ? (const void*)defer_kernel<0> : (xt == 1) ? (const void*)defer_kernel<1>
         : (xt == 2) ? (const void*)defer_kernel<2> : (const void*)defer_kernel<3>;
}

cudaError_t defer_kernel_setup(int max_smem) {
    cudaError_t e = cudaSuccess;
    for (int xt = 0; xt < 4 && e == cudaSuccess; ++xt)
        e = cudaFuncSetAttribute(defer_fn(xt), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

cudaError_t launch_defer(const Work& w, const void* X, double* Y, int64_t ldy, double* T, int64_t ldt,
                         int64_t* pivots, double* err, double* nu_out, int64_t k0, cudaStream_t st) {
    DeferParams p;
    p.m = w.m;
    p.n = w.n;
    p.ldp = w.ldp;
    p.ldx = w.ldx;
    p.ldt = ldt;
    p.ldy = ldy;
    p.d_max = w.d_max;
    p.k0 = k0;
    p.xt = w.xt;
    p.planes = static_cast<const unsigned char*>(w.planes);
    p.group_stride = w.group_stride;
    p.tile_stride = w.tile_stride;
    p.NT = w.NT;
    p.ngroups = w.ngroups;
    p.W = w.W;
    p.KMAX = w.KMAX;
    p.evict_first = w.evict_first;
    p.X = X;
    p.Y = Y;
    p.T = T;
    p.pivots = pivots;
    p.err = err;
    p.nu_out = nu_out;
    p.ctl = w.ctl;
    p.bar = &w.ctl->bar[0];
    p.hcnt = &w.ctl->bar[1];
    p.hdone = &w.ctl->bar[2];
    p.e = w.e;
    p.xn2 = w.xn2;
    p.ysb = w.ysb;
    p.vs = w.v2s;
    p.tf = w.tf;
    p.hpart = w.hpart;
    p.h = w.h;
    p.nu2part = w.nu2part;
    p.pbest_e = w.pbest_e;
    p.pbest_j = w.pbest_j;
    p.gcnt = w.gcnt;
    p.gslot = w.gslot;
    p.gsum = w.gsum;
    p.R = w.R;
    p.RS = w.RS;
    p.LC = w.LC;
    p.KC = w.KC;
    p.wait_ns = wait_limit_ns(kWaitLimitNs);
    void* args[] = {&p};
    const int threads =
        32 + ((w.xt == 0) ? TileCfg<0>::THREADS : (w.xt == 1) ? TileCfg<1>::THREADS : TileCfg<2>::THREADS);
    return cudaLaunchCooperativeKernel(defer_fn((w.xt == 1 && w.acc32) ? 3 : w.xt), dim3((unsigned)w.G_loop),
                                       dim3((unsigned)threads), args, w.loop_smem, st);
}

}  // namespace rbd
