// rbd_loop.cu -- the whole greedy loop of Algorithm 1 in ONE persistent cooperative kernel.
//
// One CTA per SM (8 consumer warps + 1 producer warp), all co-resident (cooperative launch), so
// the steps of the loop are separated by grid-wide barriers instead of kernel launches.  Every
// barrier and every mbarrier wait is bounded in time (kWaitLimitNs); a wait that runs out raises
// RBD_ETIMEOUT in the control block and sets the abort bit of the barrier word, and all CTAs leave
// the loop at their next barrier.
//
// Per basis k (k = 0 .. d_max; the last iteration only certifies E_cur and stops):
//   O1   v1 = x_i - Y t, t = T(0:k, i)            rows of this CTA's block, float-float
//   O1'  hpart[b] = Y_b' v1_b                      this CTA's partial re-orthogonalisation sums
//   ---- grid barrier 1
//   O2   h = sum_b hpart[b] (fixed order)          each CTA reduces k / G coefficients
//   ---- grid barrier 2
//   O3   v2 = v1 - Y h,  ||v2||^2 partial          float-float, as O1
//   ---- grid barrier 3
//   D    nu = ||v2|| (every CTA, fixed order); E_cur of basis k-1 = nu (the FP64 residual of the
//        column that maximised the indicator); stop tests of steps 2.4 and 2.2, identical in
//        every CTA; 1 / nu once for the pass
//   P    the fused pass (rbd_tile.cuh): T(k, :), e_j, per-CTA argmax; Y(:, k) = v2 / nu for
//        this CTA's rows
//   ---- grid barrier 4
//   A    argmax over the CTAs (every CTA); the Frobenius residual of the basis (fixed order) is
//        summed by CTA 0's producer warp during the next O1, off the critical path
//
// The A-norm form (Section 3.2, A = diag(w)) keeps this basis and T, and measures the indicator
// in ||.||_A.  Adding xi_k changes ||r_j||_A^2 by -2 c_j xi_k' A r_j + c_j^2 xi_k' A xi_k, and
// xi_k' A r_j = z' x_j with z = (I - Y Y')(w o xi_k) because r_j = (I - Y Y') x_j.  So the pass
// takes a second dot product per element, with z, and three phases come before it:
//   O3'  u = w o v2, ||v2||_A^2 partial, g_b = Y_b' u_b   (with O3, before barrier 3)
//   D    E_cur and the tolerance tests take ||v2||_A
//   O4   g = sum_b g_b, k / G coefficients per CTA;  ---- grid barrier 3b
//   O5   z = u - Y g for this block's rows (nu is applied in the pass);  ---- grid barrier 3c
//
// This is classical Gram-Schmidt applied twice (see rbd_orth.cu for why, and for its accuracy);
// Y is kept as a split FP32 copy stored ROW-BLOCK-MAJOR (block b = this CTA's R rows, columns
// RS >= R floats apart, all contiguous), so each CTA streams only its own slice of Y, with bulk
// copies, and no other CTA ever reads it.  X never changes: the producer prefetches the first tiles of the next
// pass into L2 while the orthogonalisation runs and into shared memory after barrier 3; only the
// pivot-vector tiles wait for O3.
#include <algorithm>
#include <type_traits>

#include "rbd_device.cuh"
#include "rbd_loop.cuh"
#include "rbd_tile.cuh"
#include "rbd_work.h"

namespace rbd {

struct LoopParams {
    int64_t m, n, ldp, ldx, ldt, ldy, d_max;
    int64_t k0;           // first basis index of this launch (0, or d0 when resuming)
    int xt;
    // X planes (tile-major) and pass geometry
    const unsigned char* planes;
    int64_t group_stride, tile_stride, NT, ngroups, W;
    int KMAX;
    int evict_first;
    // caller buffers
    const void* X;
    double* Y;
    double* T;
    int64_t* pivots;
    double* err;
    double* nu_out;
    const double* wts;    // A-norm form: the m weights of A = diag(wts)
    // workspace
    Ctl* ctl;
    uint32_t* bar;        // grid barrier {count, generation}
    double* e;
    const double* xn2;
    float* ysb;           // [G][2][d_max][RS] split Y, row-block-major
    float* v2s;           // tile-interleaved split v2 (pivot-vector tiles of the pass)
    float* zs;            // A-norm form: tile-interleaved split z (second pivot vector)
    double* hpart;        // [G][d_max]
    double* h;            // [d_max]
    double* nu2part;      // [2 G]: ||v2||^2 partials, then (A-norm form) ||v2||_A^2 partials
    double* pbest_e;      // [G]
    int64_t* pbest_j;     // [G]
    uint32_t* gcnt;
    double* gslot;
    double* gslot2;       // A-norm form: group partials of the dot products with z
    double* gsum;
    uint64_t wait_ns;     // bound on every wait of the loop (the exit drain keeps kWaitLimitNs)
    int R;                // rows per CTA block (multiple of 4, <= kLoopMaxRows)
    int RS;               // column stride of a Y slice (R or R + 4, RS = 4 mod 8: see loop_slice_stride)
    int LC;               // Y columns per streamed chunk (multiple of 4)
};

// ------------------------------------------------------------------------------------------
// shared-memory layout (host and device agree through this function)
// ------------------------------------------------------------------------------------------
struct LoopSmem {
    size_t bars, v1s, v2own, part, coef, v1split, scratch, total;
};

template <class Cfg>
__host__ __device__ inline LoopSmem loop_smem_layout(int R, int LC) {
    LoopSmem s;
    size_t o = (size_t)Cfg::S * Cfg::STAGE_FLOATS * 4;  // the ring: pass stages / Y chunks
    s.bars = o;
    o += (size_t)(3 * Cfg::S) * 8;                // full, empty, ybar
    o = (o + 15) & ~size_t(15);                   // 16-byte loads from the regions below
    s.v1s = o;
    o += (size_t)R * 8;
    s.v2own = o;
    o += (size_t)R * 8;
    s.part = o;
    o += (size_t)8 * (Cfg::NW * 32) * 4;          // partial sums of the slice GEMVs (8 NCONS floats)
    s.coef = o;
    o += (size_t)Cfg::S * 2 * LC * 4;             // per ring buffer: (hi, lo) x LC
    s.v1split = o;
    o += (size_t)2 * R * 4;
    s.scratch = o;
    o += (size_t)(2 * Cfg::NW + 2 * Cfg::C + 8) * 8;
    s.total = (o + 127) & ~size_t(127);
    return s;
}

// Streams columns [0, k) of this CTA's Y slice, LC columns at a time, through NB buffers made
// of consecutive stages of the pass ring (idle during the orthogonalisation), up to NB chunks in flight.
// Bulk copies are issued by consumer thread 0 and complete on ybar[buffer]; body(yh, yl, ch,
// cl, l0, lc) runs for each chunk with all consumers; load_coef(l, hi, lo) gives the
// coefficient of column l (staged in shared memory next to the chunk).  np = planes streamed.
struct YStream {
    float* ring;        // NB buffers of buf_floats floats
    int buf_floats;
    int NB;
    uint64_t* ybar;     // NB barriers
    float* coef;        // NB x 2 x LC
    const float* ysb_b; // this CTA's block of the split Y
    int64_t d_max;
    int R, LC;          // R: column stride of the slice (floats)
    uint64_t pol;
    uint32_t* bar;      // grid-barrier word (abort bit on a timeout)
    uint32_t count;     // chunks streamed so far (all calls): fixes each chunk's buffer and parity
    bool loaded;        // the slice of this step is resident in the ring
    int64_t nloaded;
    bool* ok;
    uint64_t wait_ns;
    uint32_t nissued;   // chunks issued so far (consumer thread 0) and chunks waited: at exit the
    uint32_t nwaited;   // ones in between are still landing in the ring
};

template <int NCONS, class Coef, class Body>
__device__ __forceinline__ void ystream(YStream& ys, int64_t k, int np, int tid, Ctl* ctl, Coef&& load_coef,
                                        Body&& body) {
    const int64_t nch = ceil_div(k, ys.LC);
    if (nch == 0) return;
    const int plane = ys.LC * ys.R;  // floats: offset of plane 1 inside a buffer
    auto bufof = [&](int64_t c) { return (int)((ys.count + (uint32_t)c) % (uint32_t)ys.NB); };
    auto issue = [&](int64_t c) {
        const int bf = bufof(c);
        const int64_t l0 = c * ys.LC;
        const int lc = (int)min((int64_t)ys.LC, k - l0);
        const uint32_t bytes = (uint32_t)lc * (uint32_t)ys.R * 4u;
        mbar_arrive_expect_tx(&ys.ybar[bf], (uint32_t)np * bytes);
        ys.nissued = max(ys.nissued, ys.count + (uint32_t)c + 1u);
        for (int pl = 0; pl < np; ++pl)
            bulk_g2s(ys.ring + (size_t)bf * ys.buf_floats + (size_t)pl * plane,
                     ys.ysb_b + ((int64_t)pl * ys.d_max + l0) * ys.R, bytes, &ys.ybar[bf], ys.pol);
    };
    auto stage_coef = [&](int64_t c) {
        const int bf = bufof(c);
        const int64_t l0 = c * ys.LC;
        const int lc = (int)min((int64_t)ys.LC, k - l0);
        for (int l = tid; l < lc; l += NCONS) {
            float hi, lo;
            load_coef(l0 + l, hi, lo);
            ys.coef[(bf * 2 + 0) * ys.LC + l] = hi;
            ys.coef[(bf * 2 + 1) * ys.LC + l] = lo;
        }
    };
    // Resident mode: when the whole slice fits in the ring (nch <= NB) it is loaded by the first
    // call of a step and reused by the later calls of the same step (ystream_end_step releases it).
    // A resident slice is never overwritten within the step and all its coefficients are staged
    // up front, so one barrier before the first chunk suffices; a streamed slice recycles its
    // buffers and synchronises per chunk.
    const bool resident = nch <= ys.NB;
    const bool reuse = resident && ys.loaded;
    const int64_t npre = min(nch, (int64_t)ys.NB);
    if (tid == 0 && !reuse)
        for (int64_t c = 0; c < npre; ++c) issue(c);
    for (int64_t c = 0; c < npre; ++c) stage_coef(c);
    for (int64_t c = 0; c < nch; ++c) {
        if (!resident || c == 0)
            named_bar(1, NCONS);  // coefficients visible; chunk c-1 consumed, so its buffer is free
        if (!resident && c >= 1 && c - 1 + ys.NB < nch) {
            if (tid == 0) issue(c - 1 + ys.NB);
            stage_coef(c - 1 + ys.NB);
        }
        const int bf = bufof(c);
        const uint32_t par = ((ys.count + (uint32_t)c) / (uint32_t)ys.NB) & 1u;
        if (!reuse && *ys.ok) {
            if (mbar_wait(&ys.ybar[bf], par, ys.wait_ns)) {
                ys.nwaited = max(ys.nwaited, ys.count + (uint32_t)c + 1u);
            } else {
                loop_abort(ctl, ys.bar, ST_ETIMEOUT);
                *ys.ok = false;
            }
        }
        const int64_t l0 = c * ys.LC;
        const int lc = (int)min((int64_t)ys.LC, k - l0);
        if (*ys.ok)
            body(ys.ring + (size_t)bf * ys.buf_floats, ys.ring + (size_t)bf * ys.buf_floats + plane,
                 ys.coef + (bf * 2) * ys.LC, ys.coef + (bf * 2 + 1) * ys.LC, l0, lc);
    }
    named_bar(1, NCONS);  // the last chunk is consumed before the ring is reused
    if (resident) {
        ys.loaded = true;
        ys.nloaded = nch;
    } else {
        ys.count += (uint32_t)nch;
    }
}

// End of the orthogonalisation of a step: a resident slice gives its buffers back to the ring.
__device__ __forceinline__ void ystream_end_step(YStream& ys) {
    if (ys.loaded) {
        ys.count += (uint32_t)ys.nloaded;
        ys.loaded = false;
        ys.nloaded = 0;
    }
}

// The storage type XT fixes the tile shape; WT selects the A-norm form (Section 3.2, A = diag(w)):
// a second pivot vector z = (I - Y Y')(w o v2) in the pass and three more phases per basis.
template <int XT, bool WT>
using LoopCfg = std::conditional_t<WT, TileCfgW<XT>, TileCfg<XT>>;

template <int XT, bool WT>
__global__ void __launch_bounds__(TileCfg<XT>::THREADS, 1) loop_kernel(LoopParams p) {
    using Cfg = LoopCfg<XT, WT>;
    constexpr int UB = Cfg::PL * Cfg::ESIZE;  // X bytes per element and column of a unit
    constexpr int NW = Cfg::NW, CPW = Cfg::CPW, C = Cfg::C, MT = Cfg::MT, S = Cfg::S;
    constexpr int XI = Cfg::XI_FLOATS, STAGE = Cfg::STAGE_FLOATS;
    constexpr int NCONS = NW * 32;
    constexpr int MAXRPT = kLoopMaxRows / NCONS;  // rows per consumer thread when R > NCONS

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const LoopSmem L = loop_smem_layout<Cfg>(p.R, p.LC);
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L.bars);
    uint64_t* empty = full + S;
    uint64_t* ybar = empty + S;
    double* v1s = reinterpret_cast<double*>(smem_raw + L.v1s);
    double* v2own = reinterpret_cast<double*>(smem_raw + L.v2own);
    double* part = reinterpret_cast<double*>(smem_raw + L.part);
    float* coef = reinterpret_cast<float*>(smem_raw + L.coef);
    float* v1h = reinterpret_cast<float*>(smem_raw + L.v1split);
    float* v1l = v1h + p.R;
    double* red_e = reinterpret_cast<double*>(smem_raw + L.scratch);  // NW
    int64_t* red_j = reinterpret_cast<int64_t*>(red_e + NW);          // NW
    double* grp_e = reinterpret_cast<double*>(red_j + NW);           // 2 C
    double* bcast = grp_e + 2 * C;                                   // 4 doubles
    int* sflags = reinterpret_cast<int*>(bcast + 4);                 // 8 ints

    Ctl* ctl = p.ctl;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int R = p.R, RS = p.RS;
    const int64_t r0 = b * (int64_t)R;
    const int Rb = (int)max((int64_t)0, min((int64_t)R, p.ldp - r0));  // rows of this block within ldp
    const int64_t W = p.W, NT = p.NT;
    const int64_t L0 = (W * b) / G, L1 = (W * (b + 1)) / G;
    const int64_t nunits = L1 - L0;

    if (ctl->status != 0 || ctl->stop != 0) return;  // set by the initial pass, uniform

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 2);    // X part and pivot-vector part arrive separately
            mbar_init(&empty[s], NW);
            mbar_init(&ybar[s], 1);    // Y chunks streamed through the same buffers
        }
        fence_mbar_init();
    }
    __syncthreads();

    bool ok = true;
    uint32_t gen = 0;
    YStream ys;
    ys.ring = stages;
    ys.buf_floats = loop_ybuf_stages<Cfg>(RS) * STAGE;
    ys.NB = S / loop_ybuf_stages<Cfg>(RS);
    ys.ybar = ybar;
    ys.coef = coef;
    ys.ysb_b = p.ysb + b * 2 * p.d_max * (int64_t)RS;
    ys.d_max = p.d_max;
    ys.R = RS;
    ys.LC = p.LC;
    ys.pol = l2_policy_evict_normal();
    ys.bar = p.bar;
    ys.count = 0;
    ys.loaded = false;
    ys.nloaded = 0;
    ys.ok = &ok;
    ys.wait_ns = p.wait_ns;
    ys.nissued = 0;
    ys.nwaited = 0;
    uint32_t iss_par = 0, iss_mask = 0;  // producer: parity and presence of the last issue into each stage

    // pass pipeline state (producer and consumers advance identical copies)
    int ps = 0;
    uint32_t pph = 0;
    bool preuse = false;  // producer
    int cs = 0;
    uint32_t cph = 0;     // consumers
    int64_t npref = 0;    // producer: units of the next pass whose X tiles are in flight
    int pf_s0 = 0;        // stage and phase parity of the first prefetched unit
    uint32_t pf_ph0 = 0;

    int64_t piv = ctl->pivot;
    const int mode = ctl->mode;
    const double eps_r = ctl->eps_r, eps_r22 = ctl->eps_r22, fro_tol = ctl->fro_tol;
    const unsigned char* planes = p.planes;
    const uint64_t pol_x = p.evict_first ? l2_policy_evict_first() : l2_policy_evict_normal();
    const uint64_t pol_xi = l2_policy_evict_normal();

    int64_t k = p.k0;
    int32_t stop = STOP_NONE;
    double nu = 0.0;
    for (;; ++k) {

        // Rows in quads of 4 for the column dots (Rb is a multiple of 4): 16-byte shared-memory
        // loads, four float-float chains per thread, and with the slice stride RS = 4 mod 8 (RS / 4
        // odd) the 8 threads of a quarter-warp that read 8 consecutive columns of one quad hit 8
        // different 16-byte bank groups.
        const int NQ = Rb / 4;

        // GEMV over the slice: S_r = sum_{l<k} Y_b(r, l) coef(l) for this block's rows.  Thread
        // (rfirst, q) sums row rfirst over the columns l = q, q + NSUB, ... of each chunk in two
        // alternating float-float chains; the NSUB column subsets are added in FP64 in subset
        // order (v = x - S cancels heavily when the pivot nearly lies in span(Y), so S needs more
        // than a float-float combine of many partial sums).  fin(r, i, S_r) runs for every r < R
        // in thread r - i * NCONS = tid (S_r = 0 for rows >= Rb).  Consumers only.
        const int NSUB = (R <= NCONS) ? (NCONS / R) : 1;
        const int q = (R <= NCONS) ? (tid / R) : 0;
        const int rfirst = (R <= NCONS) ? (tid % R) : tid;
        const bool active = (warp < NW) && ((R <= NCONS) ? (tid < NSUB * R) : true);
        auto block_gemv = [&](auto&& load_coef, auto&& fin) {
            float as[MAXRPT], ac[MAXRPT], bs[MAXRPT], bc[MAXRPT];
#pragma unroll
            for (int i = 0; i < MAXRPT; ++i) as[i] = ac[i] = bs[i] = bc[i] = 0.f;
            if (k > 0) {
                ystream<NCONS>(ys, k, 2, tid, ctl, load_coef,
                               [&](const float* yh, const float* yl, const float* ch, const float* cl, int64_t, int lc) {
                                   if (!active) return;
#pragma unroll
                                   for (int i = 0; i < MAXRPT; ++i) {
                                       const int r = rfirst + i * NCONS;
                                       if (r >= Rb || (R <= NCONS && i > 0)) break;
                                       int l = q;
                                       for (; l + NSUB < lc; l += 2 * NSUB) {
                                           ff_mac2(as[i], ac[i], yh[l * RS + r], yl[l * RS + r], ch[l], cl[l]);
                                           ff_mac2(bs[i], bc[i], yh[(l + NSUB) * RS + r], yl[(l + NSUB) * RS + r],
                                                   ch[l + NSUB], cl[l + NSUB]);
                                       }
                                       if (l < lc) ff_mac2(as[i], ac[i], yh[l * RS + r], yl[l * RS + r], ch[l], cl[l]);
                                   }
                               });
            }
#pragma unroll
            for (int i = 0; i < MAXRPT; ++i) ff_add(as[i], ac[i], bs[i], bc[i]);
            if (R <= NCONS) {
                if (active) part[q * R + rfirst] = ff_to_double(as[0], ac[0]);
                named_bar(1, NCONS);
                if (tid < R) {
                    double acc = 0.0;
                    if (tid < Rb && k > 0)
                        for (int qq = 0; qq < NSUB; ++qq) acc += part[qq * R + tid];
                    fin(tid, 0, acc);
                }
            } else {
#pragma unroll
                for (int i = 0; i < MAXRPT; ++i) {
                    const int r = tid + i * NCONS;
                    if (r >= R) break;
                    fin(r, i, (r < Rb && k > 0) ? ff_to_double(as[i], ac[i]) : 0.0);
                }
            }
            named_bar(1, NCONS);
        };

        // out[b][l] = Y_b(:, l)' s_b for l < k, s_b = (v1h, v1l) of this block's rows (consumers).
        // One thread per (column, row segment): the chunk's lc columns times nseg = NCONS / lc
        // segments of the block's quads, combined in segment order through shared memory.
        auto block_dots = [&](double* out) {
            ystream<NCONS>(
                ys, k, 2, tid, ctl, [&](int64_t, float& hi, float& lo) { hi = lo = 0.f; },
                [&](const float* yh, const float* yl, const float*, const float*, int64_t l0, int lc) {
                    const int nseg = max(1, min(8, NCONS / lc));
                    const int sq = (NQ + nseg - 1) / nseg;
                    // 2 x nseg x lc <= 2 NCONS floats per chunk, double-buffered by chunk parity: the
                    // one barrier per chunk below then also orders the reads of chunk c before the
                    // writes of chunk c + 2
                    float* pf = reinterpret_cast<float*>(part) + (((l0 / ys.LC) & 1) ? 2 * NCONS : 0);
                    if (tid < nseg * lc) {
                        const int l = tid % lc, sg = tid / lc;
                        const int q0 = sg * sq, q1 = min(NQ, q0 + sq);
                        const float* ch = yh + l * RS;
                        const float* cl = yl + l * RS;
                        float s4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
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
                        pf[2 * (sg * lc + l)] = s4[0];
                        pf[2 * (sg * lc + l) + 1] = c4[0];
                    }
                    named_bar(1, NCONS);
                    if (tid < lc) {
                        float s0 = pf[2 * tid], c0 = pf[2 * tid + 1];
                        for (int sg = 1; sg < nseg; ++sg)
                            ff_add_acc(s0, c0, pf[2 * (sg * lc + tid)], pf[2 * (sg * lc + tid) + 1]);
                        out[b * p.d_max + l0 + tid] = ff_to_double(s0, c0);
                    }
                });
        };
        // dst[r] = v1s[r] - sum_{l<k} Y_b(r, l) coefv[l] for this block's rows (consumers; dst may be
        // v1s).  Float-float: when the pivot nearly lies in span(Y), v1 is tiny and the coefficients
        // are not small relative to it, so Y h needs the full precision for Y'Y = I to hold.
        auto block_sub = [&](const double* coefv, double* dst) {
            block_gemv([&](int64_t l, float& hi, float& lo) { split_double(__ldcg(&coefv[l]), hi, lo); },
                       [&](int r, int, double sv) { dst[r] = (r < Rb) ? v1s[r] - sv : 0.0; });
        };
        // split copy of this block's rows of src for the pass: tile t of dstv holds
        // [hi(rows_t) | lo(rows_t)] at t * 2 * MT (consumers).
        auto write_split = [&](const double* src, float* dstv) {
            for (int r = tid; r < Rb; r += NCONS) {
                const int64_t row = r0 + r;
                const int64_t t = row / MT;
                const int64_t rt = min((int64_t)MT, p.ldp - t * MT);
                const int64_t off = t * 2 * MT + (row - t * MT);
                float hi, lo;
                split_double(src[r], hi, lo);
                dstv[off] = hi;
                dstv[off + rt] = lo;
            }
            fence_proxy_async_global();  // read by bulk copies in the pass
        };
        // producer: the first X tiles of pass k into the ring (free once every consumer is done
        // with Y), ahead of the pivot-vector tiles.
        auto prefetch_x = [&]() {
            if (warp != NW || lane != 0 || k >= p.d_max || !ok) return;
            npref = min(nunits, (int64_t)S);
            pf_s0 = ps;
            pf_ph0 = pph;
            int64_t g = L0 / NT, t = L0 - (L0 / NT) * NT;
            for (int64_t i = 0; i < npref; ++i) {
                if (preuse && !mbar_wait(&empty[ps], pph ^ 1u, p.wait_ns)) {
                    loop_abort(ctl, p.bar, ST_ETIMEOUT);
                    ok = false;
                    npref = i;
                    break;
                }
                const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                const uint32_t x_bytes = (uint32_t)(C * UB) * rows;
                float* st = stages + (size_t)ps * STAGE;
                mbar_arrive_expect_tx(&full[ps], x_bytes);
                bulk_g2s(st + XI, planes + (g * p.group_stride + t * p.tile_stride) * Cfg::ESIZE, x_bytes, &full[ps],
                         pol_x);
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
        };

        // ---------------- O1 / O1': v1 = x_i - Y t, partial h = Y_b' v1_b ----------------
        if (warp < NW) {
            // the pivot column's rows of this block (row tid + i NCONS in thread tid), held in
            // registers so that the loads overlap the coefficient loads and the stream
            double xr[MAXRPT];
#pragma unroll
            for (int i = 0; i < MAXRPT; ++i) {
                const int r = tid + i * NCONS;
                xr[i] = (r < Rb && r0 + r < p.m) ? load_x_elem(p.X, p.xt, piv * p.ldx + r0 + r) : 0.0;
            }
            const double* tcol = p.T + piv * p.ldt;
            block_gemv([&](int64_t l, float& hi, float& lo) { split_double(__ldcg(&tcol[l]), hi, lo); },
                       [&](int r, int i, double sv) {
                           const double v = (r < Rb && r0 + r < p.m) ? xr[i] - sv : 0.0;
                           v1s[r] = v;
                           split_double(v, v1h[r], v1l[r]);
                       });
            named_bar_arrive(2, NCONS + 32);  // O1's loads are done
            if (k > 0) block_dots(p.hpart);
        } else {
            // The first tiles of pass k, into L2 once O1's loads are done, while HBM is otherwise
            // idle during the orthogonalisation; the bulk copies into shared memory before
            // barrier 3 then hit L2 and leave HBM quiet while the CTAs synchronise.
            named_bar(2, NCONS + 32);
            if (lane == 0 && k < p.d_max) {
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
        }
        if (k > 0 && b == 0 && warp == NW) {
            // Frobenius residual after basis k-1 (fixed order), off the critical path: the pass
            // wrote the per-group sums before barrier 4 of the last step; phase D reads it after
            // barrier 3 of this one
            double fs = 0.0;
#pragma unroll 8
            for (int64_t gg = lane; gg < p.ngroups; gg += 32) fs += __ldcg(&p.gsum[gg]);
            fs = warp_sum_double(fs);
            if (lane == 0) ctl->fro_last = sqrt(fmax(fs, 0.0));
        }
        if (k > 0) {
            if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;   // barrier 1
            if (!ok) break;
            // ---------------- O2: h(l) = sum_b hpart[b](l), k / G coefficients per CTA ----------------
            if (warp < NW) {
                const int64_t lb0 = (k * b) / G, lb1 = (k * (b + 1)) / G;
                for (int64_t l = lb0 + warp; l < lb1; l += NW) {
                    double acc = lane_sum_ctas(p.hpart + l, p.d_max, G, lane);
                    acc = warp_sum_double(acc);
                    if (lane == 0) p.h[l] = acc;
                }
            }
            if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;   // barrier 2
            if (!ok) break;
        }

        // ---------------- O3: v2 = v1 - Y h, ||v2||^2 partial ----------------
        if (warp < NW) {
            block_sub(p.h, v2own);
            write_split(v2own, p.v2s);
            if (warp == 0) {
                double acc = 0.0;
                for (int r = lane; r < Rb; r += 32) acc += v2own[r] * v2own[r];
                acc = warp_sum_double(acc);
                if (lane == 0) p.nu2part[b] = acc;
            }
            if constexpr (WT) {
                // ||v2||_A^2 of this block (fixed order), u = w o v2 (kept in v1s and split in
                // v1h / v1l, free after O3) and the partial g_b = Y_b' u_b
                if (warp == 1) {
                    double acc = 0.0;
                    for (int r = lane; r < Rb; r += 32)
                        if (r0 + r < p.m) acc += __ldg(&p.wts[r0 + r]) * (v2own[r] * v2own[r]);
                    acc = warp_sum_double(acc);
                    if (lane == 0) p.nu2part[G + b] = acc;
                }
                for (int r = tid; r < R; r += NCONS) {
                    const double u = (r < Rb && r0 + r < p.m) ? __ldg(&p.wts[r0 + r]) * v2own[r] : 0.0;
                    v1s[r] = u;
                    split_double(u, v1h[r], v1l[r]);
                }
                named_bar(1, NCONS);
                if (k > 0) block_dots(p.hpart);
            }
        }
        if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;  // barrier 3
        if (!ok) break;
        if constexpr (!WT) {
            // every consumer is past O3, so the ring is free: the first X tiles of the pass (L2
            // hits) load during the stop decision
            ystream_end_step(ys);
            prefetch_x();
        }

        // ---------------- D: nu, certified E_cur of basis k-1, stop tests ----------------
        // A-norm form: E_cur and the tests of steps 2.2 / 2.4 take ||v2||_A; xi = v2 / nu and the
        // numerical-rank floor stay Euclidean.
        if (warp == 0) {
            // independent loads first, so that their round trips overlap
            const double xn2p = (lane == 0) ? __ldg(&p.xn2[piv]) : 0.0;
            const double frol = (lane == 0 && k > 0 && mode == MODE_FRO_REL) ? __ldcg(&ctl->fro_last) : 0.0;
            double acc = lane_sum_ctas(p.nu2part, 1, G, lane), acc2 = 0.0;
            if constexpr (WT) acc2 = lane_sum_ctas(p.nu2part + G, 1, G, lane);
            acc = warp_sum_double(acc);
            if constexpr (WT) acc2 = warp_sum_double(acc2);
            if (lane == 0) {
                const double nuv = sqrt(acc);
                const double nea = WT ? sqrt(acc2) : nuv;
                const double xin = sqrt(xn2p);
                int32_t st = STOP_NONE;
                if (k > 0) {
                    if (mode == MODE_FRO_REL) {
                        if (frol <= fro_tol) st = STOP_TOL;
                    } else if (nea <= eps_r) {
                        st = STOP_TOL;
                    }
                }
                if (st == STOP_NONE && k >= p.d_max) st = STOP_DMAX;
                if (st == STOP_NONE && (nea < eps_r22 || !(nuv > rank_floor_of(mode) * xin))) st = STOP_BREAK;
                bcast[0] = nuv;
                const double inv = recip_pos(nuv);
                bcast[1] = inv;                                   // once, for every thread of the pass
                bcast[3] = (WT && acc > 0.0) ? acc2 * (inv * inv) : 1.0;  // xi' A xi
                sflags[1] = st;
                if (b == 0) {
                    if (k > 0) {
                        p.err[k - 1] = nea;
                        ctl->err_last = nea;
                    }
                    if (st == STOP_NONE) {
                        p.pivots[k] = piv;
                        if (p.nu_out) p.nu_out[k] = nuv;
                    }
                }
            }
        }
        __syncthreads();
        nu = bcast[0];
        const double qa = bcast[3];
        stop = sflags[1];
        if (stop != STOP_NONE) break;

        if constexpr (WT) {
            // ---------------- O4: g(l) = sum_b g_b(l), k / G coefficients per CTA ----------------
            if (k > 0) {
                if (warp < NW) {
                    const int64_t lb0 = (k * b) / G, lb1 = (k * (b + 1)) / G;
                    for (int64_t l = lb0 + warp; l < lb1; l += NW) {
                        double acc = lane_sum_ctas(p.hpart + l, p.d_max, G, lane);
                        acc = warp_sum_double(acc);
                        if (lane == 0) p.h[l] = acc;
                    }
                }
                if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;  // barrier 3b
                if (!ok) break;
            }
            // ---------------- O5: z = u - Y g for this block's rows ----------------
            if (warp < NW) {
                block_sub(p.h, v1s);
                write_split(v1s, p.zs);
            }
            ystream_end_step(ys);
            __syncthreads();
            prefetch_x();
            if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;  // barrier 3c
            if (!ok) break;
        }

        // ---------------- P: the fused pass of basis k ----------------
        const double inv_nu = bcast[1];
        // Y(:, k) = v2 / nu for this block's rows (user Y and the split row-block copy)
        for (int r = tid; r < Rb; r += Cfg::THREADS) {
            const double y = v2own[r] * inv_nu;
            if (r0 + r < p.m) p.Y[(r0 + r) + k * p.ldy] = y;
            float hi, lo;
            split_double(y, hi, lo);
            p.ysb[(b * 2 + 0) * p.d_max * RS + k * RS + r] = hi;
            p.ysb[(b * 2 + 1) * p.d_max * RS + k * RS + r] = lo;
        }
        fence_proxy_async_global();  // this block of Y is streamed by bulk copies in later steps
        if (warp == NW) {
            // producer: pivot-vector tiles of the prefetched units, then the remaining units
            if (lane == 0 && ok) {
                int64_t g = L0 / NT, t = L0 - (L0 / NT) * NT;
                int sp = pf_s0;  // stage of the first prefetched unit
                for (int64_t i = 0; i < npref; ++i) {
                    const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                    const uint32_t xi_bytes = 2u * rows * 4u;
                    mbar_arrive_expect_tx(&full[sp], WT ? 2u * xi_bytes : xi_bytes);
                    bulk_g2s(stages + (size_t)sp * STAGE, p.v2s + t * 2 * MT, xi_bytes, &full[sp], pol_xi);
                    if constexpr (WT)
                        bulk_g2s(stages + (size_t)sp * STAGE + 2 * MT, p.zs + t * 2 * MT, xi_bytes, &full[sp], pol_xi);
                    if (++sp == S) sp = 0;
                    if (++t == NT) {
                        t = 0;
                        ++g;
                    }
                }
                for (int64_t i = npref; i < nunits; ++i) {
                    if (preuse && !mbar_wait(&empty[ps], pph ^ 1u, p.wait_ns)) {
                        loop_abort(ctl, p.bar, ST_ETIMEOUT);
                        ok = false;
                        break;
                    }
                    const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                    const uint32_t xi_bytes = 2u * rows * 4u;
                    const uint32_t x_bytes = (uint32_t)(C * UB) * rows;
                    float* st = stages + (size_t)ps * STAGE;
                    mbar_arrive_expect_tx(&full[ps], x_bytes);
                    bulk_g2s(st + XI, planes + (g * p.group_stride + t * p.tile_stride) * Cfg::ESIZE, x_bytes, &full[ps],
                             pol_x);
                    mbar_arrive_expect_tx(&full[ps], WT ? 2u * xi_bytes : xi_bytes);
                    bulk_g2s(st, p.v2s + t * 2 * MT, xi_bytes, &full[ps], pol_xi);
                    if constexpr (WT) bulk_g2s(st + 2 * MT, p.zs + t * 2 * MT, xi_bytes, &full[ps], pol_xi);
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
                npref = 0;
            }
        } else {
            // consumers
            float acc_s[CPW][4], acc_c[CPW][4];
            float acc2_s[WT ? CPW : 1][4], acc2_c[WT ? CPW : 1][4];  // A-norm form: dots with z
#pragma unroll
            for (int qq = 0; qq < CPW; ++qq)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc_s[qq][e] = acc_c[qq][e] = 0.f;
#pragma unroll
            for (int qq = 0; qq < (WT ? CPW : 1); ++qq)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc2_s[qq][e] = acc2_c[qq][e] = 0.f;
            double best_e = -1.0;
            int64_t best_j = INT64_MAX;
            double e_old[CPW];
#pragma unroll
            for (int qq = 0; qq < CPW; ++qq) e_old[qq] = 0.0;
            int gbuf = 0;
            FlushCtx fc;
            fc.T = p.T;
            fc.ldt = p.ldt;
            fc.e = p.e;
            fc.n = p.n;
            fc.k = k;
            fc.piv = piv;
            fc.inv_nu = inv_nu;
            fc.q = qa;
            fc.gcnt = p.gcnt;
            fc.gslot = p.gslot;
            fc.gslot2 = p.gslot2;
            fc.gsum = p.gsum;
            fc.KMAX = p.KMAX;
            fc.W = W;
            fc.NT = NT;
            fc.G = G;
            fc.b = b;
            fc.L0 = L0;
            fc.L1 = L1;
            fc.grp_e = grp_e;
            fc.flag = &sflags[2];
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
                const int64_t c0 = g * C;
                const int ncols = (int)min((int64_t)C, p.n - c0);
                if (lane == 0 && (t == 0 || u == L0)) {
#pragma unroll
                    for (int qq = 0; qq < CPW; ++qq) {
                        const int cw = warp * CPW + qq;
                        if (cw < ncols) e_old[qq] = __ldcg(&p.e[c0 + cw]);
                    }
                }
                if (ok && !mbar_wait(&full[s], ph, p.wait_ns)) {
                    loop_abort(ctl, p.bar, ST_ETIMEOUT);
                    ok = false;
                }
                const int rows = (int)min((int64_t)MT, p.ldp - t * MT);
                if (ok) {
                    const float* st = stages + (size_t)s * STAGE;
                    if constexpr (WT) {
                        if constexpr (XT == 2) {
                            if (rows == MT)
                                consume_tile_bf16_w<CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c, acc2_s, acc2_c);
                            else
                                consume_tile_bf16_w<CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c, acc2_s,
                                                                    acc2_c);
                        } else {
                            if (rows == MT)
                                consume_tile_w<Cfg::PL, CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c, acc2_s,
                                                                       acc2_c);
                            else
                                consume_tile_w<Cfg::PL, CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c, acc2_s,
                                                                        acc2_c);
                        }
                    } else if constexpr (XT == 2) {
                        if (rows == MT)
                            consume_tile_bf16<CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c);
                        else
                            consume_tile_bf16<CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c);
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
                if constexpr (WT)
                    flush_group_t<CPW, C, NCONS, true>(fc, g, warp, lane, tid, acc_s, acc_c, acc2_s, acc2_c, e_old,
                                                       best_e, best_j, gbuf);
                else
                    flush_group<CPW, C, NCONS>(fc, g, warp, lane, tid, acc_s, acc_c, e_old, best_e, best_j, gbuf);
            }
            if (lane == 0) {
                red_e[warp] = best_e;
                red_j[warp] = best_j;
            }
            named_bar(1, NCONS);
            if (tid == 0) {
                double be = -1.0;
                int64_t bj = INT64_MAX;
                for (int w = 0; w < NW; ++w)
                    if (better(red_e[w], red_j[w], be, bj)) {
                        be = red_e[w];
                        bj = red_j[w];
                    }
                p.pbest_e[b] = be;
                p.pbest_j[b] = bj;
            }
        }
        if (!grid_sync(p.bar, (uint32_t)G, gen, &sflags[0], ctl, p.wait_ns)) ok = false;  // barrier 4
        if (!ok) break;

        // ---------------- A: argmax over CTAs, Frobenius residual ----------------
        if (warp == 0) {
            // every candidate load in flight before the comparisons
            constexpr int SL = kLoopMaxCtas / 32;
            double cev[SL];
            int64_t cjv[SL];
#pragma unroll
            for (int i = 0; i < SL; ++i) {
                const int64_t cb = lane + 32 * i;
                cev[i] = (cb < G) ? __ldcg(&p.pbest_e[cb]) : -1.0;
                cjv[i] = (cb < G) ? __ldcg(reinterpret_cast<const long long*>(&p.pbest_j[cb])) : INT64_MAX;
            }
            double be = -1.0;
            int64_t bj = INT64_MAX;
#pragma unroll
            for (int i = 0; i < SL; ++i)
                if (better(cev[i], cjv[i], be, bj)) {
                    be = cev[i];
                    bj = cjv[i];
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double oe = __shfl_down_sync(0xffffffffu, be, o);
                const int64_t oj = __shfl_down_sync(0xffffffffu, bj, o);
                if (better(oe, oj, be, bj)) {
                    be = oe;
                    bj = oj;
                }
            }
            if (lane == 0) red_j[0] = (bj >= 0 && bj < p.n) ? bj : piv;
        }
        __syncthreads();
        piv = red_j[0];
        if (b == 0 && tid == 0) {
            ctl->d = k + 1;
            ctl->pivot = piv;
        }
        __syncthreads();
    }

    // ---------------- leave: drain prefetched tiles, publish the final state ----------------
    // No bulk copy may still be writing this CTA's shared memory when it exits, whether the loop
    // ended normally or a wait gave up (RBD_ETIMEOUT): these waits keep the default bound.
    if (warp == NW && lane == 0) {
        // X tiles prefetched for a pass that did not run: their phases' second arrival (no
        // pivot-vector part), then every stage whose last issue may still be in flight
        for (int64_t i = 0; i < npref; ++i) mbar_arrive(&full[(int)((pf_s0 + i) % S)]);
        for (int s = 0; s < S; ++s)
            if (((iss_mask >> s) & 1u) && !mbar_wait(&full[s], (iss_par >> s) & 1u)) {
                raise_status(ctl, ST_ETIMEOUT);
                break;
            }
    }
    if (warp < NW && tid == 0) {
        // Y chunks issued but never waited for (a wait gave up part-way through a stream)
        for (uint32_t gc = ys.nwaited; gc < ys.nissued; ++gc)
            if (!mbar_wait(&ybar[gc % (uint32_t)ys.NB], (gc / (uint32_t)ys.NB) & 1u)) {
                raise_status(ctl, ST_ETIMEOUT);
                break;
            }
    }
    if (b == 0 && tid == 0) {
        if (stop != STOP_NONE) {
            ctl->stop = stop;
            ctl->d = k;
            ctl->pivot = piv;
        }
    }
}

int loop_chunk_cols_for(int xt, int wt, int R) {
    if (xt == 0) return wt ? loop_chunk_cols<LoopCfg<0, true>>(R) : loop_chunk_cols<LoopCfg<0, false>>(R);
    if (xt == 1) return wt ? loop_chunk_cols<LoopCfg<1, true>>(R) : loop_chunk_cols<LoopCfg<1, false>>(R);
    if (xt == 2) return wt ? loop_chunk_cols<LoopCfg<2, true>>(R) : loop_chunk_cols<LoopCfg<2, false>>(R);
    return 0;
}

size_t loop_smem_bytes(int xt, int wt, int R, int LC) {
    if (xt == 0) return wt ? loop_smem_layout<LoopCfg<0, true>>(R, LC).total : loop_smem_layout<LoopCfg<0, false>>(R, LC).total;
    if (xt == 1) return wt ? loop_smem_layout<LoopCfg<1, true>>(R, LC).total : loop_smem_layout<LoopCfg<1, false>>(R, LC).total;
    if (xt == 2) return wt ? loop_smem_layout<LoopCfg<2, true>>(R, LC).total : loop_smem_layout<LoopCfg<2, false>>(R, LC).total;
    return 0;
}

static const void* loop_fn(int xt, int wt) {
    if (wt) return (xt == 0) ? (const void*)loop_kernel<0, true> : (xt == 1) ? (const void*)loop_kernel<1, true>
                                                                              : (const void*)loop_kernel<2, true>;
    return (xt == 0) ? (const void*)loop_kernel<0, false> : (xt == 1) ? (const void*)loop_kernel<1, false>
                                                                      : (const void*)loop_kernel<2, false>;
}

cudaError_t loop_kernel_setup(int max_smem) {
    cudaError_t e = cudaSuccess;
    for (int wt = 0; wt < 2 && e == cudaSuccess; ++wt)
        for (int xt = 0; xt < 3 && e == cudaSuccess; ++xt)
            e = cudaFuncSetAttribute(loop_fn(xt, wt), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    return e;
}

cudaError_t launch_loop(const Work& w, const void* X, double* Y, int64_t ldy, double* T, int64_t ldt,
                        int64_t* pivots, double* err, double* nu_out, int64_t k0, cudaStream_t st) {
    LoopParams p;
    p.k0 = k0;
    p.m = w.m;
    p.n = w.n;
    p.ldp = w.ldp;
    p.ldx = w.ldx;
    p.ldt = ldt;
    p.ldy = ldy;
    p.d_max = w.d_max;
    p.xt = w.xt;
    p.planes = static_cast<const unsigned char*>(w.planes);
    p.group_stride = w.group_stride;
    p.tile_stride = w.tile_stride;
    p.NT = w.NT;
    p.ngroups = w.ngroups;
    p.W = w.W;
    p.KMAX = w.KMAX;
    p.evict_first = w.evict_first;
    p.wait_ns = wait_limit_ns(kWaitLimitNs);
    p.X = X;
    p.Y = Y;
    p.T = T;
    p.pivots = pivots;
    p.err = err;
    p.nu_out = nu_out;
    p.wts = w.wts;
    p.ctl = w.ctl;
    p.bar = w.ctl->bar;
    p.e = w.e;
    p.xn2 = w.xn2;
    p.ysb = w.ysb;
    p.v2s = w.v2s;
    p.zs = w.zs;
    p.hpart = w.hpart;
    p.h = w.h;
    p.nu2part = w.nu2part;
    p.pbest_e = w.pbest_e;
    p.pbest_j = w.pbest_j;
    p.gcnt = w.gcnt;
    p.gslot = w.gslot;
    p.gslot2 = w.gslot + (size_t)w.ngroups * (size_t)w.KMAX * (size_t)w.C;
    p.gsum = w.gsum;
    p.R = w.R;
    p.RS = w.RS;
    p.LC = w.LC;
    void* args[] = {&p};
    if (w.wt && !w.wts) return cudaErrorInvalidValue;
    const void* fn = loop_fn(w.xt, w.wt);
    const int threads = (w.xt == 0) ? TileCfg<0>::THREADS : (w.xt == 1) ? TileCfg<1>::THREADS : TileCfg<2>::THREADS;
    return cudaLaunchCooperativeKernel(fn, dim3((unsigned)w.G_loop), dim3((unsigned)threads), args, w.loop_smem, st);
}

}  // namespace rbd
