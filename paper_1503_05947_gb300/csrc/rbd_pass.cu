// rbd_pass.cu -- the fused pass of one greedy step (Algorithm 1, steps 2.2 and 2.3):
//
//   for every column j:  c_j = xi_k' X(:, j)                    T(k, j) = c_j   (step 2.2)
//                        e_j <- e_j - c_j^2                      (Eq. (evalerr), A = I)
//   i = argmax_j e_j (lowest j on ties)                                           (step 2.3)
//   (E_cur itself, and the stop test of step 2.4, are taken by the next orthogonalisation,
//    which recomputes the residual of column i in FP64; see rbd_orth.cu)
//
// With Y orthonormal, Eq. (evalerr) for A = I reduces to ||x_j||^2 - ||c||^2, so the squared
// residual of every column is maintained by subtracting the new coefficient's square: one
// streaming pass over X per step, no m-length work per column.
//
// Layout and work split (GB300, 152 SMs, one persistent CTA per SM):
//   * X lives in HBM as tile-major FP32 planes (rbd_work.h); a unit of work is one tile of
//     MT rows x C columns (both planes contiguous, 32 KB for FP64 input).  The
//     W = NT * ngroups units are enumerated column-group-major and split into G contiguous,
//     equal ranges (one per CTA), so every SM streams the same number of bytes.
//   * One producer thread moves each unit into a shared-memory ring with two bulk (TMA)
//     copies -- the whole X tile and the matching tile of the split pivot vector --
//     completing on an mbarrier; X is read with an L2 evict-first policy so the split copy of
//     Y stays cached for the orthogonalisation kernels.
//   * Eight consumer warps each own CPW columns of the tile; lane l multiplies rows 4l..4l+3
//     of every 128-row slab in float-float arithmetic (4 independent accumulators per column).
//   * A column group split between CTAs is combined by the last CTA to arrive at the group's
//     counter, summing the partial dot products in CTA order (deterministic, no waiting).
//   * The per-CTA argmax candidates are combined by the last CTA to finish, which names the
//     next pivot and publishes the step count to the host-mapped progress word.
#include "rbd_device.cuh"
#include "rbd_tile.cuh"
#include "rbd_work.h"

namespace rbd {

struct PassParams {
    const void* planes;
    int64_t group_stride;     // elements per column group of the tile-major planes
    int64_t tile_stride;      // elements per full row tile of a group
    const float* xis;         // split unnormalised pivot vector v2, tile-interleaved
    const double* v2;         // FP64 v2, for Y(:, k)
    double* Y;
    int64_t ldy;
    float* yh;
    float* yl;
    double* T;
    int64_t ldt;
    double* e;
    int64_t m, n, ldp;
    int64_t NT, ngroups, W;
    int KMAX;
    uint32_t* gcnt;
    double* gslot;
    double* gsum;
    double* pbest_e;
    int64_t* pbest_j;
    Ctl* ctl;
    int64_t k;
    int evict_first;
    uint32_t* progress;       // host-mapped {steps finished, stop} (may be null)
};

template <int P>
__global__ void __launch_bounds__(PassCfg<P>::THREADS, RBD_PASS_MINB) pass_kernel(PassParams p) {
    using Cfg = PassCfg<P>;
    constexpr int NW = Cfg::NW, CPW = Cfg::CPW, C = Cfg::C, MT = Cfg::MT, S = Cfg::S;
    constexpr int XI = Cfg::XI_FLOATS, STAGE = Cfg::STAGE_FLOATS;
    constexpr int NCONS = NW * 32;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stages = reinterpret_cast<float*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)S * STAGE * 4);
    uint64_t* empty = full + S;
    double* red_e = reinterpret_cast<double*>(empty + S);   // NW
    int64_t* red_j = reinterpret_cast<int64_t*>(red_e + NW); // NW
    double* grp_e = reinterpret_cast<double*>(red_j + NW);   // 2 x C (double buffer)
    int* flag = reinterpret_cast<int*>(grp_e + 2 * C);
    static_assert((2 * NW + 2 * C) * 8 + 16 <= (int)Cfg::SCRATCH, "scratch too small");

    Ctl* ctl = p.ctl;
    if (ctl->stop != 0 || ctl->status != 0) return;  // uniform: set before this launch
    if (ctl->d != p.k) {
        if (threadIdx.x == 0 && blockIdx.x == 0) raise_status(ctl, ST_EINVAL);
        return;
    }
    const int64_t k = p.k;
    const int64_t piv = ctl->pivot;
    const double inv_nu = ctl->inv_nu;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t L0 = (p.W * b) / G, L1 = (p.W * (b + 1)) / G;
    const int64_t NT = p.NT;

    // Y(:, k) = v2 / nu and its split copy, for this CTA's share of the rows.
    {
        const int64_t per = round_up(ceil_div(p.ldp, G), 4);
        const int64_t r0 = b * per, r1 = min(p.ldp, r0 + per);
        for (int64_t r = r0 + tid; r < r1; r += blockDim.x) {
            const double y = (r < p.m) ? p.v2[r] * inv_nu : 0.0;
            if (r < p.m) p.Y[r + k * p.ldy] = y;
            float hi, lo;
            split_double(y, hi, lo);
            p.yh[r + k * p.ldp] = hi;
            p.yl[r + k * p.ldp] = lo;
        }
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NW) {
        // ------------------------------ producer ------------------------------
        if (lane == 0) {
            const uint64_t pol_x = p.evict_first ? l2_policy_evict_first() : l2_policy_evict_normal();
            const uint64_t pol_xi = l2_policy_evict_normal();
            const float* planes = static_cast<const float*>(p.planes);
            // running (group, tile) and (stage, phase) counters: no divisions in the loop
            int64_t g = L0 / NT, t = L0 - (L0 / NT) * NT;
            int s = 0;
            uint32_t ph = 0;
            bool reuse = false;
            for (int64_t u = L0; u < L1; ++u) {
                if (reuse && !mbar_wait(&empty[s], ph ^ 1u)) {
                    raise_status(ctl, ST_ETIMEOUT);
                    break;
                }
                const uint32_t rows = (uint32_t)min((int64_t)MT, p.ldp - t * MT);
                const uint32_t xi_bytes = 2u * rows * 4u;
                const uint32_t x_bytes = (uint32_t)(C * P) * rows * 4u;
                float* st = stages + (size_t)s * STAGE;
                mbar_arrive_expect_tx(&full[s], xi_bytes + x_bytes);
                bulk_g2s(st, p.xis + t * 2 * MT, xi_bytes, &full[s], pol_xi);
                bulk_g2s(st + XI, planes + g * p.group_stride + t * p.tile_stride, x_bytes, &full[s], pol_x);
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                    reuse = true;
                }
                if (++t == NT) {
                    t = 0;
                    ++g;
                }
            }
        }
        return;
    }

    // ------------------------------ consumers ------------------------------
    float acc_s[CPW][4], acc_c[CPW][4];
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc_s[q][e] = acc_c[q][e] = 0.f;
    double best_e = -1.0;
    int64_t best_j = INT64_MAX;
    bool ok = true;
    FlushCtx fc;
    fc.T = p.T;
    fc.ldt = p.ldt;
    fc.e = p.e;
    fc.n = p.n;
    fc.k = k;
    fc.piv = piv;
    fc.inv_nu = inv_nu;
    fc.gcnt = p.gcnt;
    fc.gslot = p.gslot;
    fc.gsum = p.gsum;
    fc.KMAX = p.KMAX;
    fc.W = p.W;
    fc.NT = NT;
    fc.G = G;
    fc.b = b;
    fc.L0 = L0;
    fc.L1 = L1;
    fc.grp_e = grp_e;
    fc.flag = flag;
    double e_old[CPW];          // e_j of this warp's columns, prefetched when a group starts
#pragma unroll
    for (int q = 0; q < CPW; ++q) e_old[q] = 0.0;
    int gbuf = 0;               // double buffer of the per-group sums in shared memory

    int64_t g_next = L0 / NT, t_next = L0 - (L0 / NT) * NT;
    int s_next = 0;
    uint32_t ph_next = 0;
    for (int64_t u = L0; u < L1; ++u) {
        const int64_t g = g_next, t = t_next;
        const int s = s_next;
        const uint32_t ph = ph_next;
        if (++s_next == S) {
            s_next = 0;
            ph_next ^= 1u;
        }
        if (++t_next == NT) {
            t_next = 0;
            ++g_next;
        }
        const int64_t c0 = g * C;
        const int ncols = (int)min((int64_t)C, p.n - c0);
        if (lane == 0 && (t == 0 || u == L0)) {
            // the finalisation at the end of the group needs e_j: load it now, off the
            // critical path (only the finaliser of column j writes e_j, after this read)
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                const int cw = warp * CPW + q;
                if (cw < ncols) e_old[q] = p.e[c0 + cw];
            }
        }
        if (ok && !mbar_wait(&full[s], ph)) {
            raise_status(ctl, ST_ETIMEOUT);
            ok = false;
        }
        const int rows = (int)min((int64_t)MT, p.ldp - t * MT);
        if (ok) {
            const float* st = stages + (size_t)s * STAGE;
            if (rows == MT)
                consume_tile<P, CPW, MT, true>(st, MT, warp, lane, acc_s, acc_c);
            else
                consume_tile<P, CPW, MT, false>(st, rows, warp, lane, acc_s, acc_c);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);

        if (t != NT - 1 && u != L1 - 1) continue;

        flush_group<CPW, C, NCONS>(fc, g, warp, lane, tid, acc_s, acc_c, e_old, best_e, best_j, gbuf);
    }

    // ---- per-CTA argmax candidate, then the grid-level last arriver ----
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
        __threadfence();
        *flag = (atomicAdd(&ctl->pass_arrive, 1u) == (uint32_t)(G - 1));
    }
    named_bar(1, NCONS);
    if (!*flag || warp != 0) return;
    __threadfence();
    double be = -1.0;
    int64_t bj = INT64_MAX;
    for (int64_t cb = lane; cb < G; cb += 32) {
        const double ce = __ldcg(&p.pbest_e[cb]);
        const int64_t cj = __ldcg(reinterpret_cast<const long long*>(&p.pbest_j[cb]));
        if (better(ce, cj, be, bj)) {
            be = ce;
            bj = cj;
        }
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
    // Frobenius residual: group sums in a fixed order
    const int64_t g0 = (p.ngroups * lane) / 32, g1 = (p.ngroups * (lane + 1)) / 32;
    double fs = 0.0;
    for (int64_t g = g0; g < g1; ++g) fs += __ldcg(&p.gsum[g]);
    fs = warp_sum_double(fs);
    if (lane == 0) {
        // The argmax names the next pivot; its E_cur is certified (recomputed in FP64 from X)
        // by the next orthogonalisation, which also takes the stop decision of step 2.4.
        ctl->err_downdate = sqrt(fmax(be, 0.0));
        ctl->fro_last = sqrt(fmax(fs, 0.0));
        ctl->d = k + 1;
        if (bj >= 0 && bj < p.n) ctl->pivot = bj;
        ctl->pass_arrive = 0;
        if (p.progress) {
            volatile uint32_t* pr = p.progress;
            pr[0] = (uint32_t)(k + 1);
            __threadfence_system();
        }
    }
}

template <int P>
static cudaError_t launch_pass_p(const Work& w, PassParams& p, cudaStream_t st) {
    pass_kernel<P><<<w.G, PassCfg<P>::THREADS, PassCfg<P>::SMEM, st>>>(p);
    return cudaGetLastError();
}

cudaError_t pass_kernel_setup(int ctas_per_sm[3]) {
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PassCfg<2>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pass_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PassCfg<1>::SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm[0], pass_kernel<2>, PassCfg<2>::THREADS,
                                                          PassCfg<2>::SMEM);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm[1], pass_kernel<1>, PassCfg<1>::THREADS,
                                                          PassCfg<1>::SMEM);
    ctas_per_sm[2] = 1;
    for (int i = 0; i < 3; ++i)
        if (ctas_per_sm[i] < 1) ctas_per_sm[i] = 1;
    return e;
}

cudaError_t launch_pass(const Work& w, double* Y, int64_t ldy, double* T, int64_t ldt, int64_t k,
                        uint32_t* progress, cudaStream_t st) {
    PassParams p;
    p.planes = w.planes;
    p.group_stride = w.group_stride;
    p.tile_stride = w.tile_stride;
    p.xis = w.v2s;
    p.v2 = w.v2;
    p.Y = Y;
    p.ldy = ldy;
    p.yh = w.yh;
    p.yl = w.yl;
    p.T = T;
    p.ldt = ldt;
    p.e = w.e;
    p.m = w.m;
    p.n = w.n;
    p.ldp = w.ldp;
    p.NT = w.NT;
    p.ngroups = w.ngroups;
    p.W = w.W;
    p.KMAX = w.KMAX;
    p.gcnt = w.gcnt;
    p.gslot = w.gslot;
    p.gsum = w.gsum;
    p.pbest_e = w.pbest_e;
    p.pbest_j = w.pbest_j;
    p.ctl = w.ctl;
    p.k = k;
    p.evict_first = w.evict_first;
    p.progress = progress;
    if (w.planes_n == 2) return launch_pass_p<2>(w, p, st);
    if (w.planes_n == 1 && w.esize == 4) return launch_pass_p<1>(w, p, st);
    return cudaErrorNotSupported;
}

}  // namespace rbd
