// rbd_tile.cuh -- the fused pass's per-tile arithmetic and per-column-group finalisation,
// shared by the stepwise pass kernel (rbd_pass.cu) and the persistent loop kernel (rbd_loop.cu).
//
//   c_j = xi_k' X(:, j)   (step 2.2, T(k, j) = c_j)
//   e_j <- e_j - c_j^2    (Eq. (evalerr) with A = I and orthonormal Y: ||x||^2 - ||c||^2)
//   A = diag(w): e_j <- e_j - c_j (2 b_j - c_j xi_k' A xi_k), b_j = z' x_j, z = (I - Y Y')(w o xi_k)
//   argmax_j e_j          (step 2.3; lowest j on ties)
#pragma once

#include "rbd_device.cuh"

namespace rbd {

// CTA that processes unit u when W units are split into G contiguous ranges
// [floor(b W / G), floor((b + 1) W / G)).
__device__ __forceinline__ int64_t unit_owner(int64_t u, int64_t W, int64_t G) {
    return ((u + 1) * G + W - 1) / W - 1;
}

// Float-float dot-product contributions of one staged tile for this warp's CPW columns.
// Stage layout: [xi hi (rows) | xi lo (rows) | pad to 2*MT | column c plane p at (c*P + p)*rows].
// FULL tiles (rows == MT) compile to straight-line code; the ragged last row tile of a column
// group takes the generic path.
template <int P, int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile(const float* __restrict__ st, int rows, int warp, int lane,
                                             float (&acc_s)[CPW][4], float (&acc_c)[CPW][4]) {
    constexpr int XI = 2 * MT;
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(st + off);
        const float4 zl = *reinterpret_cast<const float4*>(st + R + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const float* col = st + XI + (warp * CPW + q) * P * R + off;
            const float4 a = *reinterpret_cast<const float4*>(col);
            if (P == 2) {
                const float4 al = *reinterpret_cast<const float4*>(col + R);
                ff_mac2(acc_s[q][0], acc_c[q][0], a.x, al.x, zh.x, zl.x);
                ff_mac2(acc_s[q][1], acc_c[q][1], a.y, al.y, zh.y, zl.y);
                ff_mac2(acc_s[q][2], acc_c[q][2], a.z, al.z, zh.z, zl.z);
                ff_mac2(acc_s[q][3], acc_c[q][3], a.w, al.w, zh.w, zl.w);
            } else {
                ff_mac1(acc_s[q][0], acc_c[q][0], a.x, zh.x, zl.x);
                ff_mac1(acc_s[q][1], acc_c[q][1], a.y, zh.y, zl.y);
                ff_mac1(acc_s[q][2], acc_c[q][2], a.z, zh.z, zl.z);
                ff_mac1(acc_s[q][3], acc_c[q][3], a.w, zh.w, zl.w);
            }
        }
    }
}

// The A-norm form (Section 3.2): two dot products per column and row, with xi (acc) and with
// z = (I - Y Y')(w o xi) (acc2).  Stage layout: [xi hi | xi lo | z hi (at 2 MT) | z lo | pad to
// 4*MT | column c plane p at (c*P + p)*rows].
template <int P, int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile_w(const float* __restrict__ st, int rows, int warp, int lane,
                                               float (&acc_s)[CPW][4], float (&acc_c)[CPW][4],
                                               float (&acc2_s)[CPW][4], float (&acc2_c)[CPW][4]) {
    constexpr int XI = 4 * MT;
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(st + off);
        const float4 zl = *reinterpret_cast<const float4*>(st + R + off);
        const float4 wh = *reinterpret_cast<const float4*>(st + 2 * MT + off);
        const float4 wl = *reinterpret_cast<const float4*>(st + 2 * MT + R + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const float* col = st + XI + (warp * CPW + q) * P * R + off;
            const float4 a = *reinterpret_cast<const float4*>(col);
            if (P == 2) {
                const float4 al = *reinterpret_cast<const float4*>(col + R);
                ff_mac2(acc_s[q][0], acc_c[q][0], a.x, al.x, zh.x, zl.x);
                ff_mac2(acc_s[q][1], acc_c[q][1], a.y, al.y, zh.y, zl.y);
                ff_mac2(acc_s[q][2], acc_c[q][2], a.z, al.z, zh.z, zl.z);
                ff_mac2(acc_s[q][3], acc_c[q][3], a.w, al.w, zh.w, zl.w);
                ff_mac2(acc2_s[q][0], acc2_c[q][0], a.x, al.x, wh.x, wl.x);
                ff_mac2(acc2_s[q][1], acc2_c[q][1], a.y, al.y, wh.y, wl.y);
                ff_mac2(acc2_s[q][2], acc2_c[q][2], a.z, al.z, wh.z, wl.z);
                ff_mac2(acc2_s[q][3], acc2_c[q][3], a.w, al.w, wh.w, wl.w);
            } else {
                ff_mac1(acc_s[q][0], acc_c[q][0], a.x, zh.x, zl.x);
                ff_mac1(acc_s[q][1], acc_c[q][1], a.y, zh.y, zl.y);
                ff_mac1(acc_s[q][2], acc_c[q][2], a.z, zh.z, zl.z);
                ff_mac1(acc_s[q][3], acc_c[q][3], a.w, zh.w, zl.w);
                ff_mac1(acc2_s[q][0], acc2_c[q][0], a.x, wh.x, wl.x);
                ff_mac1(acc2_s[q][1], acc2_c[q][1], a.y, wh.y, wl.y);
                ff_mac1(acc2_s[q][2], acc2_c[q][2], a.z, wh.z, wl.z);
                ff_mac1(acc2_s[q][3], acc2_c[q][3], a.w, wh.w, wl.w);
            }
        }
    }
}

// Same arithmetic as consume_tile, with the pivot vector's rows of this tile taken from separate
// (hi, lo) arrays (the batched kernel keeps the whole vector in shared memory) and the stage
// holding only the X tile: column c plane p at (c*P + p)*rows.
template <int P, int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile_xi(const float* __restrict__ st, const float* __restrict__ xh,
                                                const float* __restrict__ xl, int rows, int warp, int lane,
                                                float (&acc_s)[CPW][4], float (&acc_c)[CPW][4]) {
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(xh + off);
        const float4 zl = *reinterpret_cast<const float4*>(xl + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const float* col = st + (warp * CPW + q) * P * R + off;
            const float4 a = *reinterpret_cast<const float4*>(col);
            if (P == 2) {
                const float4 al = *reinterpret_cast<const float4*>(col + R);
                ff_mac2(acc_s[q][0], acc_c[q][0], a.x, al.x, zh.x, zl.x);
                ff_mac2(acc_s[q][1], acc_c[q][1], a.y, al.y, zh.y, zl.y);
                ff_mac2(acc_s[q][2], acc_c[q][2], a.z, al.z, zh.z, zl.z);
                ff_mac2(acc_s[q][3], acc_c[q][3], a.w, al.w, zh.w, zl.w);
            } else {
                ff_mac1(acc_s[q][0], acc_c[q][0], a.x, zh.x, zl.x);
                ff_mac1(acc_s[q][1], acc_c[q][1], a.y, zh.y, zl.y);
                ff_mac1(acc_s[q][2], acc_c[q][2], a.z, zh.z, zl.z);
                ff_mac1(acc_s[q][3], acc_c[q][3], a.w, zh.w, zl.w);
            }
        }
    }
}

// BF16 storage (the precision form): FP32 products of the exact BF16 values with the leading
// FP32 part of the pivot vector, summed in FP32 over the unit's rows (16 per lane) and folded into
// the float-float accumulator once per unit.  Stage layout as above with BF16 columns.
template <int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile_bf16(const float* __restrict__ st, int rows, int warp, int lane,
                                                  float (&acc_s)[CPW][4], float (&acc_c)[CPW][4]) {
    constexpr int XI = 2 * MT;
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
    const unsigned short* xb = reinterpret_cast<const unsigned short*>(st + XI);
    float part[CPW][4];
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[q][e] = 0.f;
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(st + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            // four consecutive BF16 values; a BF16 value is the upper half of its FP32 pattern
            const uint2 u = *reinterpret_cast<const uint2*>(xb + (warp * CPW + q) * R + off);
            part[q][0] = __fmaf_rn(__uint_as_float(u.x << 16), zh.x, part[q][0]);
            part[q][1] = __fmaf_rn(__uint_as_float(u.x & 0xffff0000u), zh.y, part[q][1]);
            part[q][2] = __fmaf_rn(__uint_as_float(u.y << 16), zh.z, part[q][2]);
            part[q][3] = __fmaf_rn(__uint_as_float(u.y & 0xffff0000u), zh.w, part[q][3]);
        }
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        const float sum = __fadd_rn(__fadd_rn(part[q][0], part[q][1]), __fadd_rn(part[q][2], part[q][3]));
        ff_add(acc_s[q][0], acc_c[q][0], sum, 0.f);
    }
}

// FP32 storage with FP32 accumulation (RBD_F32_ACC32, the precision form): FP32 products of the
// stored values with the leading FP32 part of the pivot vector, summed in FP32 over the unit's rows
// (8 per lane) and folded into the float-float accumulator once per unit.  Stage layout as for
// consume_tile with one plane.
template <int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile_f32acc(const float* __restrict__ st, int rows, int warp, int lane,
                                                    float (&acc_s)[CPW][4], float (&acc_c)[CPW][4]) {
    constexpr int XI = 2 * MT;
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
    float part[CPW][4];
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[q][e] = 0.f;
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(st + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const float4 a = *reinterpret_cast<const float4*>(st + XI + (warp * CPW + q) * R + off);
            part[q][0] = __fmaf_rn(a.x, zh.x, part[q][0]);
            part[q][1] = __fmaf_rn(a.y, zh.y, part[q][1]);
            part[q][2] = __fmaf_rn(a.z, zh.z, part[q][2]);
            part[q][3] = __fmaf_rn(a.w, zh.w, part[q][3]);
        }
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        const float sum = __fadd_rn(__fadd_rn(part[q][0], part[q][1]), __fadd_rn(part[q][2], part[q][3]));
        ff_add(acc_s[q][0], acc_c[q][0], sum, 0.f);
    }
}

// BF16 storage in the A-norm form: as consume_tile_bf16, a second FP32 sum with the leading part
// of z (stage layout of consume_tile_w).
template <int CPW, int MT, bool FULL>
__device__ __forceinline__ void consume_tile_bf16_w(const float* __restrict__ st, int rows, int warp, int lane,
                                                    float (&acc_s)[CPW][4], float (&acc_c)[CPW][4],
                                                    float (&acc2_s)[CPW][4], float (&acc2_c)[CPW][4]) {
    constexpr int XI = 4 * MT;
    const int R = FULL ? MT : rows;
    const int nsl = FULL ? MT / 128 : (rows >> 7);
    const unsigned short* xb = reinterpret_cast<const unsigned short*>(st + XI);
    float part[CPW][4], part2[CPW][4];
#pragma unroll
    for (int q = 0; q < CPW; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[q][e] = part2[q][e] = 0.f;
#pragma unroll
    for (int sl = 0; sl < MT / 128; ++sl) {
        if (!FULL && sl >= nsl) break;
        const int off = sl * 128 + lane * 4;
        const float4 zh = *reinterpret_cast<const float4*>(st + off);
        const float4 wh = *reinterpret_cast<const float4*>(st + 2 * MT + off);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const uint2 u = *reinterpret_cast<const uint2*>(xb + (warp * CPW + q) * R + off);
            const float a0 = __uint_as_float(u.x << 16), a1 = __uint_as_float(u.x & 0xffff0000u);
            const float a2 = __uint_as_float(u.y << 16), a3 = __uint_as_float(u.y & 0xffff0000u);
            part[q][0] = __fmaf_rn(a0, zh.x, part[q][0]);
            part[q][1] = __fmaf_rn(a1, zh.y, part[q][1]);
            part[q][2] = __fmaf_rn(a2, zh.z, part[q][2]);
            part[q][3] = __fmaf_rn(a3, zh.w, part[q][3]);
            part2[q][0] = __fmaf_rn(a0, wh.x, part2[q][0]);
            part2[q][1] = __fmaf_rn(a1, wh.y, part2[q][1]);
            part2[q][2] = __fmaf_rn(a2, wh.z, part2[q][2]);
            part2[q][3] = __fmaf_rn(a3, wh.w, part2[q][3]);
        }
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        const float sum = __fadd_rn(__fadd_rn(part[q][0], part[q][1]), __fadd_rn(part[q][2], part[q][3]));
        ff_add(acc_s[q][0], acc_c[q][0], sum, 0.f);
        const float sum2 = __fadd_rn(__fadd_rn(part2[q][0], part2[q][1]), __fadd_rn(part2[q][2], part2[q][3]));
        ff_add(acc2_s[q][0], acc2_c[q][0], sum2, 0.f);
    }
}

// Everything the end-of-group finalisation needs.
struct FlushCtx {
    double* T;
    int64_t ldt;
    double* e;
    int64_t n;
    int64_t k;          // row of T being written (basis index)
    int64_t piv;        // column whose basis this is: its residual is set to 0
    double inv_nu;      // dot products were taken with v2; xi_k = v2 / nu
    double q;           // A-norm form: xi_k' A xi_k
    uint32_t* gcnt;     // per-group arrival counters (zero at rest)
    double* gslot;      // per-group partial sums (ngroups x KMAX x C)
    double* gslot2;     // A-norm form: the same for the dot products with z
    double* gsum;       // per-group sums of e_j
    int KMAX;
    int64_t W, NT, G, b, L0, L1;
    double* grp_e;      // shared: 2 x C (double buffer)
    int* flag;          // shared
};

// End of this CTA's share of column group g: combine the accumulators (float-float, fixed
// order), publish or combine partials of a group split between CTAs (the last CTA to arrive
// sums them in CTA order), and finalise the group's columns: T(k, j), e_j, the running argmax
// (best_e, best_j) and the group sum of e_j.  Called by all consumer threads (NCONS).
// WT (the A-norm form): the accumulators acc2 hold the dot products with z, b_j = z' x_j / nu,
// and the indicator update of Eq. (evalerr) becomes e_j <- e_j - c_j (2 b_j - c_j q).
template <int CPW, int C, int NCONS, bool WT>
__device__ __forceinline__ void flush_group_t(const FlushCtx& f, int64_t g, int warp, int lane, int tid,
                                              float (&acc_s)[CPW][4], float (&acc_c)[CPW][4],
                                              float (&acc2_s)[CPW][4], float (&acc2_c)[CPW][4],
                                              const double (&e_old)[CPW], double& best_e, int64_t& best_j,
                                              int& gbuf) {
    const int64_t c0 = g * C;
    const int ncols = (int)min((int64_t)C, f.n - c0);
    double tot[CPW], tot2[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        float sq = acc_s[q][0], cq = acc_c[q][0];
#pragma unroll
        for (int e = 1; e < 4; ++e) ff_add(sq, cq, acc_s[q][e], acc_c[q][e]);
        warp_sum_ff(sq, cq);
        tot[q] = ff_to_double(sq, cq);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc_s[q][e] = acc_c[q][e] = 0.f;
        tot2[q] = 0.0;
        if constexpr (WT) {
            float s2 = acc2_s[q][0], c2 = acc2_c[q][0];
#pragma unroll
            for (int e = 1; e < 4; ++e) ff_add(s2, c2, acc2_s[q][e], acc2_c[q][e]);
            warp_sum_ff(s2, c2);
            tot2[q] = ff_to_double(s2, c2);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc2_s[q][e] = acc2_c[q][e] = 0.f;
        }
    }
    const bool whole = (g * f.NT >= f.L0) && ((g + 1) * f.NT <= f.L1);
    if (!whole) {
        const int64_t bfirst = unit_owner(g * f.NT, f.W, f.G);
        const int64_t blast = unit_owner(g * f.NT + f.NT - 1, f.W, f.G);
        const uint32_t ncontrib = (uint32_t)(blast - bfirst + 1);
        const int64_t slot = f.b - bfirst;
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                const int cw = warp * CPW + q;
                if (cw < ncols) {
                    f.gslot[(g * f.KMAX + slot) * C + cw] = tot[q];
                    if constexpr (WT) f.gslot2[(g * f.KMAX + slot) * C + cw] = tot2[q];
                }
            }
            __threadfence();
        }
        named_bar(1, NCONS);
        if (tid == 0) *f.flag = (atomicAdd(&f.gcnt[g], 1u) == ncontrib - 1);
        named_bar(1, NCONS);
        if (!*f.flag) return;
        __threadfence();
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                const int cw = warp * CPW + q;
                if (cw < ncols) {
                    double acc = 0.0;
                    for (uint32_t sl = 0; sl < ncontrib; ++sl) acc += __ldcg(&f.gslot[(g * f.KMAX + sl) * C + cw]);
                    tot[q] = acc;
                    if constexpr (WT) {
                        double acc2 = 0.0;
                        for (uint32_t sl = 0; sl < ncontrib; ++sl)
                            acc2 += __ldcg(&f.gslot2[(g * f.KMAX + sl) * C + cw]);
                        tot2[q] = acc2;
                    }
                }
            }
        }
        if (tid == 0) f.gcnt[g] = 0;
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const int cw = warp * CPW + q;
            if (cw < ncols) {
                const int64_t j = c0 + cw;
                const double cj = tot[q] * f.inv_nu;
                f.T[j * f.ldt + f.k] = cj;
                double en;
                if constexpr (WT) {
                    const double bj = tot2[q] * f.inv_nu;
                    en = (j == f.piv) ? 0.0 : fmax(e_old[q] - cj * (2.0 * bj - cj * f.q), 0.0);
                } else {
                    en = (j == f.piv) ? 0.0 : fmax(e_old[q] - cj * cj, 0.0);
                }
                f.e[j] = en;
                f.grp_e[gbuf * C + cw] = en;
                if (better(en, j, best_e, best_j)) {
                    best_e = en;
                    best_j = j;
                }
            }
        }
    }
    // one barrier per group: thread 0 sums this buffer while the other warps move on; the
    // buffer is written again two groups later, after thread 0 has passed the next barrier
    named_bar(1, NCONS);
    if (tid == 0) {
        double sacc = 0.0;
        for (int cw = 0; cw < ncols; ++cw) sacc += f.grp_e[gbuf * C + cw];
        f.gsum[g] = sacc;
    }
    gbuf ^= 1;
}

template <int CPW, int C, int NCONS>
__device__ __forceinline__ void flush_group(const FlushCtx& f, int64_t g, int warp, int lane, int tid,
                                            float (&acc_s)[CPW][4], float (&acc_c)[CPW][4],
                                            const double (&e_old)[CPW], double& best_e, int64_t& best_j,
                                            int& gbuf) {
    flush_group_t<CPW, C, NCONS, false>(f, g, warp, lane, tid, acc_s, acc_c, acc_s, acc_c, e_old, best_e, best_j,
                                        gbuf);
}

}  // namespace rbd
