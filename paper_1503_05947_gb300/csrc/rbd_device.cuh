// rbd_device.cuh -- device-side building blocks shared by the librbd kernels.
//
//  * float-float ("ff") arithmetic: an FP64-grade quantity carried as the unevaluated sum
//    hi + lo of two FP32 numbers.  GB300 executes FP64 FMAs at ~1/64 of the FP32 rate
//    (measured: 0.59 T DFMA/s against 34.9 T FFMA/s), too slow to keep up with HBM on the
//    passes over X, so those passes run on the FP32 pipes with error-free transformations:
//    TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the FMA-based exact product (the product a*b
//    and its rounding error fma(a, b, -a*b)).  Sums of float-float products have relative
//    error ~2^-47, far inside the 1e-10 parity budget; FP64 is used for the per-column and
//    per-step scalars (coefficients, squared residuals, norms).
//  * inline PTX for mbarriers and the Blackwell bulk-copy (TMA) engine, with every wait
//    bounded in time so that no kernel can spin forever.
//  * the control block shared by the kernels of one rbd_compress call.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rbd {

// --------------------------------------------------------------------------------------
// Status / stop codes (mirror include/rbd.h)
// --------------------------------------------------------------------------------------
enum : int32_t { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENONFINITE = 4,
                 ST_ETIMEOUT = 5, ST_EUNSUPPORTED = 6 };
enum : int32_t { STOP_NONE = 0, STOP_TOL = 1, STOP_BREAK = 2, STOP_DMAX = 3 };
enum : int32_t { MODE_MAXCOL_ABS = 0, MODE_MAXCOL_REL = 1, MODE_FRO_REL = 2, MODE_NONE = 3 };


// Step 2.2 treats a pivot whose orthogonalised norm is at most kRankFloor * ||X(:, i)|| as
// already in span(Y) (numerical-rank floor; matches RBD_RANK_FLOOR in rbd.h).
constexpr double kRankFloor = 1e-12;

// The numerical-rank floor of step 2.2's break test in a tolerance mode (none without a tolerance:
// the loop then runs to d_max, stopping only on an orthogonalised vector that is zero or not
// finite).
__host__ __device__ __forceinline__ double rank_floor_of(int32_t mode) { return (mode == MODE_NONE) ? 0.0 : kRankFloor; }

// Upper bound on any device-side wait (nanoseconds of %globaltimer).
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// --------------------------------------------------------------------------------------
// Control block: one per rbd_compress call, in device workspace.
// --------------------------------------------------------------------------------------
struct Ctl {
    int64_t d;            // bases accepted so far (the step being built has index d)
    int64_t pivot;        // column orthogonalised in the current step (step 2.1's i)
    int32_t stop;         // STOP_*; once non-zero every later kernel returns at entry
    int32_t status;       // ST_* raised on the device
    uint32_t pass_arrive; // last-arriver counters (reset to 0 by the last arriver)
    uint32_t c_arrive;
    uint32_t init_arrive;
    uint32_t pad0;
    double nu;            // ||v|| of step 2.2 for the current step
    double inv_nu;        // 1 / nu
    double eps_r;         // step 2.4 threshold on E_cur (MAXCOL modes)
    double eps_r22;       // step 2.2 threshold on ||v||
    double fro_tol;       // FRO mode: tol * ||X||_F, else -1
    double x_fro;         // ||X||_F
    double x_maxcol;      // max_j ||X(:, j)||
    double err_downdate;  // sqrt(max_j e_j) of the last pass (Eq. (evalerr) form, diagnostic)
    double err_last;      // certified E_cur after the last accepted basis
    double fro_last;      // ||X - Y T||_F after the last accepted basis
    double tol;           // the user's tol
    int32_t mode;         // MODE_*
    int32_t pad1;
    int64_t d_max;
    uint32_t bar[4];      // counters of the persistent loop kernels (monotonic within a launch):
                          // {grid-barrier arrivals, shares of h summed, partial dot products
                          // published, unused}
};

// Element idx of X stored as FP64 (xt 0), FP32 (1) or BF16 (2), widened exactly to FP64.
__device__ __forceinline__ double load_x_elem(const void* X, int xt, int64_t idx) {
    if (xt == 0) return ((const double*)X)[idx];
    if (xt == 1) return (double)((const float*)X)[idx];
    return (double)__bfloat162float(((const __nv_bfloat16*)X)[idx]);
}

// --------------------------------------------------------------------------------------
// float-float helpers
// --------------------------------------------------------------------------------------
// s + e == a + b exactly (TwoSum; no precondition on |a|, |b|).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, c) += (xh + xl) * (yh + yl), dropping xl * yl (relative size <= 2^-48).
// The leading product xh * yh is split exactly into p + pe; the cross terms are small and
// are accumulated with pe into the compensation c.
__device__ __forceinline__ void ff_mac2(float& s, float& c, float xh, float xl, float yh, float yl) {
    float p = __fmul_rn(xh, yh);
    float pe = __fmaf_rn(xh, yh, -p);
    pe = __fmaf_rn(xh, yl, pe);
    pe = __fmaf_rn(xl, yh, pe);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

// (s, c) += x * (yh + yl) for an exact FP32 x.
__device__ __forceinline__ void ff_mac1(float& s, float& c, float x, float yh, float yl) {
    float p = __fmul_rn(x, yh);
    float pe = __fmaf_rn(x, yh, -p);
    pe = __fmaf_rn(x, yl, pe);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

__device__ __forceinline__ double ff_to_double(float s, float c) {
    return (double)s + (double)c;
}

// (s, c) += (s2, c2): the leading parts are added exactly (TwoSum), the compensations in FP32.
__device__ __forceinline__ void ff_add(float& s, float& c, float s2, float c2) {
    float t, e;
    two_sum(s, s2, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, e));
}

// s + e == a + b exactly, for |a| >= |b| or a == 0 (Fast2Sum).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (s, c) += (s2, c2) with the error bounded relative to the SUM (the accurate double-word addition
// of Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 2017): both parts are added with TwoSum and the result is
// renormalised twice.  ff_add bounds its error by the larger operand instead, which is too coarse
// when partial sums cancel.
__device__ __forceinline__ void ff_add_acc(float& s, float& c, float s2, float c2) {
    float sh, sl, th, tl;
    two_sum(s, s2, sh, sl);
    two_sum(c, c2, th, tl);
    sl = __fadd_rn(sl, th);
    fast_two_sum(sh, sl, sh, sl);
    sl = __fadd_rn(sl, tl);
    fast_two_sum(sh, sl, s, c);
}

// Float-float sum over the 32 lanes of a warp (fixed tree); the result is valid in lane 0.
__device__ __forceinline__ void warp_sum_ff(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_down_sync(0xffffffffu, s, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        ff_add(s, c, s2, c2);
    }
}

// x ~= hi + lo with |x - hi - lo| <= 2^-48 |x| (for |x| in the FP32 normal range).
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// Split an FP64 value into FP32 hi + lo with integer operations only (no FP64 pipe): hi is x
// rounded to nearest at 24 significant bits (a carry out of the significand moves into the
// exponent), lo the signed remainder, an integer of at most 2^28 units of x's last place, rounded
// to 24 bits by the integer-to-float conversion.  |lo| <= 2^-24 |x| and |x - hi - lo| <= 2^-48 |x|,
// as for split_double; the small |lo| matters where float-float products drop lo * lo.  Values
// outside 2^-74 <= |x| < 2^127 take the FP64 conversion path.
__device__ __forceinline__ void split_f64_fast(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t bh = (uint32_t)(b >> 32);
    const int E = (int)((bh >> 20) & 0x7ffu);
    if (E >= 949 && E <= 1149) {
        const uint32_t r29 = (uint32_t)b & 0x1fffffffu;  // the significand's low 29 bits
        const bool up = r29 >= 0x10000000u;
        const unsigned long long hb = (b & ~0x1fffffffull) + (up ? 0x20000000ull : 0ull);
        const uint32_t hbh = (uint32_t)(hb >> 32), hbl = (uint32_t)hb;
        const int Eh = (int)((hbh >> 20) & 0x7ffu);
        const uint32_t sign = bh & 0x80000000u;
        hi = __uint_as_float(sign | ((uint32_t)(Eh - 896) << 23) | ((hbh & 0xfffffu) << 3) | (hbl >> 29));
        const int rem = (int)r29 - (up ? 0x20000000 : 0);                // x - hi in units of 2^(E-1075)
        const float scale = __uint_as_float((uint32_t)(E - 948) << 23);  // 2^(E-1075), exact
        const float lv = __fmul_rn(__int2float_rn(rem), scale);
        lo = sign ? -lv : lv;
    } else {
        split_double(x, hi, lo);
    }
}

// --------------------------------------------------------------------------------------
// warp reductions
// --------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_double(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// 1 / x for a positive FP64 x by Newton's iteration y <- y + y (1 - x y) from the FP32
// reciprocal (relative error 2^-23, squared by each step: two steps reach FP64 rounding, within
// about 1 ulp) -- four FP64 FMAs instead of a division, whose FP64 sequence is long on this part.
// Outside the FP32 range it divides.
__device__ __forceinline__ double recip_pos(double x) {
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
    double y = (double)__frcp_rn((float)x);
    y = fma(y, fma(-x, y, 1.0), y);
    y = fma(y, fma(-x, y, 1.0), y);
    return y;
}

// The same order on integer keys: the FP64 bit patterns of non-negative values (which order like
// the values), LLONG_MIN for no candidate; integer compares avoid the slow FP64 pipe.
__device__ __forceinline__ bool better_key(long long k1, int64_t j1, long long k0, int64_t j0) {
    return (k1 > k0) || (k1 == k0 && j1 < j0);
}

// (value, index) max with ties to the lowest index; invalid entries carry index INT64_MAX.
__device__ __forceinline__ bool better(double e1, int64_t j1, double e0, int64_t j0) {
    return (e1 > e0) || (e1 == e0 && j1 < j0);
}

// --------------------------------------------------------------------------------------
// PTX: shared-memory addresses, mbarriers, bulk copies, L2 policies, timers
// --------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Whether the phase with the given parity has completed, without waiting (try_wait may suspend
// the thread for a while before it answers no).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete; false if limit_ns elapsed (the persistent
// kernels pass the caller's limit, rbd_set_wait_limit; their exit drains keep the default).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Bulk (TMA) copy global -> shared, completing `bytes` transaction bytes on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2, untracked; src 16-byte aligned, bytes a multiple
// of 16, the range inside one allocation.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Orders this thread's generic-proxy global writes before later async-proxy (bulk copy) reads
// of the same data.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Named barrier over `nthreads` threads (a multiple of 32) with id `id` (1..15).
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Arrive at named barrier `id` without waiting (the waiting side calls named_bar).
__device__ __forceinline__ void named_bar_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void raise_status(Ctl* ctl, int32_t st) {
    atomicCAS(&ctl->status, 0, st);
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

}  // namespace rbd
