// rbd_work.h -- workspace layout and kernel launchers of one rbd_compress call.
//
// HBM layout (all regions 256-byte aligned, carved from one workspace allocation):
//   ctl      control block (Ctl)
//   planes   X re-laid out once by the initial pass, TILE-MAJOR, so that one bulk copy moves
//            one whole work tile of the fused pass.  FP64 input -> two FP32 planes (hi, lo)
//            with hi + lo = x to 2^-48 relative; FP32 input -> one FP32 plane; BF16 input ->
//            one BF16 plane.  Columns are grouped by C and rows padded to ldp = round_up(m, 128)
//            (padding rows and the padding columns of the last group are zero).  Row tiles
//            have MT rows except the last one (rows_t = ldp - t * MT, a multiple of 128).
//            Element (row R, column J, plane p), g = J / C, c = J % C, t = R / MT, r = R % MT:
//                g * C * P * ldp  +  t * C * P * MT  +  (c * P + p) * rows_t  +  r
//   yh, yl   split FP32 copy of Y (ldp x d_max each), read by the orthogonalisation GEMVs
//   ysb      loop path: split FP32 copy of Y by row block, [G][2][d_max][RS] (RS >= R rows; the
//            stride keeps the column-parallel dot products free of shared-memory bank conflicts)
//   v1, v2   FP64 work vectors of the current step (ldp) and split copies:
//            v1h/v1l plain (ldp each); v2s tile-interleaved for the pass: tile t holds
//            [hi(rows_t) | lo(rows_t)] at offset t * 2 * MT.
//   e, xn2   running squared residuals e_j and the initial squared norms ||x_j||^2 (n each)
//   vpart    partial sums of the row-parallel GEMVs (LC_MAX x ldp)
//   hpart, h partial and final re-orthogonalisation coefficients (RC_MAX x d_max, d_max)
//   nu2part  per-row-block partial squared norms (RB; 2 G on the loop path: Euclidean, A-norm)
//   zs       loop path, A-norm form: z = (I - Y Y') (w o v2) split like v2s (the second pivot vector)
//   rb_cnt, lb_cnt, gcnt   last-arriver counters (zero at rest)
//   gslot    per-column-group partial dot products (2 x ngroups x KMAX x C: xi, then z)
//   gsum     per-column-group sums of e_j (ngroups; two copies by parity of the basis on the
//            two-barrier loop path, whose service warps read one while the pass writes the other)
//   tf       two-barrier loop path: T in FP32, group-blocked [ngroups][d_max][C], streamed per group
//            for the correction of the pass's dot products
//   pbest_e/j  per-CTA argmax candidates of the fused pass (G)
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

#include "rbd.h"

// Fused-pass tile shape (compile-time; the defaults are the tuned GB300 values).
#ifndef RBD_PASS_NW
#define RBD_PASS_NW 8      // consumer warps per CTA
#endif
#ifndef RBD_PASS_CPW
#define RBD_PASS_CPW 2     // columns per consumer warp
#endif
#ifndef RBD_PASS_MT
#define RBD_PASS_MT 256    // rows per tile (a multiple of 128)
#endif
#ifndef RBD_PASS_S2
#define RBD_PASS_S2 5      // pipeline stages, FP64 input (two planes)
#endif
#ifndef RBD_PASS_S1
#define RBD_PASS_S1 8      // pipeline stages, FP32 input (one plane)
#endif
#ifndef RBD_PASS_MINB
#define RBD_PASS_MINB 1    // resident CTAs per SM the pass kernel is compiled for
#endif

namespace rbd {

struct Ctl;

// Fused-pass configuration per number of FP32 planes (2 = FP64 input, 1 = FP32 input).
template <int P>
struct PassCfg {
    static constexpr int NW = RBD_PASS_NW;
    static constexpr int CPW = RBD_PASS_CPW;
    static constexpr int C = NW * CPW;           // columns per group
    static constexpr int MT = RBD_PASS_MT;
    static constexpr int NSLAB = MT / 128;
    static constexpr int S = (P == 2) ? RBD_PASS_S2 : RBD_PASS_S1;
    static constexpr int XI_FLOATS = 2 * MT;     // split pivot-vector tile (hi, lo)
    static constexpr int STAGE_FLOATS = XI_FLOATS + C * P * MT;
    static constexpr int THREADS = (NW + 1) * 32;
    static constexpr size_t SCRATCH = 1024;
    static constexpr size_t SMEM = (size_t)S * STAGE_FLOATS * 4 + 2 * S * 8 + SCRATCH;
    static_assert(MT % 128 == 0, "tile rows must be a multiple of 128");
};

// bf16 storage: one plane of 2-byte elements, plain FP32 accumulation.
struct PassCfgBf16 {
    static constexpr int NW = 8;
    static constexpr int CPW = 2;
    static constexpr int C = NW * CPW;
    static constexpr int MT = 512;               // rows per tile (two 256-row slabs)
    static constexpr int S = 8;
    static constexpr int XI_FLOATS = 2 * MT;
    static constexpr int STAGE_BYTES = XI_FLOATS * 4 + C * MT * 2;
    static constexpr int THREADS = (NW + 1) * 32;
    static constexpr size_t SCRATCH = 1024;
    static constexpr size_t SMEM = (size_t)S * STAGE_BYTES + 2 * S * 8 + SCRATCH;
};

// Tile configuration of the persistent loop kernel's fused pass per storage type of X
// (0: FP64 as two FP32 planes, 1: FP32, 2: BF16).  PL = planes, ESIZE = bytes per plane element.
template <int XT>
struct TileCfg;
template <>
struct TileCfg<0> : PassCfg<2> {
    static constexpr int PL = 2, ESIZE = 4;
};
template <>
struct TileCfg<1> : PassCfg<1> {
    static constexpr int PL = 1, ESIZE = 4;
};
template <>
struct TileCfg<2> {
    static constexpr int NW = PassCfgBf16::NW;
    static constexpr int CPW = PassCfgBf16::CPW;
    static constexpr int C = PassCfgBf16::C;
    static constexpr int MT = PassCfgBf16::MT;
    static constexpr int S = PassCfgBf16::S;
    static constexpr int XI_FLOATS = PassCfgBf16::XI_FLOATS;
    static constexpr int STAGE_FLOATS = PassCfgBf16::STAGE_BYTES / 4;
    static constexpr int THREADS = PassCfgBf16::THREADS;
    static constexpr int PL = 1, ESIZE = 2;
};

// The diagonal A-norm form (Section 3.2) streams a second pivot-vector tile per unit: the stage
// holds [xi hi | xi lo | z hi | z lo] (2 * MT floats each pair) ahead of the X tile.
// RBD_F32_ACC32: FP32 storage (the planes and tiles of TileCfg<1>), FP32 accumulation per tile.
template <>
struct TileCfg<3> : TileCfg<1> {};

template <int XT>
struct TileCfgW : TileCfg<XT> {
    static constexpr int XI_FLOATS = 4 * TileCfg<XT>::MT;
    static constexpr int STAGE_FLOATS = TileCfg<XT>::STAGE_FLOATS + 2 * TileCfg<XT>::MT;
};

constexpr int kGemvRows = 128;     // rows per CTA of the row-parallel GEMVs
constexpr int kGemvTargetCtas = 304;
constexpr int kLoopMaxRows = 512;  // largest row block per CTA of the persistent loop kernel
constexpr int kLoopMaxCtas = 256;  // most CTAs of a persistent loop kernel (8 per lane of a warp)

struct Work {
    // sizes
    int64_t m, n, ldx, ldp, d_max;
    int xt;                 // rbd_dtype
    int wt;                 // 1: diagonal A-norm form (weights wts, loop kernel only)
    const double* wts;      // m weights of A = diag(wts), device (caller-owned), or nullptr
    int planes_n;           // number of planes P
    int esize;              // bytes per plane element
    // pass geometry
    int C, MT;
    int64_t NT, ngroups, W;
    int64_t group_stride;   // elements per column group (C * P * ldp)
    int64_t tile_stride;    // elements per full row tile of a group (C * P * MT)
    int G;                  // pass CTAs
    int KMAX;
    int64_t RB;             // row blocks of the GEMVs (ldp / 128)
    int64_t LC_MAX, RC_MAX;
    int num_sms;
    int evict_first;
    // persistent loop kernel (use_loop = 1): its grid, row blocks and shared memory
    int use_loop;
    int G_loop;             // CTAs (one per SM at most)
    int R;                  // rows per CTA block (multiple of 4)
    int RS;                 // column stride of a CTA's Y slice: R, or R + 4, so that RS = 4 mod 8
    int LC;                 // Y columns per streamed chunk
    size_t loop_smem;       // dynamic shared memory bytes
    int use_defer;          // A = I: the two-barrier loop kernel (rbd_defer.cu) instead of rbd_loop.cu's
    int acc32;              // RBD_F32_ACC32 (xt is then RBD_F32): FP32 accumulation in the pass
    int KC;                 // d_max rounded up to 4 (coefficient and T-block rows in shared memory)
    // regions
    Ctl* ctl;
    void* planes;
    float *yh, *yl;         // stepwise path: split Y, column-major (ldp x d_max)
    float* ysb;             // loop path: split Y, row-block-major [G_loop][2][d_max][R]
    double *v1, *v2;
    float *v1h, *v1l, *v2s;
    float* zs;              // loop path: tile-interleaved split z of the A-norm form (as v2s)
    double *e, *xn2;
    double* vpart;
    double *hpart, *h;
    double* nu2part;
    uint32_t *rb_cnt, *lb_cnt, *gcnt;
    double *gslot, *gsum;   // gsum: 2 x ngroups (by parity of the basis) on the two-barrier path
    float* tf;              // two-barrier path: T in FP32, [ngroups][d_max][C]
    double* pbest_e;
    int64_t* pbest_j;
    // bytes of the zero-at-rest prefix (ctl + counters) to clear at call start
    size_t zero_bytes;
    size_t total_bytes;
    unsigned char* base;
};

// Fill sizes/geometry of `w` (region offsets in the pointer fields); false on unsupported sizes.
// loop_max_smem > 0 allows the persistent loop kernel with at most that much shared memory.
// wt = 1 plans the loop kernel of the A-norm form (larger pass stages); the workspace layout
// does not depend on wt.
// allow_defer = false keeps the four-barrier loop kernel for A = I (the no-tolerance mode, whose
// bases past the numerical rank need nu from v2 itself).
bool plan_work(Work& w, int64_t m, int64_t n, int64_t ldx, int64_t d_max, int xt, int num_sms,
               int pass_ctas_per_sm, int loop_max_smem, int wt = 0, bool allow_defer = true);
// Carve the regions of `w` out of `base` (at least w.total_bytes, 256-byte aligned).
void carve_work(Work& w, void* base);

// Per-device state: SM count and the one-time kernel attribute setup (cached per device; the
// first call on a device, with that device current, does the setup).  RBD_STEPWISE=1 reports no
// loop-kernel shared memory, which selects the stepwise path.
struct DeviceState {
    int num_sms = 0;
    int pass_ctas_per_sm[3] = {1, 1, 1};
    int loop_max_smem = 0;  // 0: the persistent loop kernels are not used on this device
    bool ready = false;
};
cudaError_t device_state(DeviceState& out);

// Stream-ordered scratch for the calls that allocate: from a memory pool the library creates per
// device, which keeps up to kPoolKeepBytes of freed memory reserved for the next call (the
// default pool returns freed memory to the system at every synchronisation, and mapping it again
// costs ~1 ms per GB).  Freed with cudaFreeAsync.
constexpr uint64_t kPoolKeepBytes = 4ull << 30;
cudaError_t lib_malloc_async(void** p, size_t bytes, cudaStream_t st);
// The storage type of X (RBD_F32_ACC32 stores FP32) and its element size.
inline int storage_of(int t) { return (t == RBD_F32_ACC32) ? (int)RBD_F32 : t; }
inline int elem_bytes(int t) { return (t == RBD_F64) ? 8 : (t == RBD_BF16) ? 2 : 4; }

// The bound on device-side waits the next launches take: the caller's (rbd_set_wait_limit), or
// dflt when none is set.
uint64_t wait_limit_ns(uint64_t dflt);
// cudaError_t -> rbd_status (allocation failures are RBD_ENOMEM, every other error RBD_ECUDA).
rbd_status map_cuda(cudaError_t e);
// The argument rules of rbd_compress (and of every entry point that takes its arguments).
rbd_status validate(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx, double tol, rbd_tol_mode mode,
                    int64_t d_max, int64_t start, const double* Y, int64_t ldy, const double* T, int64_t ldt,
                    const int64_t* pivots, const double* err);

// ---- launchers (each returns the cudaError_t of its launch) ----
// With w.wts set: e_j = ||x_j||_A^2 (xn2 stays Euclidean) and the tolerance scales in A-norms.
cudaError_t launch_init(const Work& w, const void* X, double tol, int mode, int64_t start,
                        cudaStream_t st);
cudaError_t launch_orth_a1(const Work& w, const void* X, const double* T, int64_t ldt, int64_t k,
                           cudaStream_t st);
cudaError_t launch_orth_a2(const Work& w, int64_t k, cudaStream_t st);
cudaError_t launch_orth_c(const Work& w, int64_t k, int64_t* pivots, double* nu_out, double* err,
                          uint32_t* progress, cudaStream_t st);
cudaError_t launch_pass(const Work& w, double* Y, int64_t ldy, double* T, int64_t ldt, int64_t k,
                        uint32_t* progress, cudaStream_t st);
cudaError_t launch_project(const double* Y, int64_t m, int64_t d, int64_t ldy, const void* V, int vt,
                           int64_t k, int64_t ldv, double* C, int64_t ldc, cudaStream_t st);
// Restore the loop state after k0 bases (rbd_compress_resume): e_j, the group sums, the split
// copy of Y for the path in use, and fro_last / pivot / d in the control block.
cudaError_t launch_resume(const Work& w, const double* Y, int64_t ldy, const double* T, int64_t ldt,
                          const int64_t* pivots, int64_t k0, int64_t next_pivot, cudaStream_t st);
// Xt(j, i) = X(i, j) for an m x n column-major X (ldx) and the n x m column-major Xt (ld = n); esize
// is the element size in bytes (8, 4 or 2).
cudaError_t launch_transpose(const void* X, int esize, int64_t m, int64_t n, int64_t ldx, void* Xt, int num_sms,
                             cudaStream_t st);
cudaError_t launch_reconstruct(const double* Y, int64_t m, int64_t d, int64_t ldy, const double* T, int64_t n,
                               int64_t ldt, double* Xr, int64_t ldxr, cudaStream_t st);
// Dynamic shared-memory opt-in for the pass kernels and their resident CTAs per SM, indexed by
// storage type (once per device).
cudaError_t pass_kernel_setup(int ctas_per_sm[3]);

// Persistent loop kernel: shared-memory bytes for a plan (0 if the storage type has no loop
// kernel), one-time attribute setup, and the cooperative launch of the whole greedy loop.
size_t loop_smem_bytes(int xt, int wt, int R, int LC);
int loop_chunk_cols_for(int xt, int wt, int R);
cudaError_t loop_kernel_setup(int max_smem);
cudaError_t launch_loop(const Work& w, const void* X, double* Y, int64_t ldy, double* T, int64_t ldt,
                        int64_t* pivots, double* err, double* nu_out, int64_t k0, cudaStream_t st);
// The two-barrier persistent loop kernel (A = I): shared-memory bytes, Y columns per streamed chunk,
// one-time attribute setup and the cooperative launch.
size_t defer_smem_bytes(int xt, int R, int KC);
int defer_chunk_cols(int xt, int RS);
cudaError_t defer_kernel_setup(int max_smem);
cudaError_t launch_defer(const Work& w, const void* X, double* Y, int64_t ldy, double* T, int64_t ldt,
                         int64_t* pivots, double* err, double* nu_out, int64_t k0, cudaStream_t st);

}  // namespace rbd
