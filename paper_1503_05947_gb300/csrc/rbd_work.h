// rbd_work.h -- workspace layout and kernel launchers of one rbd_compress call.
//
// HBM layout (all regions 256-byte aligned, carved from one workspace allocation):
//   ctl      control block (Ctl)
//   planes   X re-laid out once, column-major with leading dimension ldp = round_up(m, 128),
//            rows m..ldp-1 zero:  FP64 input -> two FP32 planes (hi, lo) with
//            hi + lo = x to 2^-48 relative;  FP32 input -> one FP32 plane;  BF16 -> one BF16
//            plane.  Plane p of column j starts at planes + (p * n + j) * ldp elements.
//   yh, yl   split FP32 copy of Y (ldp x d_max each), read by the orthogonalisation GEMVs
//   v1,v2    FP64 work vectors of the current step (ldp) and their split copies
//   e, xn2   running squared residuals e_j and the initial squared norms ||x_j||^2 (n each)
//   vpart    partial sums of the row-parallel GEMVs (LC_MAX x ldp)
//   hpart, h partial and final re-orthogonalisation coefficients (RC_MAX x d_max, d_max)
//   nu2part  per-row-block partial squared norms (RB)
//   rb_cnt, lb_cnt, gcnt   last-arriver counters (zero at rest)
//   gslot    per-column-group partial dot products (ngroups x KMAX x C)
//   gsum     per-column-group sums of e_j (ngroups)
//   pbest_e/j  per-CTA argmax candidates of the fused pass (G)
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace rbd {

struct Ctl;

// Fused-pass tile configuration, per number of FP32 planes (2 = FP64 input, 1 = FP32 input).
// bf16 storage uses its own configuration (PassCfgBf16).
template <int P>
struct PassCfg {
    static constexpr int NW = 8;                 // consumer warps
    static constexpr int CPW = 2;                // columns per consumer warp
    static constexpr int C = NW * CPW;           // columns per group
    static constexpr int MT = 256;               // rows per tile (two 128-row slabs)
    static constexpr int S = (P == 2) ? 5 : 8;   // pipeline stages
    static constexpr int XI_FLOATS = 2 * MT;     // split pivot-vector tile (hi, lo)
    static constexpr int STAGE_FLOATS = XI_FLOATS + C * P * MT;
    static constexpr int THREADS = (NW + 1) * 32;
    static constexpr size_t SCRATCH = 1024;
    static constexpr size_t SMEM = (size_t)S * STAGE_FLOATS * 4 + 2 * S * 8 + SCRATCH;
};

struct PassCfgBf16 {
    static constexpr int NW = 8;
    static constexpr int CPW = 2;
    static constexpr int C = NW * CPW;
    static constexpr int MT = 512;               // rows per tile (two 256-row slabs)
    static constexpr int S = 8;
    static constexpr int XI_FLOATS = MT;         // hi part of the pivot vector only
    static constexpr int STAGE_BYTES = XI_FLOATS * 4 + C * MT * 2;
    static constexpr int THREADS = (NW + 1) * 32;
    static constexpr size_t SCRATCH = 1024;
    static constexpr size_t SMEM = (size_t)S * STAGE_BYTES + 2 * S * 8 + SCRATCH;
};

constexpr int kGemvRows = 128;     // rows per CTA of the row-parallel GEMVs
constexpr int kGemvTargetCtas = 304;

struct Work {
    // sizes
    int64_t m, n, ldx, ldp, d_max;
    int xt;                 // rbd_dtype
    int planes_n;           // number of planes
    int esize;              // bytes per plane element
    // pass geometry
    int C, MT;
    int64_t NT, ngroups, W;
    int G;                  // pass CTAs
    int KMAX;
    int64_t RB;             // row blocks of the GEMVs (ldp / 128)
    int64_t LC_MAX, RC_MAX;
    int num_sms;
    int evict_first;
    // regions
    Ctl* ctl;
    void* planes;
    float *yh, *yl;
    double *v1, *v2;
    float *v1h, *v1l, *v2h, *v2l;
    double *e, *xn2;
    double* vpart;
    double *hpart, *h;
    double* nu2part;
    uint32_t *rb_cnt, *lb_cnt, *gcnt;
    double *gslot, *gsum;
    double* pbest_e;
    int64_t* pbest_j;
    // bytes of the zero-at-rest prefix (ctl + counters) to clear at call start
    size_t zero_bytes;
    size_t total_bytes;
    unsigned char* base;
};

// Fill sizes/geometry of `w` (no pointers); returns false on unsupported sizes.
bool plan_work(Work& w, int64_t m, int64_t n, int64_t ldx, int64_t d_max, int xt, int num_sms);
// Carve the regions of `w` out of `base` (at least w.total_bytes, 256-byte aligned).
void carve_work(Work& w, void* base);

// ---- launchers (each returns the cudaError_t of its launch) ----
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
// Dynamic shared-memory opt-in for the pass kernels (once per device).
cudaError_t pass_kernel_setup();

}  // namespace rbd
