/*
 * rbd.h -- C ABI of the GB300 (sm_103a) Reduced Basis Decomposition library, librbd.so.
 *
 * Reduced Basis Decomposition (Y. Chen, "Reduced Basis Decomposition: a Certified and Fast
 * Lossy Data Compression Algorithm", arXiv 1503.05947) approximates a data matrix
 * X in R^{m x n} by Y T, Y in R^{m x d} with orthonormal columns and T in R^{d x n}, through
 * the greedy loop of Algorithm 1 (Section 3.1).  Every step of that loop runs in this
 * library's CUDA kernels on the GPU; nothing falls back to the CPU.
 *
 * Conventions for every entry point:
 *   - Matrices are COLUMN-MAJOR with an explicit leading dimension (ld >= number of rows):
 *     element (r, c) of a matrix A with leading dimension lda is A[r + c * lda].
 *     Column j of X is the data entry X(:, j) of Section 3.1.
 *   - Indices are 0-based (the paper counts from 1).
 *   - Unless stated otherwise, array pointers are DEVICE pointers owned by the caller; the
 *     library neither frees nor keeps them after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *     device work of a call is ordered on that stream.
 *   - Errors are returned as rbd_status codes.  No call aborts, traps or throws.  Device-side
 *     conditions (non-finite input, a bounded wait that ran out) are reported through the
 *     status of the call that launched the kernels; such a call synchronises `stream`.
 *   - The library is not re-entrant on a single stream for overlapping calls that share a
 *     workspace; distinct workspaces on distinct streams may run concurrently.
 *   - Scratch that a call allocates itself (stream-ordered, freed on the stream before the call
 *     returns) comes from a memory pool the library creates per device.  The pool keeps up to
 *     4 GiB of freed scratch reserved for later calls instead of returning it to the system at
 *     each synchronisation (mapping it again costs about 1 ms per GB); that reserve is held
 *     until the process exits.  Entry points that take a workspace use the caller's instead.
 */
#ifndef RBD_H
#define RBD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rbd_status {
    RBD_OK = 0,
    RBD_EINVAL = 1,        /* an argument is out of range, NULL where required, or misaligned */
    RBD_ENOMEM = 2,        /* device or pinned host allocation failed, or workspace too small */
    RBD_ECUDA = 3,         /* a CUDA runtime call failed (launch error, bad stream, ...) */
    RBD_ENONFINITE = 4,    /* X holds a NaN or an infinity */
    RBD_ETIMEOUT = 5,      /* a bounded device-side wait ran out (the kernel returned early) */
    RBD_EUNSUPPORTED = 6   /* a value outside the supported range (|x| >= 2^127 in the FP64
                              form), or a shape the kernels do not support */
} rbd_status;

/* Storage type of X (and of out-of-sample vectors).  Y, T and all indicators are FP64. */
typedef enum rbd_dtype {
    RBD_F64 = 0,
    RBD_F32 = 1,
    RBD_BF16 = 2,
    /* FP32 storage whose fused pass sums each tile's products in FP32 and folds the sum into an
       FP64-grade accumulator once per tile (as BF16 storage does): the precision form with FP32
       accumulation.  The orthogonalisation, the running indicator and the certified E_cur stay
       FP64-grade; T(k, j) carries the FP32 accumulation error (~2^-20 ||X(:, j)||), so pivots
       near a tie may differ from an FP64 run's.  RBD_F32 keeps FP64-grade dot products.
       rbd_compress and its device-buffer variants (not the weighted, batched or stepwise paths). */
    RBD_F32_ACC32 = 3
} rbd_dtype;

/* How the tolerance `tol` of Algorithm 1 (epsilon_R) is applied. */
typedef enum rbd_tol_mode {
    /* Algorithm 1 as printed: step 2.4 stops when E_cur = max_j ||X(:,j) - Y T(:,j)|| <= tol,
       step 2.2 breaks when the orthogonalised pivot has ||v|| < tol. */
    RBD_TOL_MAXCOL_ABS = 0,
    /* the same with epsilon_R = tol * max_j ||X(:,j)||. */
    RBD_TOL_MAXCOL_REL = 1,
    /* step 2.4 stops when ||X - Y T||_F <= tol * ||X||_F (the Frobenius error is the square
       root of the sum of the per-column squared residuals); step 2.2 breaks when
       ||v|| < tol * ||X||_F / sqrt(n). */
    RBD_TOL_FRO_REL = 2,
    /* no tolerance: exactly d_max bases.  Neither step 2.4's test nor step 2.2's break (nor the
       numerical-rank floor) applies; only an orthogonalised vector that is zero or not finite
       stops the loop.  A measurement mode (every pass streams X once whatever the data): past
       X's numerical rank the bases are rounding noise and carry no information.  It runs in the
       four-barrier loop kernel (which forms ||v|| from the orthogonalised vector itself), so
       not with RBD_F32_ACC32; not taken by the batched form. */
    RBD_TOL_NONE = 3
} rbd_tol_mode;

/* Why the greedy loop ended. */
typedef enum rbd_stop_reason {
    RBD_STOP_NONE = 0,
    RBD_STOP_TOL = 1,      /* step 2.4: the error indicator reached the tolerance */
    RBD_STOP_BREAK = 2,    /* step 2.2: the next pivot's orthogonalised norm was below the
                              tolerance, or below the numerical-rank floor (RBD_RANK_FLOOR) */
    RBD_STOP_DMAX = 3      /* d reached d_max */
} rbd_stop_reason;

/* Step 2.2 also breaks when ||v|| <= RBD_RANK_FLOOR * ||X(:, i)|| for the pivot column i:
   such a column already lies in span(Y) up to rounding, and normalising it would add a basis
   vector made of rounding noise (the paper's test alone never fires when tol = 0). */
#define RBD_RANK_FLOOR 1e-12

/* Summary written to host memory by rbd_compress / rbd_compress_host. */
typedef struct rbd_result {
    int64_t d;            /* number of bases produced (columns of Y, rows of T) */
    int64_t next_pivot;   /* argmax of the last step 2.3: the column the next basis would use */
    int32_t stop_reason;  /* an rbd_stop_reason */
    int32_t launches;     /* kernels this call launched */
    double err_last;      /* E_cur after the last basis (max column residual), 0 if d = 0 */
    double fro_last;      /* ||X - Y T||_F after the last basis, from the summed indicators */
    double x_fro;         /* ||X||_F */
    double x_maxcol;      /* max_j ||X(:, j)|| */
} rbd_result;

/* Bytes of device workspace rbd_compress needs for these sizes (0 on invalid sizes).
   The workspace holds the re-laid-out X (the same number of bytes as an FP64 X for
   RBD_F64, as the input for RBD_F32/RBD_BF16, with columns padded to 128 rows), one split
   FP32 copy of Y, and O(m + n + d_max) vectors. */
size_t rbd_compress_workspace_bytes(int64_t m, int64_t n, int64_t d_max, rbd_dtype xt);

/*
 * rbd_compress -- Algorithm 1 of Section 3.1: (Y, T) = RBD(X, epsilon_R, d_max).
 *
 *  X       [in]  device, m x n column-major, leading dimension ldx >= m, storage type xt.
 *                Read only.  For RBD_F64 every element must satisfy |x| < 2^127.
 *  tol     [in]  epsilon_R >= 0, interpreted according to `mode`.
 *  d_max   [in]  1 <= d_max <= min(m, n): capacity of the outputs and the loop limit.
 *  start   [in]  0 <= start < n: the column of step 1 (the paper draws it at random or takes a
 *                user input; pass a random index for the paper's behaviour).
 *  Y       [out] device, m x d_max, column-major, ldy >= m.  Y(:, k) = xi_k.
 *  T       [out] device, d_max x n, column-major, ldt >= d_max.  T(k, :) = xi_k' X.
 *  pivots  [out] device, d_max int64: pivots[k] = the column of X that gave xi_k.
 *  err     [out] device, d_max doubles: err[k] = E_cur of step 2.3 after basis k,
 *                max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)||, evaluated through Eq. (evalerr)
 *                with A = I (squared column norm minus the squared coefficients, FP64).
 *  nu      [out] device, d_max doubles, or NULL: nu[k] = ||v|| of step 2.2 for basis k, the
 *                FP64 residual of column pivots[k] against bases 0..k-1 recomputed from X.
 *  workspace, workspace_bytes
 *          [in]  device scratch of at least rbd_compress_workspace_bytes(m, n, d_max, xt)
 *                bytes, 256-byte aligned; or NULL/0, in which case the call allocates it
 *                stream-ordered from the library's pool and frees it before returning.
 *  stream  [in]  cudaStream_t as void*.
 *  result  [out] host, or NULL: summary (d, stop reason, last indicator, norms of X).
 *
 *  Only the first `d` columns of Y, rows of T and entries of pivots/err/nu are written.
 *  The call synchronises `stream` once at the end (to learn d); every step of the loop is
 *  ordered on `stream` without host round trips.
 *  Errors: RBD_EINVAL for bad sizes, leading dimensions, start, tol, mode, dtype or NULL
 *  outputs; RBD_ENOMEM if the workspace is too small or cannot be allocated;
 *  RBD_ENONFINITE if X holds NaN/Inf; RBD_EUNSUPPORTED for |x| >= 2^127 in the FP64 form;
 *  RBD_ETIMEOUT / RBD_ECUDA for device failures.  On error the outputs are unspecified.
 */
rbd_status rbd_compress(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                        double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                        double* Y, int64_t ldy, double* T, int64_t ldt,
                        int64_t* pivots, double* err, double* nu,
                        void* workspace, size_t workspace_bytes,
                        void* stream, rbd_result* result);

/*
 * rbd_compress_weighted -- Algorithm 1 with the error measured in the A-norm of a diagonal
 * A = diag(w) (Section 3.2, "general diagonal matrix": some components of each entry are to be
 * kept better than others), ||v||_A = sqrt(sum_r w[r] v[r]^2).
 *
 *  Reading of the paper: the bases stay the Euclidean Gram-Schmidt bases of step 2.2 and
 *  T = Y' X as in rbd_compress (the paper expands Y'AX and Y'AY to evaluate Eq. (evalerr) for
 *  c = T(:, j), which an A-orthonormal basis would not need); the A-norm enters the indicator of
 *  step 2.3 and the tolerance tests of steps 2.2 and 2.4.
 *
 *  w       [in]  device, m doubles, 8-byte aligned, each finite and > 0 (checked on the device:
 *                RBD_EINVAL otherwise).  Read only; caller-owned.
 *  Other arguments, outputs and errors as rbd_compress, with these differences:
 *  err     [out] err[k] = max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)||_A (certified: the A-norm of
 *                the residual of the column that attains it, recomputed from X).
 *  nu      [out] nu[k] stays the Euclidean ||v|| of step 2.2 that normalises xi_k.
 *  tol     MAXCOL_ABS compares err with tol; MAXCOL_REL scales tol by max_j ||x_j||_A; FRO_REL
 *          stops when sqrt(sum_j ||x_j - Y T(:, j)||_A^2) <= tol * sqrt(sum_j ||x_j||_A^2).
 *  result  x_fro and x_maxcol are the A-norm values.
 *  The numerical-rank floor of step 2.2 stays Euclidean.  The workspace is the one of
 *  rbd_compress_workspace_bytes.  RBD_EUNSUPPORTED where the persistent loop kernel does not fit
 *  (more than 512 rows per SM), since the A-norm form runs in that kernel only.
 */
rbd_status rbd_compress_weighted(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                                 const double* w, double tol, rbd_tol_mode mode, int64_t d_max,
                                 int64_t start, double* Y, int64_t ldy, double* T, int64_t ldt,
                                 int64_t* pivots, double* err, double* nu,
                                 void* workspace, size_t workspace_bytes,
                                 void* stream, rbd_result* result);

/*
 * rbd_compress_rows -- the row-space form (Section 3.1: each column of the data matrix is an
 * entry, "or row if we are compressing the row space"): Algorithm 1 on the ROWS of X, i.e.
 * rbd_compress applied to X' (n x m).
 *
 *  X       [in]  device, m x n column-major, ldx >= m, storage type xt (read only).  The call
 *                transposes it once into a stream-ordered scratch copy of m * n elements.
 *  start   [in]  0 <= start < m: the row of step 1.
 *  Y       [out] device, n x d_max, column-major, ldy >= n: the bases of the row space.
 *  T       [out] device, d_max x m, column-major, ldt >= d_max: T(k, i) = xi_k' X(i, :)'.
 *  pivots  [out] row indices of X; err, nu, result as rbd_compress (over rows).
 *  Requires 1 <= d_max <= min(m, n).  Errors as rbd_compress; RBD_ENOMEM if the scratch copy
 *  cannot be allocated.  The workspace is always library-allocated.
 */
rbd_status rbd_compress_rows(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                             double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                             double* Y, int64_t ldy, double* T, int64_t ldt,
                             int64_t* pivots, double* err, double* nu,
                             void* stream, rbd_result* result);

/*
 * rbd_compress_resume -- continue a compression to a larger d_max: Algorithm 1's loop picks up
 * after d0 bases from its outputs (a checkpoint of the greedy state).
 *
 *  X, xt, m, n, ldx, tol, mode, workspace, stream, result  as for rbd_compress (the same X,
 *                tolerance and mode as the call being continued).
 *  d0          [in]  1 <= d0 <= d_max: bases already in Y, T, pivots (and err, nu).
 *  next_pivot  [in]  the column the next basis uses (rbd_result.next_pivot of that call).
 *  d_max       [in]  the new limit; Y, T, pivots, err, nu must have capacity d_max, and hold the
 *                    first d0 columns / rows / entries.
 *  The running indicator e_j, the Frobenius residual and the split copy of Y are rebuilt from
 *  Y(:, 0:d0), T(0:d0, :) and pivots with the operations and order the loop used.  On the
 *  stepwise path the continued run then gives the bits of one rbd_compress call with this d_max.
 *  The persistent two-barrier kernel forms each basis at the start of the next one (its second
 *  Gram-Schmidt sweep is deferred); resumed at d0 it takes basis d0 - 1 as the caller's Y holds
 *  it, so the continued run has the same pivots, d and stop as one call, and Y, T, err and nu
 *  equal to its accuracy rather than bit for bit.  err[d0 - 1] is rewritten (certified again);
 *  entries from d0 on are new.
 *  Errors: those of rbd_compress, and RBD_EINVAL for d0 or next_pivot out of range.
 */
rbd_status rbd_compress_resume(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                               double tol, rbd_tol_mode mode, int64_t d0, int64_t next_pivot,
                               int64_t d_max, double* Y, int64_t ldy, double* T, int64_t ldt,
                               int64_t* pivots, double* err, double* nu,
                               void* workspace, size_t workspace_bytes,
                               void* stream, rbd_result* result);

/*
 * rbd_compress_host -- rbd_compress on HOST buffers (end-to-end form).
 *
 * Same arguments and layout as rbd_compress, but X, Y, T, pivots, err and nu (nu may be
 * NULL) are HOST pointers.  The call allocates device buffers stream-ordered, copies X to
 * the device, runs the loop, copies the first d columns/rows/entries back and frees the
 * device buffers.  Pinned host buffers make the copies asynchronous DMA transfers; pageable
 * ones work but are staged by the CUDA driver.  Returns after the results are in host memory.
 */
rbd_status rbd_compress_host(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                             double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                             double* Y, int64_t ldy, double* T, int64_t ldt,
                             int64_t* pivots, double* err, double* nu,
                             void* stream, rbd_result* result);

/* Size of the fixed device workspace of rbd_compress_noalloc (64 MiB per device). */
#define RBD_NOALLOC_SCRATCH_BYTES (64u << 20)

/*
 * rbd_compress_noalloc -- rbd_compress without any memory allocation.  The paper has no
 * counterpart: this is a deployment form of Algorithm 1, with the same arguments, layout,
 * outputs and results as rbd_compress, but its workspace is a fixed array of
 * RBD_NOALLOC_SCRATCH_BYTES in device memory that belongs to the library (one per device).
 *
 * For callers that cannot allocate while they compress: a serving loop that bans allocator
 * calls on its hot path (device allocation may synchronise the device or grow a memory pool),
 * a process whose device memory is already held by another caching allocator, or code under
 * a hard memory cap.  The call allocates nothing: no device memory, no pinned or mapped host
 * memory, no CUDA events (so rbd_set_profiling has no effect on it).
 *
 *  X, xt, m, n, ldx, tol, mode, d_max, start, Y, ldy, T, ldt, pivots, err, nu, stream, result
 *          as for rbd_compress (device pointers; result on the host).
 *
 *  The first call on a device, made with that device current, sets the kernels' attributes
 *  and looks up the array's device address (cudaGetSymbolAddress); make it before any stream
 *  capture begins.  The call synchronises `stream` at its end, like rbd_compress.
 *  Calls that overlap on one device (several host threads, or several streams) share the one
 *  array and race: the caller must serialise them.
 *  result->launches counts the kernels this call enqueued: the stepwise path (RBD_STEPWISE=1,
 *  or a problem the persistent kernel cannot take) enqueues every step up to d_max, and the
 *  steps after the stop return at entry, so the count can exceed rbd_compress's.
 *  Errors: those of rbd_compress, and RBD_ENOMEM when the workspace these sizes need
 *  (rbd_compress_workspace_bytes) is larger than RBD_NOALLOC_SCRATCH_BYTES -- for an FP64 X
 *  roughly m * n <= 7 million elements (less when d_max is a large fraction of m).
 */
rbd_status rbd_compress_noalloc(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                                double tol, rbd_tol_mode mode, int64_t d_max, int64_t start,
                                double* Y, int64_t ldy, double* T, int64_t ldt,
                                int64_t* pivots, double* err, double* nu,
                                void* stream, rbd_result* result);

/*
 * rbd_project -- the out-of-sample map of Section 3.1, v_C = Y' v, for k vectors at once:
 * C = Y' V.
 *
 *  Y  [in]  device, m x d FP64 column-major, ldy >= m (orthonormal columns from rbd_compress).
 *  V  [in]  device, m x k column-major, ldv >= m, storage type vt.
 *  C  [out] device, d x k FP64 column-major, ldc >= d.
 *  d = 0 or k = 0 is a no-op.  Stream-ordered; does not synchronise.  For tall Y the rows are
 *  split across CTAs and a stream-ordered scratch of (splits x d x k) doubles holds the partial
 *  products (allocated from the library's pool and freed on the stream; if that allocation fails the
 *  rows are not split).  Dot products are
 *  evaluated with FP64-grade (float-float, relative error below 2^-44) accuracy.
 *  Errors: RBD_EINVAL for bad sizes/leading dimensions/NULL; RBD_ECUDA on launch failure.
 */
rbd_status rbd_project(const double* Y, int64_t m, int64_t d, int64_t ldy,
                       const void* V, rbd_dtype vt, int64_t k, int64_t ldv,
                       double* C, int64_t ldc, void* stream);

/*
 * rbd_reconstruct -- "Uncompress" of Section 3.1: Xr = Y T, i.e. column j of the approximation
 * of X is Y T(:, j) (and Y c for a compressed out-of-sample vector c = rbd_project's output).
 *
 *  Y   [in]  device, m x d FP64 column-major, ldy >= m.
 *  T   [in]  device, d x n FP64 column-major, ldt >= d (pass T + j0 * ldt for columns j0..).
 *  Xr  [out] device, m x n FP64 column-major, ldxr >= m.
 *  d = 0 writes zeros; n = 0 is a no-op.  Stream-ordered; does not synchronise.  Sums over the d
 *  bases are evaluated in order with FP64-grade (float-float) accuracy.
 *  Errors: RBD_EINVAL for bad sizes, leading dimensions or NULL pointers; RBD_ECUDA on launch
 *  failure.
 */
rbd_status rbd_reconstruct(const double* Y, int64_t m, int64_t d, int64_t ldy,
                           const double* T, int64_t n, int64_t ldt,
                           double* Xr, int64_t ldxr, void* stream);

/*
 * Batched form (an extension: the paper compresses one matrix at a time): many independent
 * matrices, each with its own sizes, tolerance and outputs, compressed by Algorithm 1 in ONE
 * persistent launch.  The plan orders the matrices by estimated work (m n d, with d the hint or
 * d_max) and gives the largest a team of up to 16 CTAs; each CTA takes the next member slot from
 * the queue and runs that matrix's greedy loop with its team to the end.  Results match
 * rbd_compress on each matrix to its accuracy; the plan's launch shape (rbd_batch_config) changes
 * them by rounding only.
 *
 * Limits: every matrix has m <= 4096 rows and d_max <= 512 (larger matrices: rbd_compress);
 * storage type RBD_F64 or RBD_F32, the same for the whole batch.
 */
typedef struct rbd_instance {
    const void* X;        /* device, m x n column-major, ldx >= m */
    int64_t m, n, ldx;
    double tol;           /* epsilon_R, interpreted by `mode` (an rbd_tol_mode) */
    int32_t mode;
    int32_t d_hint;       /* expected number of bases, or 0 (= d_max): used only to order the
                             queue and size teams of CTAs for large matrices; results do not
                             depend on it */
    int64_t d_max;        /* 1 <= d_max <= min(m, n, 512) */
    int64_t start;        /* 0 <= start < n */
    double* Y;            /* device outputs as for rbd_compress */
    int64_t ldy;
    double* T;
    int64_t ldt;
    int64_t* pivots;
    double* err;
    double* nu;           /* may be NULL */
} rbd_instance;

/* Per-matrix summary of a batched run (device memory, written by the kernels). */
typedef struct rbd_batch_result {
    int64_t d;
    int64_t next_pivot;
    int32_t stop_reason;  /* an rbd_stop_reason */
    int32_t status;       /* RBD_OK, or RBD_ENONFINITE / RBD_EUNSUPPORTED for this matrix */
    double err_last;
    double fro_last;
    double x_fro;
    double x_maxcol;
} rbd_batch_result;

typedef struct rbd_batch_plan_s* rbd_batch_plan;

/* Device workspace a plan needs for this batch (0 if a descriptor is invalid). */
size_t rbd_batch_workspace_bytes(const rbd_instance* inst, int64_t count, rbd_dtype xt);

/* Validate the batch (host array of `count` descriptors), lay the workspace out (caller-owned,
   256-byte aligned, at least rbd_batch_workspace_bytes) and upload the descriptor table on
   `stream` (the call synchronises it).  The plan keeps device pointers only; the descriptors'
   buffers must stay valid while the plan is used.  Errors: RBD_EINVAL, RBD_EUNSUPPORTED (a matrix
   beyond the limits), RBD_ENOMEM (workspace too small), RBD_ECUDA. */
rbd_status rbd_batch_plan_create(rbd_batch_plan* plan, const rbd_instance* inst, int64_t count,
                                 rbd_dtype xt, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* Run the whole batch: a memset, the initial pass over every matrix and the persistent kernel,
   all stream-ordered; no host synchronisation and no allocation, so a run can be captured in a
   CUDA graph and replayed.  results: device array of `count` rbd_batch_result. */
rbd_status rbd_batch_run(rbd_batch_plan plan, rbd_batch_result* results, void* stream);

/* The launch shape of a batched run (one per plan; the tuner picks it per batch). */
typedef struct rbd_batch_config {
    int32_t cols;       /* columns per group of the fused pass: 16 or 32 (a CTA's 8 consumer warps
                           take 2 or 4 columns each) */
    int32_t tile_rows;  /* rows per tile of X streamed into a ring stage: 128 or 256 */
    int32_t team_pct;   /* team sizing: a matrix gets ceil(team_pct / 100 * work / share) member
                           CTAs (share = the batch's work per CTA), at most 16; 75, 150 or 300
                           (default 150) */
    int32_t stages;     /* ring stages of the pass, 2 ..  (128 KiB / stage bytes); 0 = the most */
} rbd_batch_config;

/* Autotuner: time the run of this batch under every launch shape (cols x tile_rows x team_pct,
   each at its deepest ring), then the ring depths of the fastest, and keep the winner in the plan
   (its workspace holds every candidate's layout: rbd_batch_workspace_bytes is the largest).  A
   shape changes the results by rounding only: the tile rows not at all (each column's products
   are summed over the same rows in the same order), the team size the grouping of the sums of h
   and ||v2||^2 over row blocks, the group width that of the Frobenius sum over columns.  A plan
   gives the same bits run after run (and under graph replay).  Synchronises `stream`; the outputs
   hold the results of the last trial.  *chosen (may be NULL) receives the choice. */
rbd_status rbd_batch_tune(rbd_batch_plan plan, rbd_batch_result* results, void* stream,
                          rbd_batch_config* chosen);

/* The plan's current launch shape, and a shape to apply without tuning (e.g. one cached from an
   earlier tuning of a batch like this one).  set_config re-lays the workspace out and uploads the
   descriptor table on `stream` (synchronised).  Errors: RBD_EINVAL for a shape outside the
   values above. */
rbd_status rbd_batch_plan_config(rbd_batch_plan plan, rbd_batch_config* cfg);
rbd_status rbd_batch_plan_set_config(rbd_batch_plan plan, const rbd_batch_config* cfg, void* stream);

rbd_status rbd_batch_plan_destroy(rbd_batch_plan plan);

/* One-shot convenience: plan (with a stream-ordered workspace allocation), run, copy the
   results to the HOST array `results`, destroy.  Synchronises `stream`. */
rbd_status rbd_compress_batched(const rbd_instance* inst, int64_t count, rbd_dtype xt,
                                rbd_batch_result* results, void* stream);

/*
 * rbd_grad -- adjoint of the differentiation form (an extension: the paper has no gradient).
 * For the FIXED pivot set of a compression (Y, T, pivots from rbd_compress: A = X(:, pivots)
 * = Y R with R = T(:, pivots) upper triangular, T = Y' X) and fixed out-of-sample data Xo,
 *     L(X) = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2
 * and its gradient with respect to X,
 *     G = 2 w_rec E,  G(:, pivots) += [-2 w_rec E T' + 2 w_proj (Xo - Y C) C'] R^-T,
 * with E = X - Y T and C = Y' Xo (the out-of-sample map of Section 3.1).
 *
 *  X       [in]  device, m x n, ldx >= m, storage type xt (the matrix that was compressed).
 *  Y, T    [in]  device FP64, m x d (ldy >= m) and d x n (ldt >= d), as rbd_compress wrote them.
 *  pivots  [in]  device, d distinct int64 column indices (rbd_compress's pivots).
 *  d       [in]  0 <= d <= min(m, n, 256).
 *  Xo      [in]  device, m x k, ldxo >= m, storage type xt; may be NULL when k = 0.
 *  w_rec, w_proj [in] weights of the two terms.
 *  G       [out] device FP64, m x n, ldg >= m; or NULL to evaluate the loss only.
 *  loss    [out] device, one double: L(X).
 *  stream  [in]  cudaStream_t as void*.  Stream-ordered; allocates its workspace stream-ordered
 *                (from the library's pool) and frees it; does not synchronise.
 *  Errors: RBD_EINVAL for bad sizes, leading dimensions or NULL arguments; RBD_EUNSUPPORTED for
 *  d > 256; RBD_ENOMEM / RBD_ECUDA on allocation or launch failures.
 */
rbd_status rbd_grad(const void* X, rbd_dtype xt, int64_t m, int64_t n, int64_t ldx,
                    const double* Y, int64_t ldy, const double* T, int64_t ldt,
                    const int64_t* pivots, int64_t d,
                    const void* Xo, int64_t k, int64_t ldxo,
                    double w_rec, double w_proj,
                    double* G, int64_t ldg, double* loss, void* stream);

/*
 * rbd_grad_batched -- rbd_grad for many independent instances at once (the differentiation form
 * of a batch of matrices): each of rbd_grad's kernels is launched once for the whole batch, the
 * out-of-sample map C = Y' Xo once per instance.  Each instance's loss and gradient are those of
 * rbd_grad on it, to the bit (the same kernels and summation order).
 *
 *  items   [in]  host array of `count` descriptors, fields as rbd_grad's arguments; every G is
 *                non-NULL (gradients) or every G is NULL (losses only).
 *  count   [in]  1 .. 65535.
 *  xt, w_rec, w_proj, stream  as for rbd_grad (one storage type and one pair of weights for the
 *                batch).  Stream-ordered; one stream-ordered workspace allocation, freed before
 *                return; does not synchronise.
 *  Errors: those of rbd_grad for any instance; RBD_EINVAL for count out of range or a mix of NULL
 *  and non-NULL G.
 */
typedef struct rbd_grad_item {
    const void* X;        /* device, m x n, ldx >= m */
    int64_t m, n, ldx;
    const double* Y;      /* device FP64, m x d, ldy >= m */
    int64_t ldy;
    const double* T;      /* device FP64, d x n, ldt >= d */
    int64_t ldt;
    const int64_t* pivots;/* device, d entries */
    int64_t d;            /* 0 <= d <= min(m, n, 256) */
    const void* Xo;       /* device, m x k, ldxo >= m; may be NULL when k = 0 */
    int64_t k, ldxo;
    double* G;            /* device FP64, m x n, ldg >= m; or NULL */
    int64_t ldg;
    double* loss;         /* device, one double */
} rbd_grad_item;

rbd_status rbd_grad_batched(const rbd_grad_item* items, int64_t count, rbd_dtype xt,
                            double w_rec, double w_proj, void* stream);

/* Per-kernel timing of the most recent rbd_compress call on this host thread, taken with
   CUDA events recorded on the call's stream around each launch when profiling is enabled
   (rbd_set_profiling(1)).  Times are in milliseconds. */
typedef struct rbd_profile {
    int64_t pass_launches;   /* fused passes over X (one per basis) */
    double pass_ms;          /* stepwise path: summed durations of the pass kernels */
    int64_t orth_launches;   /* stepwise path: orthogonalisation kernels */
    double orth_ms;
    double init_ms;          /* the initial norm / re-layout pass */
    int64_t pass_bytes;      /* algorithmic bytes of X streamed by the passes */
    int64_t loop_launches;   /* persistent path: 1 (the whole greedy loop in one kernel) */
    double loop_ms;          /* persistent path: duration of that kernel */
    int32_t loop_kernel;     /* 1 if the persistent loop kernel ran, 0 for the stepwise path */
    int32_t reserved;
} rbd_profile;

void rbd_set_profiling(int enabled);

/*
 * rbd_set_wait_limit -- bound, in nanoseconds, on every device-side wait of the persistent kernels
 * launched from now on (the loop kernels of rbd_compress and its variants, and the batched run):
 * grid barriers, shared-memory barrier phases, team barriers.  A wait that runs out does not
 * trap: the kernel records RBD_ETIMEOUT, its CTAs leave at their next barrier once their copies
 * in flight have landed, and the call returns RBD_ETIMEOUT (a batched run marks the matrices it
 * stopped).  0 restores the defaults (2 s for barrier waits, 10 s for a batched team barrier).
 * Process-wide; returns the previous setting.  The paper has no counterpart: this is the
 * failure-detection bound of the GPU path, settable so that tests can make a wait run out.
 */
uint64_t rbd_set_wait_limit(uint64_t ns);
rbd_status rbd_get_profile(rbd_profile* out);

const char* rbd_status_string(rbd_status s);

/* Library version: major * 10000 + minor * 100 + patch. */
int rbd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RBD_H */
