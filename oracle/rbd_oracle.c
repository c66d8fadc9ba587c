/*
 * rbd_oracle.c -- plain, slow FP64 CPU oracle for Reduced Basis Decomposition.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  The product (the CUDA library) never calls it and
 * shares no code with it.
 *
 * What it follows (Y. Chen, "Reduced Basis Decomposition: a Certified and Fast Lossy Data
 * Compression Algorithm", arXiv 1503.05947):
 *   - Algorithm 1 (Section 3.1), taken step by step in the paper's order:
 *       1.   d = 1, E_cur = +inf, i = start column;
 *       2.1  v = X(:, i);
 *       2.2  modified Gram-Schmidt of v against xi_1..xi_{d-1}; break if ||v|| < eps_R;
 *            else xi_d = v / ||v||, Y(:, d) = xi_d, T(d, :) = xi_d' X;
 *       2.3  E_cur = max_j ||X(:, j) - Y(:, 1:d) T(:, j)||, i = argmax_j of the same;
 *       2.4  stop if E_cur <= eps_R, else d = d + 1.
 *   - Section 3.2, Eq. (evalerr) with A = I: the error of column j is its Euclidean residual.
 *     The oracle evaluates it from the DEFINITION, as the norm of the explicit residual
 *     R(:, j) = X(:, j) - sum_{l <= d} xi_l T(l, j), the terms summed in the order l = 1..d.
 *   - Section 3.2 with a general DIAGONAL A = diag(w), w_r > 0 (rbd_oracle_compress_weighted):
 *     the basis stays the Euclidean Gram-Schmidt basis of Algorithm 1 and T = Y' X, and only the
 *     error of step 2.3 is measured in the A-norm, ||v||_A = sqrt(sum_r w_r v_r^2) (Eq. (evalerr)
 *     with c = T(:, j) = Y' v; the paper pre-computes Y'AX and Y'AY for it, which an
 *     A-orthonormal basis would not need).  The oracle evaluates ||R(:, j)||_A of the explicit
 *     residual; step 2.2's break test and step 2.4's E_cur use the same A-norm, the
 *     normalisation xi_d = v / ||v|| and the rank floor stay Euclidean.
 *   - Section 3.1, "Evaluate the compression of out-of-sample data": v_C = Y' v.
 *   - Section 3.1, "Uncompress": X(:, j) ~ Y T(:, j).
 *
 * Readings where the paper is silent or garbled (all shared with the CUDA path's contract):
 *   - 0-based indices; the start column is an argument (Algorithm 1 step 1 allows "a user
 *     input").
 *   - Modified Gram-Schmidt is applied twice (one re-orthogonalisation sweep).
 *   - argmax ties resolve to the lowest column index.
 *   - norms are Euclidean (A = I); step 2.2 breaks on ||v|| < eps_R (strict), step 2.4 stops on
 *     E_cur <= eps_R, both as printed.
 *   - step 2.2 also breaks when ||v|| <= rank_floor * ||X(:, i)|| (a numerical-rank floor; the
 *     paper's test alone never fires when eps_R = 0 and would then normalise rounding noise).
 *   - the line "T = T(:, 1:d-1)" of step 2.2 is read as T = T(1:d-1, :) (T is d x n).
 *   - tolerance modes: MAXCOL_ABS uses eps_R = tol; MAXCOL_REL uses eps_R = tol * max_j ||x_j||;
 *     FRO_REL stops in step 2.4 when ||X - Y T||_F <= tol ||X||_F and uses
 *     eps_R = tol ||X||_F / sqrt(n) in step 2.2.
 *
 * Compiled with -O2 -ffp-contract=off and no fast-math: every sum is a plain left-to-right
 * loop in IEEE double.
 *
 * Parity pins: this file is checked (tests/test_oracle_*.py) against orthonormality, the
 * definition of the indicator recomputed from scratch, Householder QR of the pivot columns,
 * brute-force least-squares pivots on tiny inputs, closed forms on orthogonal columns, exact
 * recovery of the paper's rank-1/2/3 functions (Section 4.2.1), the paper's pointwise error
 * bound for its 5001 x 5001 example (Section 4.2.2) and the Eckart-Young bound; the diagonal
 * A-norm form against the A-norm indicator recomputed from scratch, least-squares brute force
 * in the A-norm, closed forms on coordinate-aligned columns, termination and scaling.  Planted
 * mistakes (RBD_ORACLE_MUTANT) must each fail at least one of those pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENONFINITE 4

#define TOL_MAXCOL_ABS 0
#define TOL_MAXCOL_REL 1
#define TOL_FRO_REL 2

#ifndef RBD_ORACLE_MUTANT
#define RBD_ORACLE_MUTANT 0
#endif

/* sum_r a[r] * b[r], left to right */
static double dot(const double* a, const double* b, int64_t m) {
    double s = 0.0;
    for (int64_t r = 0; r < m; ++r) s += a[r] * b[r];
    return s;
}

static double norm2(const double* a, int64_t m) { return sqrt(dot(a, a, m)); }

/* ||a||_A = sqrt(sum_r w[r] a[r]^2) for A = diag(w), left to right; w == NULL is A = I. */
static double norm_a(const double* a, const double* w, int64_t m) {
    if (!w) return norm2(a, m);
    double s = 0.0;
    for (int64_t r = 0; r < m; ++r) s += w[r] * (a[r] * a[r]);
    return sqrt(s);
}

int rbd_oracle_version(void) { return 1; }

#ifdef _OPENMP
#include <omp.h>
/* The OpenMP build (the all-core CPU baseline): threads for the column loops of Algorithm 1. */
void rbd_oracle_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int rbd_oracle_threads(void) { return omp_get_max_threads(); }
#else
void rbd_oracle_set_threads(int n) { (void)n; }
int rbd_oracle_threads(void) { return 1; }
#endif

/*
 * Algorithm 1.  X is m x n column-major (leading dimension ldx).  Outputs, with capacity d_max:
 *   Y       m x d_max, column-major (ldy): Y(:, k) = xi_k
 *   T       d_max x n, column-major (ldt): T(k, :) = xi_k' X
 *   pivots  pivots[k] = column of X whose orthonormalisation gave xi_k
 *   err     err[k]   = E_cur after basis k was added = max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)||
 *   nu      nu[k]    = ||v|| of step 2.2 for basis k (the true residual of column pivots[k]
 *                      against bases 0..k-1)
 *   fro     fro[k]   = ||X - Y(:, 0:k) T(0:k, :)||_F
 *   next_pivot       = the argmax of the last step 2.3 (the column the next basis would use)
 *   d_out            = number of bases produced
 */
static int compress_core(const double* X, int64_t m, int64_t n, int64_t ldx, const double* w, double tol,
                         int mode, int64_t d_max, int64_t start, double rank_floor, double* Y, int64_t ldy,
                         double* T, int64_t ldt, int64_t* pivots, double* err, double* nu, double* fro,
                         int64_t* next_pivot, int64_t* d_out) {
    if (!X || !Y || !T || !pivots || !err || !nu || !fro || !next_pivot || !d_out) return ORC_EINVAL;
    if (m < 1 || n < 1 || ldx < m || ldy < m || d_max < 1 || ldt < d_max) return ORC_EINVAL;
    if (d_max > m || d_max > n) return ORC_EINVAL;
    if (start < 0 || start >= n) return ORC_EINVAL;
    if (!(tol >= 0.0) || !(rank_floor >= 0.0)) return ORC_EINVAL;
    if (mode != TOL_MAXCOL_ABS && mode != TOL_MAXCOL_REL && mode != TOL_FRO_REL) return ORC_EINVAL;
    *d_out = 0;
    *next_pivot = start;

    double* R = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* v = (double*)malloc(sizeof(double) * (size_t)m);
    double* ecol = (double*)malloc(sizeof(double) * (size_t)n);
    if (!R || !v || !ecol) {
        free(R);
        free(v);
        free(ecol);
        return ORC_ENOMEM;
    }

    /* R = X; column norms for the relative tolerance modes. */
    double maxcol = 0.0, fro2x = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const double* xj = X + j * ldx;
        for (int64_t r = 0; r < m; ++r) {
            if (!isfinite(xj[r])) {
                free(R);
                free(v);
                free(ecol);
                return ORC_ENONFINITE;
            }
            R[j * m + r] = xj[r];
        }
        double nj = norm_a(xj, w, m);
        if (nj > maxcol) maxcol = nj;
        fro2x += nj * nj;
    }
    double frox = sqrt(fro2x);
    double eps_r = tol;
    if (mode == TOL_MAXCOL_REL) eps_r = tol * maxcol;
    if (mode == TOL_FRO_REL) eps_r = tol * frox / sqrt((double)n);

    int64_t i = (RBD_ORACLE_MUTANT == 4) ? 0 : start; /* step 1 */
    int64_t d = 0;     /* number of bases built so far (the paper's d - 1) */
    while (d < d_max) {
        /* step 2.1 */
        memcpy(v, X + i * ldx, sizeof(double) * (size_t)m);
        double xin = norm2(v, m);
        /* step 2.2: modified Gram-Schmidt, then one re-orthogonalisation sweep */
        int sweeps = (RBD_ORACLE_MUTANT == 1) ? 1 : 2;
        for (int s = 0; s < sweeps; ++s) {
            int64_t jend = (RBD_ORACLE_MUTANT == 10) ? d - 1 : d;
            for (int64_t j = 0; j < jend; ++j) {
                const double* xi = Y + j * ldy;
                double c = dot(v, xi, m);
                if (RBD_ORACLE_MUTANT == 2) c = -c;
                for (int64_t r = 0; r < m; ++r) v[r] -= c * xi[r];
            }
        }
        double vn = norm2(v, m);
        double vna = (RBD_ORACLE_MUTANT == 15) ? vn : norm_a(v, w, m);
        if (vna < eps_r || vn <= rank_floor * xin) break;
        double* xi = Y + d * ldy;
        for (int64_t r = 0; r < m; ++r) xi[r] = (RBD_ORACLE_MUTANT == 6) ? v[r] : v[r] / vn;
        /* T(d, :) = xi_d' X (columns are independent; an OpenMP build gives each to one thread) */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            T[j * ldt + d] = dot((RBD_ORACLE_MUTANT == 7) ? v : xi, X + j * ldx, m);
        /* step 2.3: explicit residual and its column norms (independent columns), then their sum,
           max and argmax (lowest index) in column order */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
            double c = T[j * ldt + d];
            double* rj = R + j * m;
            for (int64_t r = 0; r < m; ++r) rj[r] -= c * xi[r];
            double ej = (RBD_ORACLE_MUTANT == 14) ? norm2(rj, m) : norm_a(rj, w, m);
            if (RBD_ORACLE_MUTANT == 5) ej = ej * ej;
            ecol[j] = ej;
        }
        double ecur = -1.0, fro2 = 0.0;
        int64_t inext = 0;
        for (int64_t j = 0; j < n; ++j) {
            double ej = ecol[j];
            fro2 += ej * ej;
            int better = (RBD_ORACLE_MUTANT == 3) ? (ej >= ecur) : (ej > ecur);
            if (better) {
                ecur = ej;
                inext = j;
            }
        }
        pivots[d] = i;
        nu[d] = vn;
        err[d] = ecur;
        fro[d] = sqrt(fro2);
        d += 1;
        i = inext;
        /* step 2.4 */
        int stop;
        if (mode == TOL_FRO_REL)
            stop = ((RBD_ORACLE_MUTANT == 9) ? fro2 : sqrt(fro2)) <= tol * frox;
        else
            stop = (RBD_ORACLE_MUTANT == 8) ? (ecur < eps_r) : (ecur <= eps_r);
        if (stop) break;
    }
    *d_out = d;
    *next_pivot = i;
    free(R);
    free(v);
    free(ecol);
    return ORC_OK;
}

int rbd_oracle_compress(const double* X, int64_t m, int64_t n, int64_t ldx, double tol, int mode,
                        int64_t d_max, int64_t start, double rank_floor, double* Y, int64_t ldy,
                        double* T, int64_t ldt, int64_t* pivots, double* err, double* nu,
                        double* fro, int64_t* next_pivot, int64_t* d_out) {
    return compress_core(X, m, n, ldx, NULL, tol, mode, d_max, start, rank_floor, Y, ldy, T, ldt, pivots, err,
                         nu, fro, next_pivot, d_out);
}

/*
 * Algorithm 1 with the error of steps 2.2-2.4 in the A-norm of A = diag(w) (Section 3.2, "general
 * diagonal matrix"): w holds m weights, each finite and > 0.  Outputs as rbd_oracle_compress, with
 * err[k] = max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)||_A and fro[k] = sqrt(sum_j ||.||_A^2); nu[k] stays
 * the Euclidean ||v|| that normalises xi_k.  The relative tolerance modes scale by max_j ||x_j||_A and
 * sqrt(sum_j ||x_j||_A^2).
 */
int rbd_oracle_compress_weighted(const double* X, int64_t m, int64_t n, int64_t ldx, const double* w, double tol,
                                 int mode, int64_t d_max, int64_t start, double rank_floor, double* Y, int64_t ldy,
                                 double* T, int64_t ldt, int64_t* pivots, double* err, double* nu, double* fro,
                                 int64_t* next_pivot, int64_t* d_out) {
    if (!w || m < 1) return ORC_EINVAL;
    for (int64_t r = 0; r < m; ++r)
        if (!isfinite(w[r]) || !(w[r] > 0.0)) return ORC_EINVAL;
    return compress_core(X, m, n, ldx, w, tol, mode, d_max, start, rank_floor, Y, ldy, T, ldt, pivots, err, nu,
                         fro, next_pivot, d_out);
}

/* Out-of-sample map (Section 3.1): C(:, k) = Y' V(:, k) for k < nv; C is d x nv (ldc). */
int rbd_oracle_project(const double* Y, int64_t m, int64_t d, int64_t ldy, const double* V,
                       int64_t nv, int64_t ldv, double* C, int64_t ldc) {
    if (!Y || !V || !C || m < 1 || d < 0 || nv < 0 || ldy < m || ldv < m || ldc < d) return ORC_EINVAL;
    for (int64_t k = 0; k < nv; ++k)
        for (int64_t l = 0; l < d; ++l) C[k * ldc + l] = dot(Y + l * ldy, V + k * ldv, m);
    return ORC_OK;
}

/*
 * Adjoint of the differentiation form (not in the paper): for the FIXED pivot set P of a
 * compression, with A = X(:, P) = Y R (Gram-Schmidt in pivot order: Y = Q, R = T(:, P) upper
 * triangular) and T = Y' X,
 *     L(X) = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2      (Xo fixed out-of-sample data).
 * Writing P_A = A A^+ (the orthogonal projector onto span A), L = w_rec tr(X'(I - P_A)X) +
 * w_proj tr(Xo' P_A Xo), and the projector derivative dP_A = (I - P_A) dA A^+ + (A^+)' dA' (I - P_A)
 * with A^+ = R^-1 Y' give
 *     dL/dX          = 2 w_rec E,                                   E = X - Y T,
 *     dL/dX(:, P)   += [-2 w_rec E T' + 2 w_proj (Xo - Y C) C'] R^-T, C = Y' Xo.
 * Steps in this order: E; C; Z = -2 w_rec E T' + 2 w_proj (Xo - Y C) C' (m x d); W = Z R^-T by
 * back substitution row by row (W R' = Z, R upper triangular); G = 2 w_rec E; G(:, P(l)) += W(:, l);
 * loss = w_rec ||E||_F^2 + w_proj ||C||_F^2.  Plain FP64 loops.
 */
int rbd_oracle_grad(const double* X, int64_t m, int64_t n, int64_t ldx, const double* Y, int64_t ldy,
                    const double* T, int64_t ldt, const int64_t* piv, int64_t d, const double* Xo, int64_t k,
                    int64_t ldxo, double w_rec, double w_proj, double* G, int64_t ldg, double* loss) {
    if (!X || !Y || !T || !G || !loss || m < 1 || n < 1 || d < 0 || d > n || d > m || k < 0) return ORC_EINVAL;
    if (ldx < m || ldy < m || ldt < (d > 0 ? d : 1) || ldg < m || (k > 0 && (!Xo || ldxo < m))) return ORC_EINVAL;
    if (d > 0 && !piv) return ORC_EINVAL;
    double* E = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double* C = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1) * (size_t)(k > 0 ? k : 1));
    double* Z = (double*)malloc(sizeof(double) * (size_t)m * (size_t)(d > 0 ? d : 1));
    if (!E || !C || !Z) {
        free(E);
        free(C);
        free(Z);
        return ORC_ENOMEM;
    }
    /* E = X - Y T */
    double e2 = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t r = 0; r < m; ++r) {
            double v = X[j * ldx + r];
            for (int64_t l = 0; l < d; ++l) v -= Y[l * ldy + r] * T[j * ldt + l];
            E[j * m + r] = v;
            e2 += v * v;
        }
    /* C = Y' Xo */
    double c2 = 0.0;
    for (int64_t q = 0; q < k; ++q)
        for (int64_t l = 0; l < d; ++l) {
            double v = dot(Y + l * ldy, Xo + q * ldxo, m);
            C[q * d + l] = v;
            c2 += v * v;
        }
    /* Z = -2 w_rec E T' + 2 w_proj (Xo - Y C) C' */
    for (int64_t l = 0; l < d; ++l)
        for (int64_t r = 0; r < m; ++r) {
            double a = 0.0;
            for (int64_t j = 0; j < n; ++j) a += E[j * m + r] * T[j * ldt + l];
            double b = 0.0;
            for (int64_t q = 0; q < k; ++q) {
                double res = Xo[q * ldxo + r];
                for (int64_t l2 = 0; l2 < d; ++l2) res -= Y[l2 * ldy + r] * C[q * d + l2];
                b += res * C[q * d + l];
            }
            double zr = (RBD_ORACLE_MUTANT == 12) ? (2.0 * w_rec * a + 2.0 * w_proj * b)
                                                  : (-2.0 * w_rec * a + 2.0 * w_proj * b);
            Z[l * m + r] = zr;
        }
    /* W = Z R^-T: for each row, W R' = Z with R(a, b) = T(a, P(b)) upper triangular */
    if (RBD_ORACLE_MUTANT != 11) {
        for (int64_t r = 0; r < m; ++r)
            for (int64_t a = d - 1; a >= 0; --a) {
                double v = Z[a * m + r];
                for (int64_t b = a + 1; b < d; ++b) v -= Z[b * m + r] * T[piv[b] * ldt + a];
                Z[a * m + r] = v / T[piv[a] * ldt + a];
            }
    }
    /* G = 2 w_rec E, then the pivot columns */
    for (int64_t j = 0; j < n; ++j)
        for (int64_t r = 0; r < m; ++r) G[j * ldg + r] = 2.0 * w_rec * E[j * m + r];
    if (RBD_ORACLE_MUTANT != 13)
        for (int64_t l = 0; l < d; ++l)
            for (int64_t r = 0; r < m; ++r) G[piv[l] * ldg + r] += Z[l * m + r];
    *loss = w_rec * e2 + w_proj * c2;
    free(E);
    free(C);
    free(Z);
    return ORC_OK;
}

/* Uncompress (Section 3.1): Xr(:, j) = Y T(:, j), summed over bases l = 0..d-1 in order. */
int rbd_oracle_reconstruct(const double* Y, int64_t m, int64_t d, int64_t ldy, const double* T,
                           int64_t n, int64_t ldt, double* Xr, int64_t ldx) {
    if (!Y || !T || !Xr || m < 1 || d < 0 || n < 0 || ldy < m || ldt < d || ldx < m) return ORC_EINVAL;
    for (int64_t j = 0; j < n; ++j) {
        double* xr = Xr + j * ldx;
        for (int64_t r = 0; r < m; ++r) xr[r] = 0.0;
        for (int64_t l = 0; l < d; ++l) {
            double c = T[j * ldt + l];
            const double* y = Y + l * ldy;
            for (int64_t r = 0; r < m; ++r) xr[r] += y[r] * c;
        }
    }
    return ORC_OK;
}
