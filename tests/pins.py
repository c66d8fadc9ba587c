"""Pins: checks of a compress implementation against what the paper and the mathematics fix.

Each ``pin_*`` takes ``compress(X, tol, d_max, start=0, mode="maxcol_abs")`` returning a dict
with ``Y`` (m x d), ``T`` (d x n), ``pivots``, ``err``, ``nu`` and ``d``, and raises
AssertionError when the implementation disagrees with:

* orthonormality of Y (with one re-orthogonalisation sweep, to a few ulps even when the pivot
  columns are ill-conditioned);
* the definition of the indicator of step 2.3 (max column residual), recomputed from scratch;
* T = Y' X (step 2.2's T(d, :) = xi_d' X, equal to the out-of-sample map on in-sample columns);
* Householder QR (LAPACK) of the pivot columns: Gram-Schmidt of the chosen columns must give
  the same Q and R up to column signs, with R = T(:, pivots) upper triangular;
* brute force on tiny inputs: the next pivot maximises the least-squares residual against the
  span of the columns chosen so far (independent of Gram-Schmidt and of the error update);
* closed forms on exactly orthogonal columns: pivots in decreasing norm order after the start,
  each indicator equal to the largest remaining norm, lowest index on exact ties;
* exact recovery of rank-r data and of the paper's rank-1/2/3 functions (Section 4.2.1);
* the paper's pointwise error bound for its 5001 x 5001 example (Section 4.2.2);
* the Eckart-Young lower bound from the singular values;
* termination exactly as printed in Algorithm 1 (step 2.4 stops on E_cur <= eps_R).

These pins are used on the CPU oracle (tests/test_oracle_pins.py), on oracle builds with
planted mistakes (tests/test_oracle_mutants.py, each mutant must fail at least one pin) and on
the CUDA path (tests/test_gpu_*.py).
"""
from __future__ import annotations

import json
import os

import numpy as np

import gen

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _decay(m, n, seed, rate=0.25, noise=0.0, rank=None):
    r = min(m, n) if rank is None else rank
    s = 2.0 ** (-rate * np.arange(r))
    return gen.lowrank_haar(m, n, s, seed, noise)


def pin_orthonormal(compress):
    """Y'Y = I: on a well-conditioned run and on one whose pivot columns are ill-conditioned
    (singular values down to 1e-13), where one Gram-Schmidt sweep alone loses orthogonality."""
    for X, dmax in ((_decay(300, 200, 1, noise=1e-6), 48),
                    (gen.lowrank_haar(90, 70, 10.0 ** (-np.arange(45) / 3.4), 11), 45)):
        r = compress(X, 0.0, dmax)
        d = r["d"]
        assert d >= 8, f"run too short to test ({d})"
        Y = r["Y"]
        dev = np.abs(Y.T @ Y - np.eye(d)).max()
        assert dev <= 10 * d * EPS, f"|Y'Y - I| = {dev:.3e} > {10 * d * EPS:.3e} (d={d})"


def pin_indicator_definition(compress):
    """err[k] = max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)|| and the argmax is the next pivot."""
    X = _decay(160, 120, 2, rate=0.2, noise=1e-7)
    r = compress(X, 0.0, 30)
    d = r["d"]
    assert d == 30, f"expected 30 bases, got {d}"
    scale = np.linalg.norm(X, axis=0).max()
    for k in range(d):
        R = X - r["Y"][:, :k + 1] @ r["T"][:k + 1, :]
        cn = np.linalg.norm(R, axis=0)
        assert abs(r["err"][k] - cn.max()) <= 1e-12 * scale, f"err[{k}] {r['err'][k]} vs {cn.max()}"
        srt = np.sort(cn)
        if k + 1 < d and srt[-1] - srt[-2] > 1e-9 * scale:
            assert r["pivots"][k + 1] == int(np.argmax(cn)), f"pivot {k + 1}"


def pin_T_is_projection(compress):
    """T = Y' X for every column (in-sample projection)."""
    X = _decay(200, 150, 3, rate=0.15, noise=1e-6)
    r = compress(X, 0.0, 40)
    Tp = r["Y"].T @ X
    scale = np.linalg.norm(X, axis=0)
    dev = (np.abs(r["T"] - Tp) / scale[None, :]).max()
    assert dev <= 1e-13, f"|T - Y'X| / ||x_j|| = {dev:.3e}"


def pin_qr_equivalence(compress):
    """Gram-Schmidt of the pivot columns equals Householder QR of X(:, pivots) (sign-fixed),
    and T(:, pivots) is that upper-triangular R with a positive diagonal."""
    X = _decay(150, 100, 4, rate=0.2, noise=1e-6)
    r = compress(X, 0.0, 25)
    P = r["pivots"]
    q, rr = np.linalg.qr(X[:, P])
    sg = np.sign(np.diag(rr))
    q = q * sg
    rr = rr * sg[:, None]
    assert np.abs(r["Y"] - q).max() <= 1e-10, f"|Y - Q| = {np.abs(r['Y'] - q).max():.3e}"
    tp = r["T"][:, P]
    scale = np.abs(rr).max()
    assert np.abs(np.tril(tp, -1)).max() <= 1e-13 * scale, "T(:, P) not upper triangular"
    assert (np.diag(tp) > 0).all(), "T(:, P) diagonal not positive"
    assert np.abs(tp - rr).max() <= 1e-12 * scale, f"|T(:,P) - R| = {np.abs(tp - rr).max():.3e}"


def pin_bruteforce_tiny(compress):
    """On tiny inputs the next pivot maximises min_c ||x_j - X(:, P) c|| (least squares)."""
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(40):
        m = int(rng.integers(2, 9))
        n = int(rng.integers(2, 9))
        X = np.asfortranarray(rng.standard_normal((m, n)))
        start = int(rng.integers(0, n))
        dmax = min(m, n)
        r = compress(X, 0.0, dmax, start=start)
        assert r["pivots"][0] == start
        scale = np.linalg.norm(X, axis=0).max()
        for k in range(r["d"]):
            A = X[:, r["pivots"][:k + 1]]
            res = np.empty(n)
            for j in range(n):
                c, *_ = np.linalg.lstsq(A, X[:, j], rcond=None)
                res[j] = np.linalg.norm(X[:, j] - A @ c)
            assert abs(r["err"][k] - res.max()) <= 1e-11 * scale, f"trial {trial} step {k}"
            srt = np.sort(res)
            if k + 1 < r["d"] and n > 1 and srt[-1] - srt[-2] > 1e-8 * scale:
                assert r["pivots"][k + 1] == int(np.argmax(res)), f"trial {trial} pivot {k + 1}"
                checked += 1
    assert checked > 20


def pin_closed_form_orthogonal(compress):
    """Orthogonal columns with distinct norms: after the start, pivots follow decreasing norm
    and err[k] is the largest norm not yet chosen (0 once all are chosen)."""
    norms = np.array([3.0, 7.0, 1.0, 5.0, 2.0, 6.0, 4.0])
    X = gen.orthogonal_columns(12, norms, seed=3)
    start = 2
    r = compress(X, 0.0, 7, start=start)
    order = [start] + [int(j) for j in np.argsort(-norms) if j != start]
    assert list(r["pivots"]) == order, f"pivots {list(r['pivots'])} != {order}"
    for k in range(r["d"]):
        remaining = [norms[j] for j in range(7) if j not in order[:k + 1]]
        expect = max(remaining) if remaining else 0.0
        assert abs(r["err"][k] - expect) <= 1e-14 * norms.max(), f"err[{k}] {r['err'][k]} != {expect}"
        assert abs(r["nu"][k] - norms[order[k]]) <= 1e-14 * norms.max(), f"nu[{k}]"


def pin_ties_lowest_index(compress):
    """Exact ties in step 2.3 go to the lowest column index."""
    X = gen.orthogonal_columns(9, np.full(6, 2.0), seed=4)
    r = compress(X, 0.0, 6, start=3)
    assert list(r["pivots"]) == [3, 0, 1, 2, 4, 5], f"pivots {list(r['pivots'])}"


def pin_start_column(compress):
    """Step 1: the first basis comes from the given start column."""
    X = _decay(64, 48, 6, rate=0.3)
    for s in (0, 5, 47):
        r = compress(X, 0.0, 4, start=s)
        assert r["pivots"][0] == s
        x = X[:, s]
        assert np.abs(r["Y"][:, 0] - x / np.linalg.norm(x)).max() <= 1e-15 * 8


def pin_exact_rank(compress):
    """Rank-r data is recovered exactly in r steps (with a tolerance, or through the
    numerical-rank floor of step 2.2 when tol = 0)."""
    for rank in (1, 5, 17):
        rng = np.random.default_rng(100 + rank)
        X = np.asfortranarray(rng.standard_normal((120, rank)) @ rng.standard_normal((rank, 90)))
        for tol, mode in ((1e-10, "maxcol_rel"), (0.0, "maxcol_abs")):
            r = compress(X, tol, 60, mode=mode)
            assert r["d"] == rank, f"rank {rank} tol {tol}: d = {r['d']}"
            res = np.abs(X - r["Y"] @ r["T"]).max()
            assert res <= 1e-12 * np.abs(X).max(), f"rank {rank}: residual {res:.3e}"


def pin_paper_rank_functions(compress):
    """Section 4.2.1: the three tensorial functions are decomposed exactly with d = 1, 2, 3."""
    g = _golden("paper_rank_functions.json")
    for case in g["cases"]:
        X = gen.paper_rank_function(1000, case["which"])
        for tol in (1e-10, 0.0):
            r = compress(X, tol, 10)
            assert r["d"] == case["intrinsic_dimension"], f"{case['function']}: d = {r['d']}"
            assert np.abs(X - r["Y"] @ r["T"]).max() <= 1e-12


def pin_paper_approx_example(compress):
    """Section 4.2.2: 5001 x 5001 grid, d = 22: pointwise error below 1e-6, ratio above 110."""
    g = _golden("paper_approx_example.json")
    X = gen.paper_approx_function(g["grid"])
    r = compress(X, 0.0, g["d"])
    assert r["d"] == g["d"]
    pw = np.abs(X - r["Y"] @ r["T"]).max()
    assert pw < g["pointwise_error_below"], f"pointwise error {pw:.3e}"
    m, n = X.shape
    assert m * n / ((m + n) * r["d"]) > g["compression_ratio_above"]
    # RBD matches SVD: e_S(d) <= e_R(d) (Eckart-Young) and e_R(d) within a small factor of e_S(d)
    from scipy.sparse.linalg import svds
    cmp_ = g["svd_comparison"]
    u, s, vt = svds(X, k=cmp_["d_range"][1] + 2)
    o = np.argsort(s)[::-1]
    u, s, vt = u[:, o], s[o], vt[o]
    xf = float(np.linalg.norm(X))
    for d in range(cmp_["d_range"][0], cmp_["d_range"][1] + 1):
        e_r = np.linalg.norm(X - r["Y"][:, :d] @ r["T"][:d])
        e_s = np.linalg.norm(X - (u[:, :d] * s[:d]) @ vt[:d])
        assert e_r >= e_s * (1 - 1e-6) - 1e-12 * xf, f"d={d}: below the SVD error"
        assert e_r <= cmp_["frobenius_ratio_at_most"] * e_s + 1e-12 * xf, f"d={d}: {e_r:.3e} vs SVD {e_s:.3e}"
    del u, vt


def pin_eckart_young(compress):
    """No rank-d approximation beats the truncated SVD: ||X - YT||_F^2 >= sum_{i>=d} s_i^2,
    ||X - YT||_2 >= s_d; and the max column residual bounds the Frobenius one."""
    X = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5, m=256, n=128)
    r = compress(X, 0.0, 40)
    s = np.linalg.svd(X, compute_uv=False)
    n = X.shape[1]
    for d in (4, 10, 20, 40):
        E = X - r["Y"][:, :d] @ r["T"][:d]
        fro = np.linalg.norm(E)
        assert fro >= np.sqrt((s[d:] ** 2).sum()) * (1 - 1e-10), f"d={d} below Eckart-Young (F)"
        assert np.linalg.norm(E, 2) >= s[d] * (1 - 1e-10), f"d={d} below Eckart-Young (2)"
        assert r["err"][d - 1] >= fro / np.sqrt(n) * (1 - 1e-12)


def pin_nu_matches_indicator(compress):
    """The orthogonalised norm of the next pivot (step 2.2) equals the previous indicator
    E_cur of step 2.3 (both are that column's residual), and E_cur is non-increasing."""
    X = _decay(180, 140, 7, rate=0.25, noise=1e-6)
    r = compress(X, 0.0, 36)
    e, nu = r["err"], r["nu"]
    scale = np.linalg.norm(X, axis=0).max()
    assert np.all(np.abs(nu[1:] - e[:-1]) <= 1e-11 * scale), "nu[k] != err[k-1]"
    assert np.all(np.diff(e) <= 1e-12 * scale), "E_cur increased"


def pin_termination(compress):
    """Step 2.4 stops on E_cur <= eps_R (inclusive), step 2.2 breaks on ||v|| < eps_R; the
    relative and Frobenius modes scale eps_R as documented."""
    norms = np.array([8.0, 4.0, 2.0, 1.0])
    X = gen.orthogonal_columns(6, norms, seed=9)
    assert compress(X, 4.0, 4)["d"] == 1          # E_1 = 4 <= 4
    assert compress(X, 3.99, 4)["d"] == 2         # E_1 = 4 > 3.99, E_2 = 2 <= 3.99
    assert compress(X, 0.5, 4, mode="maxcol_rel")["d"] == 1     # eps_R = 0.5 * 8 = 4
    assert compress(X, 9.0, 4)["d"] == 0          # ||x_0|| = 8 < 9: step 2.2 breaks at once
    # Frobenius: ||X||_F = sqrt(85); after 1 basis sqrt(21) = 4.58 <= 0.5 sqrt(85) = 4.61
    assert compress(X, 0.5, 4, mode="fro_rel")["d"] == 1
    assert compress(X, 0.45, 4, mode="fro_rel")["d"] == 2


def pin_zero_matrix(compress):
    """An all-zero X has nothing to compress: no basis is produced."""
    X = np.zeros((5, 4), order="F")
    assert compress(X, 0.0, 3)["d"] == 0


# ---------------------------------------------------------------------------------------------
# Diagonal A-norm (Section 3.2, "general diagonal matrix"): compress(..., weights=w) keeps the
# Euclidean Gram-Schmidt basis and T = Y' X and measures the error of steps 2.2-2.4 in
# ||v||_A = sqrt(sum_r w_r v_r^2).
# ---------------------------------------------------------------------------------------------
def _anorm(R, w):
    return np.sqrt((w[:, None] * R * R).sum(axis=0))


def pin_w_indicator_definition(compress):
    """With weights: err[k] = max_j ||X(:, j) - Y(:, 0:k) T(0:k, j)||_A from scratch, its argmax
    is the next pivot, Y'Y = I and T = Y' X (the basis stays Euclidean)."""
    X = _decay(150, 110, 21, rate=0.2, noise=1e-7)
    w = gen.row_weights(150, seed=1)
    r = compress(X, 0.0, 28, weights=w)
    d = r["d"]
    assert d == 28, f"expected 28 bases, got {d}"
    Y = r["Y"]
    assert np.abs(Y.T @ Y - np.eye(d)).max() <= 10 * d * EPS, "Y'Y != I"
    scale = np.linalg.norm(X, axis=0)
    assert (np.abs(r["T"] - Y.T @ X) / scale[None, :]).max() <= 1e-13, "T != Y'X"
    sa = _anorm(X, w).max()
    for k in range(d):
        cn = _anorm(X - Y[:, :k + 1] @ r["T"][:k + 1, :], w)
        assert abs(r["err"][k] - cn.max()) <= 1e-12 * sa, f"err[{k}] {r['err'][k]} vs {cn.max()}"
        srt = np.sort(cn)
        if k + 1 < d and srt[-1] - srt[-2] > 1e-9 * sa:
            assert r["pivots"][k + 1] == int(np.argmax(cn)), f"pivot {k + 1}"


def pin_w_bruteforce_tiny(compress):
    """Tiny inputs with weights: the next pivot maximises ||x_j - X(:, P) c||_A over j, c the
    Euclidean least-squares coefficients (T = Y' X), independent of Gram-Schmidt and the update."""
    rng = np.random.default_rng(25)
    checked = 0
    for trial in range(40):
        m = int(rng.integers(2, 9))
        n = int(rng.integers(2, 9))
        X = np.asfortranarray(rng.standard_normal((m, n)))
        w = np.exp(rng.uniform(np.log(0.05), np.log(20.0), m))
        start = int(rng.integers(0, n))
        r = compress(X, 0.0, min(m, n), start=start, weights=w)
        assert r["pivots"][0] == start
        sa = _anorm(X, w).max()
        for k in range(r["d"]):
            A = X[:, r["pivots"][:k + 1]]
            res = np.empty(n)
            for j in range(n):
                c, *_ = np.linalg.lstsq(A, X[:, j], rcond=None)
                res[j] = np.sqrt((w * (X[:, j] - A @ c) ** 2).sum())
            assert abs(r["err"][k] - res.max()) <= 1e-11 * sa, f"trial {trial} step {k}"
            srt = np.sort(res)
            if k + 1 < r["d"] and n > 1 and srt[-1] - srt[-2] > 1e-8 * sa:
                assert r["pivots"][k + 1] == int(np.argmax(res)), f"trial {trial} pivot {k + 1}"
                checked += 1
    assert checked > 20


def pin_w_closed_form_orthogonal(compress):
    """Columns norms[j] e_p(j): no column has a component along another, so each residual is the
    column itself and the pivots follow decreasing ||x_j||_A = norms[j] sqrt(w[p(j)]) (an order the
    weights make different from the Euclidean one); err[k] is the largest A-norm not yet chosen
    and nu[k] the chosen column's Euclidean norm."""
    norms = np.array([3.0, 7.0, 1.0, 5.0, 2.0, 6.0, 4.0])
    X = gen.orthogonal_columns(12, norms, seed=3)
    rows = np.argmax(np.abs(X), axis=0)
    w = np.full(12, 1.0)
    w[rows] = np.array([16.0, 0.25, 30.0, 1.0, 9.0, 0.5, 2.0])
    an = norms * np.sqrt(w[rows])
    assert len(set(np.round(an, 9))) == 7 and list(np.argsort(-an)) != list(np.argsort(-norms))
    start = 2
    r = compress(X, 0.0, 7, start=start, weights=w)
    order = [start] + [int(j) for j in np.argsort(-an) if j != start]
    assert list(r["pivots"]) == order, f"pivots {list(r['pivots'])} != {order}"
    for k in range(r["d"]):
        remaining = [an[j] for j in range(7) if j not in order[:k + 1]]
        expect = max(remaining) if remaining else 0.0
        assert abs(r["err"][k] - expect) <= 1e-14 * an.max(), f"err[{k}] {r['err'][k]} != {expect}"
        assert abs(r["nu"][k] - norms[order[k]]) <= 1e-14 * norms.max(), f"nu[{k}]"


def pin_w_termination(compress):
    """Steps 2.2 and 2.4 compare the A-norm with eps_R; the relative modes scale by the A-norms
    of X."""
    norms = np.array([8.0, 4.0, 2.0, 1.0])
    X = gen.orthogonal_columns(6, norms, seed=9)
    rows = np.argmax(np.abs(X), axis=0)
    w = np.full(6, 1.0)
    w[rows] = np.array([0.25, 6.25, 1.0, 9.0])   # A-norms 4, 10, 2, 3
    r = compress(X, 0.0, 4, start=1, weights=w)
    assert r["pivots"].tolist() == [1, 0, 3, 2]
    assert np.abs(r["err"] - np.array([4.0, 3.0, 2.0, 0.0])).max() <= 1e-14 * 10
    assert compress(X, 4.0, 4, start=1, weights=w)["d"] == 1     # E_1 = 4 <= 4
    assert compress(X, 3.99, 4, start=1, weights=w)["d"] == 2    # E_2 = 3 <= 3.99
    assert compress(X, 2.5, 4, start=1, weights=w)["d"] == 3     # E_3 = 2 <= 2.5
    # eps_R = 0.35 max_j ||x_j||_A = 3.5 (the Euclidean maximum would give 2.8 and d = 3)
    assert compress(X, 0.35, 4, start=1, mode="maxcol_rel", weights=w)["d"] == 2
    # step 2.2 on the start column: ||x_0||_A = 4 < 5 <= ||x_0|| = 8
    assert compress(X, 5.0, 4, start=0, weights=w)["d"] == 0
    # Frobenius in the A-norm: ||X||_F,A = sqrt(129) = 11.36; after one basis sqrt(29) = 5.39,
    # after two sqrt(13) = 3.61
    assert compress(X, 0.48, 4, start=1, mode="fro_rel", weights=w)["d"] == 1
    assert compress(X, 0.47, 4, start=1, mode="fro_rel", weights=w)["d"] == 2


def pin_w_scaling(compress):
    """A = alpha diag(w): the same bases and pivots, errors times sqrt(alpha); A = I (all weights
    one) gives the unweighted result."""
    X = _decay(120, 90, 23, rate=0.25, noise=1e-7)
    w = gen.row_weights(120, seed=2)
    r1 = compress(X, 0.0, 20, weights=w)
    r4 = compress(X, 0.0, 20, weights=4.0 * w)
    assert list(r1["pivots"]) == list(r4["pivots"])
    assert np.abs(r1["Y"] - r4["Y"]).max() <= 1e-13
    sa = r1["err"].max()
    assert np.abs(r4["err"] - 2.0 * r1["err"]).max() <= 1e-12 * sa
    ru = compress(X, 0.0, 20)
    ri = compress(X, 0.0, 20, weights=np.ones(120))
    assert list(ru["pivots"]) == list(ri["pivots"])
    assert np.abs(ru["err"] - ri["err"]).max() <= 1e-13 * ru["err"].max()


W_PINS = [pin_w_indicator_definition, pin_w_bruteforce_tiny, pin_w_closed_form_orthogonal, pin_w_termination,
          pin_w_scaling]


FAST_PINS = [pin_orthonormal, pin_indicator_definition, pin_T_is_projection, pin_qr_equivalence,
             pin_bruteforce_tiny, pin_closed_form_orthogonal, pin_ties_lowest_index, pin_start_column,
             pin_exact_rank, pin_eckart_young, pin_nu_matches_indicator, pin_termination,
             pin_zero_matrix]
