"""Precision forms: X stored in FP32 or BF16 (the CUDA path through the C ABI, against the FP64
CPU oracle run on the same stored values).

* FP32 storage keeps float-float accumulation of the dot products, so it meets the plain-form
  parity bar on the stored values: identical pivots; Y, T, err, nu within 1e-10 (normwise).
  The cases keep nu / ||x_i|| above about 1e-4: a basis vector xi = v / nu carries the rounding of
  v (2^-47 relative in float-float, 2^-53 in the oracle) amplified by ||x_i|| / nu, and past an
  amplification of ~1e3 the two sides' rounding alone approaches the 1e-10 bar.
* BF16 storage accumulates the dot products in FP32 (the precision form).  Its pivots are not
  pinned to the oracle's (the running indicator carries the FP32 accumulation error); it is
  checked against what still holds exactly: Y'Y = I, T = Y'X within the FP32 accumulation bound,
  the certified indicator err[k] equal to the true residual of the next pivot, that pivot's
  residual within the indicator's error of the column maximum, and a reconstruction error within
  a few percent of the oracle's at the same d.
* The 65536 x 16384 parametric snapshot workload in all three storage types: reconstruction
  error against the FP64 matrix on sampled columns.
"""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device, to_numpy

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def _stored(Xn, dtype):
    """Device tensor in the storage type and the FP64 values it holds (what the oracle sees)."""
    X = to_device(Xn, dtype)
    return X, to_numpy(X)


def _run(rbd, X, tol, d_max, mode="maxcol_abs", start=0, accumulate="exact"):
    r = rbd.compress(X, tol, d_max, start=start, tol_mode=mode, accumulate=accumulate)
    return {"Y": to_numpy(r.Y), "T": to_numpy(r.T), "pivots": r.pivots.cpu().numpy(),
            "err": r.err.cpu().numpy(), "nu": r.nu.cpu().numpy(), "d": r.d, "next": r.next_pivot,
            "stop": r.stop_reason}


def _parity(Xs, ref, got, what):
    scale = np.linalg.norm(Xs, axis=0)
    assert got["d"] == ref["d"], f"{what}: d {got['d']} != {ref['d']}"
    assert np.array_equal(got["pivots"], ref["pivots"]), f"{what}: pivots differ"
    if ref["d"] == 0:
        return
    assert np.linalg.norm(got["Y"] - ref["Y"], axis=0).max() <= TOL, what
    assert (np.abs(got["T"] - ref["T"]) / np.maximum(scale, 1e-300)[None, :]).max() <= TOL, what
    assert np.abs(got["err"] - ref["err"]).max() <= TOL * scale.max(), what
    assert np.abs(got["nu"] - ref["nu"]).max() <= TOL * scale.max(), what


# ---------------------------------------------------------------- FP32 storage: exact parity
FP32_CASES = [
    ("decay 1024x512", lambda: gen.decay_matrix_c1(seed=0, noise_sigma=1e-5), 1e-6, 64, "maxcol_abs"),
    ("parametric 4096x1024", lambda: gen.parametric_snapshots(4096, 1024, seed=2), 1e-5, 48, "maxcol_rel"),
    ("lowrank 2500x640 fro", lambda: gen.lowrank_haar(2500, 640, 2.0 ** (-np.arange(120) / 6), seed=5), 1e-5, 64,
     "fro_rel"),
    ("ragged 777x333", lambda: gen.decay_matrix_c1(seed=4, noise_sigma=1e-4, m=777, n=333), 1e-5, 40, "maxcol_rel"),
    ("ragged 1000x77", lambda: gen.decay_matrix_c1(seed=6, noise_sigma=1e-4, m=1000, n=77), 0.0, 77, "maxcol_abs"),
]


@pytest.mark.parametrize("case", FP32_CASES, ids=[c[0] for c in FP32_CASES])
def test_fp32_storage_matches_oracle(rbd, oracle_mod, case):
    name, build, tol, d_max, mode = case
    X, Xs = _stored(np.asfortranarray(build()), torch.float32)
    ref = oracle_mod.compress(Xs, tol, d_max, 0, mode)
    got = _run(rbd, X, tol, d_max, mode)
    _parity(Xs, ref, got, f"FP32 {name}")


# ---------------------------------------------------------------- BF16 storage: invariants
def _bf16_checks(Xs, got, ref, t_bound=2e-6, what=""):
    m, n = Xs.shape
    d = got["d"]
    assert d >= 2, what
    Y, T = got["Y"], got["T"]
    scale = np.linalg.norm(Xs, axis=0)
    # Y'Y = I: the orthogonalisation runs in FP64-grade arithmetic whatever the storage type
    assert np.abs(Y.T @ Y - np.eye(d)).max() <= 1e-12, what
    # T = Y'X up to the FP32 accumulation of the pass: |dT(k, j)| <= 2^-20 ||x_j|| (per-unit FP32
    # partial sums of 16 products) + 2^-24 ||x_j|| (the pivot vector's leading FP32 part)
    dT = np.abs(T - Y.T @ Xs) / np.maximum(scale, 1e-300)[None, :]
    assert dT.max() <= t_bound, f"{what}: |T - Y'X| / |x_j| = {dT.max():.2e}"
    # err[k] certifies E_cur: the true residual of the next pivot against Y(:, 0:k+1)
    nxt = list(got["pivots"][1:]) + [got["next"]]
    for k in range(d):
        i = nxt[k]
        Yk = Y[:, :k + 1]
        r = np.linalg.norm(Xs[:, i] - Yk @ (Yk.T @ Xs[:, i]))
        assert abs(got["err"][k] - r) <= 1e-10 * scale.max(), f"{what}: err[{k}]"
    # the pivot is the column maximum up to the indicator's accumulated error
    for k in range(min(d - 1, 16)):
        Yk = Y[:, :k + 1]
        R2 = np.sum((Xs - Yk @ (Yk.T @ Xs)) ** 2, axis=0)
        assert R2[nxt[k]] >= R2.max() - 1e-4 * scale.max() ** 2, f"{what}: pivot {k + 1}"
    # compression quality at the same d as the oracle on the same stored values
    if ref is not None and ref["d"] == d:
        e_got = np.linalg.norm(Xs - Y @ T)
        e_ref = np.linalg.norm(Xs - ref["Y"] @ ref["T"])
        assert e_got <= 1.05 * e_ref + 1e-12 * np.linalg.norm(Xs), f"{what}: {e_got:.3e} vs {e_ref:.3e}"


BF16_CASES = [
    ("parametric 4096x1024", lambda: gen.parametric_snapshots(4096, 1024, seed=2), 1e-3, 24, "maxcol_rel"),
    ("decay 2048x600", lambda: gen.lowrank_haar(2048, 600, 2.0 ** (-np.arange(200) / 8), seed=8), 3e-2, 48,
     "maxcol_rel"),
    ("ragged 1000x333 fro", lambda: gen.decay_matrix_c1(seed=9, noise_sigma=1e-4, m=1000, n=333), 1e-2, 40,
     "fro_rel"),
]


@pytest.mark.parametrize("case", BF16_CASES, ids=[c[0] for c in BF16_CASES])
def test_bf16_storage_invariants(rbd, oracle_mod, case):
    name, build, tol, d_max, mode = case
    X, Xs = _stored(np.asfortranarray(build()), torch.bfloat16)
    got = _run(rbd, X, tol, d_max, mode)
    ref = oracle_mod.compress(Xs, tol, d_max, 0, mode)
    _bf16_checks(Xs, got, ref, what=f"BF16 {name}")


# ------------------------------------------- FP32 storage, FP32 accumulation (RBD_F32_ACC32)
ACC32_CASES = [
    ("parametric 4096x1024", lambda: gen.parametric_snapshots(4096, 1024, seed=2), 1e-5, 48, "maxcol_rel"),
    ("decay 2048x600", lambda: gen.lowrank_haar(2048, 600, 2.0 ** (-np.arange(200) / 8), seed=8), 1e-4, 64,
     "maxcol_rel"),
    ("ragged 1000x333 fro", lambda: gen.decay_matrix_c1(seed=9, noise_sigma=1e-4, m=1000, n=333), 1e-4, 40,
     "fro_rel"),
]


@pytest.mark.parametrize("case", ACC32_CASES, ids=[c[0] for c in ACC32_CASES])
def test_fp32_accumulation_invariants(rbd, oracle_mod, case):
    """The precision form with FP32 accumulation: per-tile FP32 sums of 8 products per lane, so T
    carries ~2^-20 relative error and pivots are not pinned to the oracle's; the invariants that
    still hold exactly are checked as for BF16 storage, on the same stored values."""
    name, build, tol, d_max, mode = case
    X, Xs = _stored(np.asfortranarray(build()), torch.float32)
    got = _run(rbd, X, tol, d_max, mode, accumulate="fp32")
    ref = oracle_mod.compress(Xs, tol, d_max, 0, mode)
    _bf16_checks(Xs, got, ref, what=f"FP32-acc {name}")


def test_fp32_accumulation_against_exact_form(rbd):
    """While the columns' residuals stay above the running indicator's FP32 floor (T is accurate to
    ~1e-8 ||x_j||, so e_j = ||x_j||^2 - sum T^2 carries ~2e-8 ||x_j||^2; here d <= 8, relative
    residual ~6e-5), FP32 accumulation picks the same pivots as the FP64-grade form and reconstructs
    X as well at equal d.  Past that floor its pivots follow the indicator's rounding (the certified
    E_cur stays exact, the basis converges more slowly)."""
    X, Xs = _stored(np.asfortranarray(gen.parametric_snapshots(4096, 1024, seed=2)), torch.float32)
    for d in (4, 6, 8):
        a = _run(rbd, X, 0.0, d)
        b = _run(rbd, X, 0.0, d, accumulate="fp32")
        assert a["d"] == b["d"] == d and np.array_equal(a["pivots"], b["pivots"])
        ea = np.linalg.norm(Xs - a["Y"] @ a["T"])
        eb = np.linalg.norm(Xs - b["Y"] @ b["T"])
        assert abs(eb - ea) <= 1e-3 * ea, (d, ea, eb)
        dT = np.abs(b["T"] - b["Y"].T @ Xs) / np.linalg.norm(Xs, axis=0)[None, :]
        assert dT.max() <= 5e-8, dT.max()


def test_fp32_accumulation_rejected_where_unsupported(rbd):
    X, _ = _stored(np.asfortranarray(gen.parametric_snapshots(512, 256, seed=2)), torch.float32)
    with pytest.raises(rbd.RbdError):
        rbd.compress(X, 0.0, 8, weights=torch.ones(512, dtype=torch.float64, device="cuda"), accumulate="fp32")
    with pytest.raises(ValueError):
        rbd.compress(X.double(), 0.0, 8, accumulate="fp32")


def test_bf16_deterministic(rbd):
    X, _ = _stored(np.asfortranarray(gen.parametric_snapshots(4096, 1024, seed=2)), torch.bfloat16)
    a = _run(rbd, X, 1e-3, 24, "maxcol_rel")
    b = _run(rbd, X, 1e-3, 24, "maxcol_rel")
    assert np.array_equal(a["pivots"], b["pivots"])
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["Y"], b["Y"])


# ---------------------------------------------------------------- full-size precision workload
def test_parametric_65536x16384_three_storage_types(rbd):
    """X_ij = 1 / sqrt((s_i - mu1_j)^2 + mu2_j^2), 65536 x 16384, d_max 256, tol 0 (the loop runs
    to the numerical-rank floor, or to d_max where rounding keeps the residual above it).
    Relative reconstruction error against the FP64 matrix on 64 sampled columns."""
    m, n, d_max = 65536, 16384, 256
    X64 = gen.parametric_snapshots_torch(m, n, device="cuda")
    rng = np.random.default_rng(0)
    cols = torch.from_numpy(np.sort(rng.choice(n, 64, replace=False))).cuda()
    Xs = X64[:, cols]
    bounds = {torch.float64: 1e-8, torch.float32: 1e-6, torch.bfloat16: 5e-3}
    for dt, bound in bounds.items():
        X = X64 if dt == torch.float64 else X64.t().contiguous().to(dt).t()
        r = rbd.compress(X, 0.0, d_max)
        assert r.d >= 10
        Yt = r.Y
        rel = ((Xs - Yt @ r.T[:, cols]).norm() / Xs.norm()).item()
        assert rel <= bound, f"{dt}: relative error {rel:.3e} > {bound:.0e}"
        orth = (Yt.t() @ Yt - torch.eye(r.d, device="cuda", dtype=torch.float64)).abs().max().item()
        assert orth <= 1e-12, f"{dt}: Y'Y - I = {orth:.2e}"
        del X, r
        torch.cuda.empty_cache()
