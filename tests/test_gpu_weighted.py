"""The diagonal A-norm form (Section 3.2, A = diag(w); rbd_compress_weighted through the C ABI)
against the FP64 oracle on the same stored values.

Bar (float-float dot products, as the plain form): identical d and pivots; Y, T and nu within
1e-10 normwise (Y columns are unit vectors, T(k, j) relative to ||x_j||), err within 1e-10 of
max_j ||x_j||_A.  The cases keep nu / ||x_i|| above ~1e-3 (the two sides' rounding is amplified by
||x_i|| / nu at each step; see test_gpu_precision.py).  Also: the weighted pins on the CUDA path,
all-ones weights give the unweighted result, invalid weights fail with RBD_EINVAL, BF16 storage
against the exact properties, and the 8192 x 8192 image workload on its first steps and on
sampled columns.
"""
import numpy as np
import pytest
import torch

import gen
import pins
from gpu_util import gpu_compress, to_device, to_numpy

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def _wdev(w):
    return torch.as_tensor(np.ascontiguousarray(w, dtype=np.float64), device="cuda:0")


def _run(rbd, X, w, tol, d_max, mode="maxcol_abs", start=0):
    r = rbd.compress(X, tol, d_max, start=start, tol_mode=mode, weights=_wdev(w))
    return {"Y": to_numpy(r.Y), "T": to_numpy(r.T), "pivots": r.pivots.cpu().numpy(), "err": r.err.cpu().numpy(),
            "nu": r.nu.cpu().numpy(), "d": r.d, "next": r.next_pivot, "stop": r.stop_reason, "res": r}


def _parity(Xs, w, ref, got, what, kmax=None):
    scale = np.linalg.norm(Xs, axis=0)
    ascale = np.sqrt((w[:, None] * Xs * Xs).sum(axis=0)).max()
    if kmax is None:
        assert got["d"] == ref["d"], f"{what}: d {got['d']} != {ref['d']}"
        kmax = ref["d"]
    assert np.array_equal(got["pivots"][:kmax], ref["pivots"][:kmax]), f"{what}: pivots differ"
    if kmax == 0:
        return
    dy = np.linalg.norm(got["Y"][:, :kmax] - ref["Y"][:, :kmax], axis=0).max()
    assert dy <= TOL, f"{what}: Y {dy:.3e}"
    dt = (np.abs(got["T"][:kmax] - ref["T"][:kmax]) / np.maximum(scale, 1e-300)[None, :]).max()
    assert dt <= TOL, f"{what}: T {dt:.3e}"
    de = np.abs(got["err"][:kmax] - ref["err"][:kmax]).max()
    assert de <= TOL * ascale, f"{what}: err {de:.3e}"
    dn = np.abs(got["nu"][:kmax] - ref["nu"][:kmax]).max()
    assert dn <= TOL * scale.max(), f"{what}: nu {dn:.3e}"


CASES = [
    ("decay 1024x512 abs", lambda: gen.decay_matrix_c1(seed=0, noise_sigma=1e-5), 1e-6, 64, "maxcol_abs", 0),
    ("ragged 777x333 rel", lambda: gen.decay_matrix_c1(seed=4, noise_sigma=1e-4, m=777, n=333), 1e-4, 40,
     "maxcol_rel", 17),
    ("lowrank 2500x640 fro", lambda: gen.lowrank_haar(2500, 640, 2.0 ** (-np.arange(120) / 6), seed=5), 1e-5, 64,
     "fro_rel", 3),
    ("ragged 1000x77 full", lambda: gen.decay_matrix_c1(seed=6, noise_sigma=1e-4, m=1000, n=77), 0.0, 77,
     "maxcol_abs", 76),
    ("tall 20000x300", lambda: gen.lowrank_haar(20000, 300, 2.0 ** (-np.arange(300) / 8), seed=8, noise_sigma=1e-9),
     1e-6, 80, "maxcol_rel", 0),
    # more than 256 rows per CTA (two rows per consumer thread in the Gram-Schmidt phases)
    ("tall 50000x120", lambda: gen.lowrank_haar(50000, 120, 2.0 ** (-np.arange(120) / 6), seed=9, noise_sigma=1e-9),
     1e-6, 40, "fro_rel", 5),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_weighted_matches_oracle(rbd, oracle_mod, case, dtype):
    name, build, tol, d_max, mode, start = case
    Xn = np.asfortranarray(build())
    X = to_device(Xn, dtype)
    Xs = to_numpy(X)
    w = gen.row_weights(Xn.shape[0], seed=31)
    ref = oracle_mod.compress(Xs, tol, d_max, start, mode, weights=w)
    got = _run(rbd, X, w, tol, d_max, mode, start)
    _parity(Xs, w, ref, got, name)
    assert got["next"] == ref["next_pivot"] or got["d"] == d_max


@pytest.mark.parametrize("pin", pins.W_PINS, ids=lambda p: p.__name__)
def test_weighted_pins_on_cuda_path(rbd, pin):
    pin(gpu_compress)


def test_unit_weights_equal_unweighted_path(rbd, monkeypatch):
    Xn = gen.decay_matrix_c1(seed=2, noise_sigma=1e-5, m=1500, n=700)
    X = to_device(Xn)
    w1 = torch.ones(1500, dtype=torch.float64, device="cuda")
    b = rbd.compress(X, 1e-6, 80, tol_mode="maxcol_abs", weights=w1)
    # the four-barrier kernel of the unweighted form takes the same operations for the basis and
    # T as the A-norm form; the indicator update differs by rounding only
    monkeypatch.setenv("RBD_LOOP_CLASSIC", "1")
    a = rbd.compress(X, 1e-6, 80, tol_mode="maxcol_abs")
    monkeypatch.delenv("RBD_LOOP_CLASSIC")
    assert a.d == b.d and torch.equal(a.pivots, b.pivots)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T) and torch.equal(a.nu, b.nu)
    assert torch.allclose(a.err, b.err, rtol=1e-14, atol=0.0)
    # the default (two-barrier) unweighted kernel: the same pivots, Y and T at the parity bar
    c = rbd.compress(X, 1e-6, 80, tol_mode="maxcol_abs")
    assert c.d == b.d and torch.equal(c.pivots, b.pivots)
    scale = np.linalg.norm(Xn, axis=0)
    assert np.linalg.norm(to_numpy(c.Y) - to_numpy(b.Y), axis=0).max() <= 1e-10
    assert (np.abs(to_numpy(c.T) - to_numpy(b.T)) / scale[None, :]).max() <= 1e-10
    assert (c.err - b.err).abs().max().item() <= 1e-10 * scale.max()


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_invalid_weights_rejected(rbd, bad):
    X = to_device(gen.decay_matrix_c1(seed=0, m=300, n=100))
    w = np.ones(300)
    w[137] = bad
    with pytest.raises(rbd.RbdError) as ei:
        rbd.compress(X, 0.0, 10, weights=_wdev(w))
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        rbd.compress(X, 0.0, 10, weights=torch.ones(299, dtype=torch.float64, device="cuda"))


def test_weighted_bf16_storage_properties(rbd):
    """BF16 storage, FP32-accumulated dot products: Y'Y = I, T = Y'X within the FP32 bound, and
    the certified err[k] equal to the A-norm residual of pivot k+1 recomputed from scratch."""
    Xn = gen.parametric_snapshots(4096, 1024, seed=2)
    X = to_device(Xn, torch.bfloat16)
    Xs = to_numpy(X)
    w = gen.row_weights(4096, seed=5)
    r = _run(rbd, X, w, 1e-3, 24, "maxcol_rel")
    d = r["d"]
    assert d >= 5
    Y = r["Y"]
    assert np.abs(Y.T @ Y - np.eye(d)).max() <= 1e-12
    scale = np.linalg.norm(Xs, axis=0)
    # per-unit FP32 partial sums plus the pivot vector's leading FP32 part (as the plain BF16 form)
    assert (np.abs(r["T"] - Y.T @ Xs) / scale[None, :]).max() <= 2.0 ** -20 + 2.0 ** -24
    for k in range(d - 1):
        j = r["pivots"][k + 1]
        res = Xs[:, j] - Y[:, :k + 1] @ (Y[:, :k + 1].T @ Xs[:, j])
        ra = np.sqrt((w * res * res).sum())
        assert abs(r["err"][k] - ra) <= 1e-9 * np.sqrt((w[:, None] * Xs * Xs).sum(axis=0)).max(), k


def test_image_workload_weighted(rbd, oracle_mod):
    """The 8192 x 8192 image-like field with row weights: the first 6 steps against the oracle,
    then d_max = 512 on the CUDA path with sampled columns' A-norm residuals under err."""
    q = gen.image_like_u8(8192, seed=1)
    Xn = np.asfortranarray(q.astype(np.float64) / 255.0)
    X = to_device(Xn)
    w = gen.row_weights(8192, seed=7)
    ref = oracle_mod.compress(Xn, 1e-3, 6, 0, "fro_rel", weights=w)
    got = _run(rbd, X, w, 1e-3, 6, "fro_rel")
    _parity(Xn, w, ref, got, "image 8192 first steps", kmax=6)
    full = _run(rbd, X, w, 1e-3, 512, "fro_rel")
    d = full["d"]
    assert d >= 100
    e = full["err"]
    rng = np.random.default_rng(0)
    cols = rng.choice(8192, 64, replace=False)
    Y = full["Y"]
    Tc = full["T"][:, cols]
    res = Xn[:, cols] - Y @ Tc
    ra = np.sqrt((w[:, None] * res * res).sum(axis=0))
    ascale = np.sqrt((w[:, None] * Xn * Xn).sum(axis=0)).max()
    assert (ra <= e[d - 1] + 1e-9 * ascale).all()
    # T(:, j) = Y' x_j on the sampled columns
    assert np.abs(Tc - Y.T @ Xn[:, cols]).max() <= 1e-10 * np.linalg.norm(Xn[:, cols], axis=0).max()
