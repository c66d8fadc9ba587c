"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Bar (plain FP64 form): identical pivot sequences; ||Y(:,k) - Y_ref(:,k)|| <= 1e-10 (unit
columns); |T(k,j) - T_ref(k,j)| <= 1e-10 ||x_j||; |err_k - err_ref_k| <= 1e-10 max_j ||x_j||.
The pins of tests/pins.py are also applied to the CUDA path.
"""
import numpy as np
import pytest
import torch

import gen
import pins
from gpu_util import gpu_compress, to_device, to_numpy

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as rbd
    rbd.load()


def assert_parity(X, ref, got, tol=TOL, what=""):
    scale = np.linalg.norm(X, axis=0)
    assert got["d"] == ref["d"], f"{what}: d {got['d']} != {ref['d']}"
    d = ref["d"]
    assert np.array_equal(got["pivots"], ref["pivots"]), f"{what}: pivots differ"
    if d == 0:
        return
    dY = np.linalg.norm(got["Y"] - ref["Y"], axis=0).max()
    dT = (np.abs(got["T"] - ref["T"]) / np.maximum(scale, 1e-300)[None, :]).max()
    dE = np.abs(got["err"] - ref["err"]).max() / scale.max()
    dN = np.abs(got["nu"] - ref["nu"]).max() / scale.max()
    assert dY <= tol, f"{what}: |dY| {dY:.3e}"
    assert dT <= tol, f"{what}: |dT|/|x_j| {dT:.3e}"
    assert dE <= tol, f"{what}: |derr| {dE:.3e}"
    assert dN <= tol, f"{what}: |dnu| {dN:.3e}"


def test_config_small_decay_1024x512(oracle_mod):
    """The small FP64 workload: 1024 x 512, s_i = 2^(-i/4), noise sd 1e-5, d_max 64, tol 1e-6."""
    X = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)
    ref = oracle_mod.compress(X, 1e-6, 64)
    got = gpu_compress(X, 1e-6, 64)
    assert_parity(X, ref, got, what="1024x512")
    assert got["result"].stop_reason == "d_max"


def test_config_small_decay_tiny_noise(oracle_mod):
    """Same workload with noise sd 1e-10 (the other reading of N(0, 1e-10))."""
    X = gen.decay_matrix_c1(seed=0, noise_sigma=1e-10)
    ref = oracle_mod.compress(X, 1e-6, 64)
    got = gpu_compress(X, 1e-6, 64)
    assert_parity(X, ref, got, what="1024x512 sd 1e-10")


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 3), (5, 5), (33, 17), (127, 64), (128, 128), (129, 130), (300, 41),
          (513, 200), (1000, 333), (3000, 1001), (257, 2049), (20000, 150)]


@pytest.mark.parametrize("m,n", SHAPES, ids=lambda v: str(v))
def test_ragged_shapes(oracle_mod, m, n):
    """Shapes spanning several row tiles / column groups with ragged tails."""
    r = min(m, n)
    X = gen.lowrank_haar(m, n, 2.0 ** (-0.3 * np.arange(r)), seed=m * 7 + n, noise_sigma=1e-9)
    d_max = min(r, 24)
    start = (m + n) % n
    ref = oracle_mod.compress(X, 0.0, d_max, start=start)
    got = gpu_compress(X, 0.0, d_max, start=start)
    assert_parity(X, ref, got, what=f"{m}x{n}")


@pytest.mark.parametrize("mode,tol", [("maxcol_abs", 1e-3), ("maxcol_rel", 1e-4), ("fro_rel", 1e-3),
                                      ("fro_rel", 1e-2)])
def test_tolerance_modes(oracle_mod, mode, tol):
    X = gen.lowrank_haar(400, 300, 2.0 ** (-0.25 * np.arange(300)), seed=3, noise_sigma=1e-8)
    ref = oracle_mod.compress(X, tol, 200, mode=mode)
    got = gpu_compress(X, tol, 200, mode=mode)
    assert ref["d"] < 200
    assert_parity(X, ref, got, what=mode)
    assert got["result"].stop_reason in ("tol", "break")


def test_padded_leading_dimension(oracle_mod):
    """X with ldx > m (a column-major view into a taller buffer)."""
    X = gen.decay_matrix_c1(seed=4, m=200, n=150)
    big = np.zeros((256, 150), order="F")
    big[:200] = X
    Xb = to_device(big)[:200, :]
    import paper_1503_05947_gb300 as rbd
    r = rbd.compress(Xb, 0.0, 30)
    ref = oracle_mod.compress(X, 0.0, 30)
    got = {"Y": to_numpy(r.Y), "T": to_numpy(r.T), "pivots": r.pivots.cpu().numpy(), "err": r.err.cpu().numpy(),
           "nu": r.nu.cpu().numpy(), "d": r.d}
    assert_parity(X, ref, got, what="ldx 256")


def test_deterministic_and_host_entry_point(oracle_mod):
    """Two runs are bitwise identical; rbd_compress_host gives the same bits as rbd_compress."""
    import paper_1503_05947_gb300 as rbd
    X = gen.decay_matrix_c1(seed=5, m=700, n=400)
    a = gpu_compress(X, 0.0, 40)
    b = gpu_compress(X, 0.0, 40)
    for key in ("Y", "T", "pivots", "err", "nu"):
        assert np.array_equal(a[key], b[key]), key
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory().t()
    h = rbd.compress_host(Xh, 0.0, 40)
    assert np.array_equal(h.pivots.numpy(), a["pivots"])
    assert np.array_equal(np.asfortranarray(h.Y.numpy()), a["Y"])
    assert np.array_equal(np.asfortranarray(h.T.numpy()), a["T"])
    assert np.array_equal(h.err.numpy(), a["err"])


def test_project_matches_oracle(oracle_mod):
    import paper_1503_05947_gb300 as rbd
    X = gen.decay_matrix_c1(seed=6, m=1000, n=300)
    r = rbd.compress(to_device(X), 0.0, 50)
    ref = oracle_mod.compress(X, 0.0, 50)
    for k in (1, 7, 64, 100):
        V = gen.out_of_sample(1000, k, seed=k)
        C = to_numpy(rbd.project(r.Y, to_device(V)))
        Cref = oracle_mod.project(to_numpy(r.Y), V)
        assert np.abs(C - Cref).max() <= 1e-12 * np.linalg.norm(V, axis=0).max()
    # in-sample columns map to T (the projection of Section 3.1 on X itself)
    Cx = to_numpy(rbd.project(r.Y, to_device(X)))
    assert np.abs(Cx - ref["T"]).max() <= TOL * np.linalg.norm(X, axis=0).max()
    # FP32 vectors: the same map on the FP32 values
    V32 = gen.out_of_sample(1000, 9, seed=9).astype(np.float32)
    C32 = to_numpy(rbd.project(r.Y, to_device(V32, torch.float32)))
    Cref32 = oracle_mod.project(to_numpy(r.Y), V32.astype(np.float64))
    assert np.abs(C32 - Cref32).max() <= 1e-12


def test_nonfinite_and_range_errors():
    import paper_1503_05947_gb300 as rbd
    X = np.asfortranarray(np.random.default_rng(0).standard_normal((64, 32)))
    X[3, 5] = np.nan
    with pytest.raises(rbd.RbdError) as ei:
        rbd.compress(to_device(X), 0.0, 8)
    assert ei.value.status == 4
    X[3, 5] = 2.0 ** 130
    with pytest.raises(rbd.RbdError) as ei:
        rbd.compress(to_device(X), 0.0, 8)
    assert ei.value.status == 6
    # the library stays usable afterwards
    X[3, 5] = 1.0
    assert rbd.compress(to_device(X), 0.0, 8).d == 8


@pytest.mark.parametrize("pin", pins.FAST_PINS, ids=lambda p: p.__name__)
def test_pins_on_cuda_path(pin):
    pin(gpu_compress)


def test_paper_rank_functions_on_cuda_path():
    pins.pin_paper_rank_functions(gpu_compress)


def test_paper_approx_example_on_cuda_path():
    pins.pin_paper_approx_example(gpu_compress)


def test_workspace_supplied_by_caller(oracle_mod):
    import paper_1503_05947_gb300 as rbd
    X = gen.decay_matrix_c1(seed=8, m=512, n=256)
    nbytes = rbd.workspace_bytes(512, 256, 32)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda:0")
    r = rbd.compress(to_device(X), 0.0, 32, workspace=ws)
    ref = oracle_mod.compress(X, 0.0, 32)
    assert np.array_equal(r.pivots.cpu().numpy(), ref["pivots"])
    small = torch.empty(nbytes // 2, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(rbd.RbdError) as ei:
        rbd.compress(to_device(X), 0.0, 32, workspace=small)
    assert ei.value.status == 2


@pytest.mark.parametrize("xt", [torch.float64, torch.float32], ids=["fp64", "fp32"])
def test_no_tolerance_mode_runs_to_d_max(oracle_mod, xt):
    """tol_mode "none" (a measurement mode): exactly d_max bases past the numerical rank of X, with
    finite outputs; up to that rank, the oracle's bases (a run that breaks there)."""
    import paper_1503_05947_gb300 as rbd
    Xt = to_device(gen.lowrank_haar(3000, 900, 2.0 ** (-0.5 * np.arange(20)), seed=21), xt)
    Xs = to_numpy(Xt)
    b = rbd.compress(Xt, 0.0, 40, tol_mode="none")
    assert b.d == 40 and b.stop_reason == "d_max"
    assert torch.isfinite(b.Y).all() and torch.isfinite(b.T).all() and torch.isfinite(b.err).all()
    ref = oracle_mod.compress(Xs, 0.0, 40)
    # the bases before the orthogonalised pivots reach rounding level (nu >= 1e-4 ||x_i||; FP32
    # storage rounding keeps the oracle going to d_max, past the 20 significant directions)
    cond = ref["nu"] / np.linalg.norm(Xs[:, ref["pivots"]], axis=0)
    k = int(np.argmax(cond < 1e-4)) if (cond < 1e-4).any() else ref["d"]
    assert 18 <= k <= 24
    # (err[k - 1] is the residual of the next pivot, already at rounding level: not compared)
    cut = {key: (v[:, :k] if key == "Y" else v[:k]) for key, v in ref.items() if key in ("Y", "T", "pivots", "nu")}
    cut["err"] = ref["err"][:k - 1]
    cut["d"] = k
    got = {"Y": to_numpy(b.Y[:, :k]), "T": to_numpy(b.T[:k]), "pivots": b.pivots[:k].cpu().numpy(),
           "err": b.err[:k - 1].cpu().numpy(), "nu": b.nu[:k].cpu().numpy(), "d": k}
    assert_parity(Xs, cut, got, what="no-tolerance run up to the rank")
