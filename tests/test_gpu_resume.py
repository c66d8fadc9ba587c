"""Resuming a compression to a larger d_max (rbd_compress_resume through the C ABI): the greedy
loop continued from its outputs after d0 bases gives the same bits as one call with the larger
d_max, on the persistent-kernel path and on the stepwise path, for FP64 and FP32 storage and the
three tolerance modes; a run stopped by its tolerance stays stopped."""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def _same(a, b):
    assert a.d == b.d and a.stop_reason == b.stop_reason and a.next_pivot == b.next_pivot
    assert torch.equal(a.pivots, b.pivots)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T)
    assert torch.equal(a.err, b.err) and torch.equal(a.nu, b.nu)
    assert a.fro_last == b.fro_last


CASES = [
    ("decay 1024x512 fp64", lambda: gen.decay_matrix_c1(seed=0, noise_sigma=1e-5), torch.float64, 1e-6, "maxcol_abs",
     20, 64),
    ("lowrank 1500x700 fro fp64", lambda: gen.lowrank_haar(1500, 700, np.logspace(0, -8, 90), seed=7),
     torch.float64, 1e-9, "fro_rel", 33, 120),
    ("decay 777x333 fp32", lambda: gen.decay_matrix_c1(seed=3, noise_sigma=1e-5, m=777, n=333), torch.float32,
     1e-5, "maxcol_rel", 9, 40),
]


@pytest.mark.parametrize("stepwise", [False, True], ids=["persistent", "stepwise"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_resume_equals_one_call(rbd, monkeypatch, case, stepwise):
    if stepwise:
        monkeypatch.setenv("RBD_STEPWISE", "1")
    name, build, dtype, tol, mode, d0, d_max = case
    X = to_device(np.asfortranarray(build()), dtype)
    full = rbd.compress(X, tol, d_max, tol_mode=mode)
    first = rbd.compress(X, tol, d0, tol_mode=mode)
    assert first.d == d0 and first.stop_reason == "d_max"
    cont = rbd.compress_resume(X, first, tol, d_max, tol_mode=mode)
    _same(cont, full)
    # resuming in two hops
    mid = rbd.compress_resume(X, first, tol, (d0 + d_max) // 2, tol_mode=mode)
    _same(rbd.compress_resume(X, mid, tol, d_max, tol_mode=mode), full)


def test_resume_after_tolerance_stop(rbd):
    X = to_device(np.asfortranarray(gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)))
    done = rbd.compress(X, 1e-3, 64)
    assert done.stop_reason == "tol" and done.d < 64
    again = rbd.compress_resume(X, done, 1e-3, 64)
    assert again.d == done.d and again.stop_reason == "tol"
    finer = rbd.compress_resume(X, done, 1e-4, 64)
    ref = rbd.compress(X, 1e-4, 64)
    # the finer tolerance continues where the coarse one stopped: the same pivots as a fresh run
    assert finer.d == ref.d and torch.equal(finer.pivots, ref.pivots)
    assert (finer.Y - ref.Y).abs().max().item() == 0.0
