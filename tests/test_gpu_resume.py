"""Resuming a compression to a larger d_max (rbd_compress_resume through the C ABI).

The greedy loop of Algorithm 1 (Section 3.1) carries its state from one basis to the next; a run
continued from its outputs after d0 bases must therefore reach what one call with the larger d_max
reaches.  On the stepwise path the continued run replays the same operations: the same bits.  The
persistent two-barrier kernel forms basis k-1 at the start of basis k (its second Gram-Schmidt
sweep is deferred), so a run that resumes at d0 forms basis d0 - 1's successor from the caller's
outputs instead: the same pivots, d and stop, and Y, T, err and nu within the plain-form parity
bar.  Every continued run is also held to that bar against the FP64 CPU oracle, for FP64 and FP32
storage, the three tolerance modes and two hops; a run stopped by its tolerance stays stopped.
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


def _same(a, b):
    assert a.d == b.d and a.stop_reason == b.stop_reason and a.next_pivot == b.next_pivot
    assert torch.equal(a.pivots, b.pivots)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T)
    assert torch.equal(a.err, b.err) and torch.equal(a.nu, b.nu)
    assert a.fro_last == b.fro_last


def _close(Xs, a, b, what=""):
    """a and b within the plain-form parity bar: identical pivots, d, stop and next pivot;
    ||dY(:,k)|| <= 1e-10, |dT(k,j)| <= 1e-10 ||x_j||, |derr|, |dnu| <= 1e-10 max_j ||x_j||."""
    assert a.d == b.d and a.stop_reason == b.stop_reason and a.next_pivot == b.next_pivot, what
    assert torch.equal(a.pivots, b.pivots), what
    scale = np.linalg.norm(Xs, axis=0)
    dY = np.linalg.norm(to_numpy(a.Y) - to_numpy(b.Y), axis=0).max()
    dT = (np.abs(to_numpy(a.T) - to_numpy(b.T)) / np.maximum(scale, 1e-300)[None, :]).max()
    dE = (a.err - b.err).abs().max().item() / scale.max()
    dN = (a.nu - b.nu).abs().max().item() / scale.max()
    assert max(dY, dT, dE, dN) <= TOL, f"{what}: dY {dY:.2e} dT {dT:.2e} derr {dE:.2e} dnu {dN:.2e}"
    assert abs(a.fro_last - b.fro_last) <= TOL * np.linalg.norm(Xs), what


def _vs_oracle(oracle_mod, Xs, got, tol, d_max, mode, what=""):
    ref = oracle_mod.compress(Xs, tol, d_max, mode=mode)
    assert got.d == ref["d"] and np.array_equal(got.pivots.cpu().numpy(), ref["pivots"]), what
    scale = np.linalg.norm(Xs, axis=0)
    dY = np.linalg.norm(to_numpy(got.Y) - ref["Y"], axis=0).max()
    dT = (np.abs(to_numpy(got.T) - ref["T"]) / np.maximum(scale, 1e-300)[None, :]).max()
    dE = np.abs(got.err.cpu().numpy() - ref["err"]).max() / scale.max()
    dN = np.abs(got.nu.cpu().numpy() - ref["nu"]).max() / scale.max()
    assert max(dY, dT, dE, dN) <= TOL, f"{what}: dY {dY:.2e} dT {dT:.2e} derr {dE:.2e} dnu {dN:.2e}"


CASES = [
    ("decay 1024x512 fp64", lambda: gen.decay_matrix_c1(seed=0, noise_sigma=1e-5), torch.float64, 1e-6, "maxcol_abs",
     20, 64),
    # (singular values down to 1e-3: a FRO_REL tolerance far below the running indicator's rounding
    # floor, ~1e-8 relative, would decide the stop on noise, and the last steps' ||x_i|| / nu would
    # amplify rounding past the parity bar)
    ("lowrank 1500x700 fro fp64", lambda: gen.lowrank_haar(1500, 700, np.logspace(0, -3, 60), seed=7),
     torch.float64, 1e-5, "fro_rel", 23, 80),
    ("decay 777x333 fp32", lambda: gen.decay_matrix_c1(seed=3, noise_sigma=1e-5, m=777, n=333), torch.float32,
     1e-5, "maxcol_rel", 9, 40),
]


@pytest.mark.parametrize("stepwise", [False, True], ids=["persistent", "stepwise"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_resume_equals_one_call(rbd, oracle_mod, monkeypatch, case, stepwise):
    if stepwise:
        monkeypatch.setenv("RBD_STEPWISE", "1")
    name, build, dtype, tol, mode, d0, d_max = case
    X = to_device(np.asfortranarray(build()), dtype)
    Xs = to_numpy(X)  # the stored values (what the oracle sees)
    full = rbd.compress(X, tol, d_max, tol_mode=mode)
    first = rbd.compress(X, tol, d0, tol_mode=mode)
    assert first.d == d0 and first.stop_reason == "d_max"
    cont = rbd.compress_resume(X, first, tol, d_max, tol_mode=mode)
    # resuming in two hops
    mid = rbd.compress_resume(X, first, tol, (d0 + d_max) // 2, tol_mode=mode)
    two = rbd.compress_resume(X, mid, tol, d_max, tol_mode=mode)
    if stepwise:
        _same(cont, full)
        _same(two, full)
    else:
        _close(Xs, cont, full, f"{name} one hop")
        _close(Xs, two, full, f"{name} two hops")
    _vs_oracle(oracle_mod, Xs, cont, tol, d_max, mode, f"{name} one hop vs oracle")
    _vs_oracle(oracle_mod, Xs, two, tol, d_max, mode, f"{name} two hops vs oracle")


def test_resume_after_tolerance_stop(rbd, oracle_mod):
    Xn = np.asfortranarray(gen.decay_matrix_c1(seed=0, noise_sigma=1e-5))
    X = to_device(Xn)
    done = rbd.compress(X, 1e-3, 64)
    assert done.stop_reason == "tol" and done.d < 64
    again = rbd.compress_resume(X, done, 1e-3, 64)
    assert again.d == done.d and again.stop_reason == "tol"
    finer = rbd.compress_resume(X, done, 1e-4, 64)
    ref = rbd.compress(X, 1e-4, 64)
    # the finer tolerance continues where the coarse one stopped: a fresh run's pivots and bases
    _close(Xn, finer, ref, "finer tolerance")
    _vs_oracle(oracle_mod, Xn, finer, 1e-4, 64, "maxcol_abs", "finer tolerance vs oracle")
