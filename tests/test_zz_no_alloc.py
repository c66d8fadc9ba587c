"""rbd_compress_noalloc (the allocation-free form, fixed device workspace) against rbd_compress.

Both run the same kernels, so the bar is the parity bar of the CUDA path: identical pivots and
d; Y, T, err and nu within 1e-10 (Y columns in norm, T relative to ||x_j||, err and nu relative
to max_j ||x_j||).  Each case makes two calls in a row to check that the fixed workspace is
brought back to its starting state.  This file is collected last so that it also runs after
every other GPU test in the same process.
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


def _host(r):
    return {"Y": to_numpy(r.Y), "T": to_numpy(r.T), "pivots": r.pivots.cpu().numpy(),
            "err": r.err.cpu().numpy(), "nu": r.nu.cpu().numpy(), "d": r.d, "stop": r.stop_reason,
            "next": r.next_pivot}


def _close(Xn, a, b, what):
    assert a["d"] == b["d"], f"{what}: d {a['d']} != {b['d']}"
    assert a["stop"] == b["stop"], f"{what}: stop {a['stop']} != {b['stop']}"
    assert a["next"] == b["next"], f"{what}: next pivot differs"
    assert np.array_equal(a["pivots"], b["pivots"]), f"{what}: pivots differ"
    scale = np.linalg.norm(Xn, axis=0)
    assert np.linalg.norm(a["Y"] - b["Y"], axis=0).max(initial=0.0) <= TOL, what
    assert (np.abs(a["T"] - b["T"]) / np.maximum(scale, 1e-300)[None, :]).max(initial=0.0) <= TOL, what
    assert np.abs(a["err"] - b["err"]).max(initial=0.0) <= TOL * scale.max(), what
    assert np.abs(a["nu"] - b["nu"]).max(initial=0.0) <= TOL * scale.max(), what


CASES = [
    # (name, X builder, dtype, tol, d_max, mode, start)
    ("decay 1024x512 fp64", lambda: gen.decay_matrix_c1(seed=0, noise_sigma=1e-5), torch.float64, 1e-6, 64,
     "maxcol_abs", 0),
    ("lowrank 1500x700 fp64 fro", lambda: gen.lowrank_haar(1500, 700, np.logspace(0, -8, 90), seed=7), torch.float64, 1e-9, 120,
     "fro_rel", 13),
    ("decay 777x333 fp32", lambda: gen.decay_matrix_c1(seed=3, noise_sigma=1e-5, m=777, n=333), torch.float32,
     1e-5, 40, "maxcol_rel", 5),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_compress_twice(rbd, case):
    name, build, dtype, tol, d_max, mode, start = case
    Xn = np.asfortranarray(build())
    X = to_device(Xn, dtype)
    Xn = to_numpy(X)  # the values the kernels see (after any rounding to the storage type)
    ref = _host(rbd.compress(X, tol, d_max, start=start, tol_mode=mode))
    assert ref["d"] >= 2
    for call in range(2):
        r = rbd.compress_noalloc(X, tol, d_max, start=start, tol_mode=mode)
        _close(Xn, _host(r), ref, f"{name}, call {call + 1}")
        assert r.launches == 2  # the initial pass and the persistent loop kernel


def test_noalloc_preallocated_outputs(rbd):
    """Outputs passed in: the call itself makes no allocation; two calls, same results."""
    Xn = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)
    X = to_device(Xn)
    m, n = X.shape
    d_max = 48
    out = {"Y": rbd.colmajor_empty(m, d_max, torch.float64, X.device),
           "T": rbd.colmajor_empty(d_max, n, torch.float64, X.device),
           "pivots": torch.empty(d_max, dtype=torch.int64, device=X.device),
           "err": torch.empty(d_max, dtype=torch.float64, device=X.device),
           "nu": torch.empty(d_max, dtype=torch.float64, device=X.device)}
    ref = _host(rbd.compress(X, 1e-6, d_max))
    for call in range(2):
        got = _host(rbd.compress_noalloc(X, 1e-6, d_max, out=out))
        _close(Xn, got, ref, f"preallocated, call {call + 1}")
        assert got["Y"].shape == (m, d_max) and got["d"] == d_max


def test_noalloc_rejects_oversize(rbd):
    """A problem whose workspace exceeds the fixed array is refused with RBD_ENOMEM before any
    kernel runs; the next call still works."""
    m, n, d_max = 4096, 2048, 16
    assert rbd.workspace_bytes(m, n, d_max, torch.float64) > (64 << 20)
    X = torch.zeros((n, m), dtype=torch.float64, device="cuda:0").t()
    with pytest.raises(rbd.RbdError) as ei:
        rbd.compress_noalloc(X, 0.0, d_max)
    assert ei.value.status == 2  # RBD_ENOMEM
    Xn = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)
    Xs = to_device(Xn)
    ref = _host(rbd.compress(Xs, 1e-6, 32))
    _close(Xn, _host(rbd.compress_noalloc(Xs, 1e-6, 32)), ref, "after oversize")


def test_noalloc_stepwise_path(rbd, monkeypatch):
    """The per-step launch sequence (RBD_STEPWISE=1) of the allocation-free form, which enqueues
    every step without a host-visible progress word, against rbd_compress on the same path."""
    monkeypatch.setenv("RBD_STEPWISE", "1")
    Xn = gen.decay_matrix_c1(seed=0, noise_sigma=1e-5)
    X = to_device(Xn)
    ref = _host(rbd.compress(X, 1e-3, 64))
    assert 2 <= ref["d"] < 64  # stops on the tolerance, so later launches return at entry
    for call in range(2):
        got = rbd.compress_noalloc(X, 1e-3, 64)
        _close(Xn, _host(got), ref, f"stepwise, call {call + 1}")
        # every step up to d_max is enqueued (init, then per step the orthogonalisation kernels
        # and the pass): 4 d_max + 3 launches, whatever step the device stopped at
        assert got.launches == 4 * 64 + 3
