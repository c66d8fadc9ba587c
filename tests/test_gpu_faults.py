"""Failure detection on the GPU path without a GPU fault.

Every device-side wait of the persistent kernels (grid barriers, shared-memory barrier phases,
the service warp's counter, a batched team barrier) is bounded in time.  rbd_set_wait_limit
shortens that bound to 100 ns, so that some wait runs out: the kernel records RBD_ETIMEOUT, its
CTAs leave at their next barrier after their copies in flight have landed, and the call returns
the status instead of trapping or hanging.  With the default bound restored, the next call on the
same inputs must give the same bits as before the failure (the context stays usable and nothing
of the failed call leaks into the next one).
"""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device

pytestmark = pytest.mark.gpu

ETIMEOUT = 5


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def _same(a, b):
    assert a.d == b.d and torch.equal(a.pivots, b.pivots)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T) and torch.equal(a.err, b.err)


def _times_out(rbd, fn):
    prev = rbd.set_wait_limit(100)
    try:
        with pytest.raises(rbd.RbdError) as ei:
            fn()
        assert ei.value.status == ETIMEOUT
    finally:
        rbd.set_wait_limit(prev)


@pytest.mark.parametrize("classic", [False, True], ids=["two-barrier", "four-barrier"])
def test_loop_kernel_wait_runs_out(rbd, monkeypatch, classic):
    if classic:
        monkeypatch.setenv("RBD_LOOP_CLASSIC", "1")
    X = to_device(gen.decay_matrix_c1(seed=0, noise_sigma=1e-5, m=4096, n=2048))
    ref = rbd.compress(X, 0.0, 48)
    assert ref.d == 48
    _times_out(rbd, lambda: rbd.compress(X, 0.0, 48))
    _same(rbd.compress(X, 0.0, 48), ref)


def test_weighted_form_wait_runs_out(rbd):
    Xn = gen.decay_matrix_c1(seed=1, noise_sigma=1e-5, m=3000, n=1200)
    X = to_device(Xn)
    w = torch.as_tensor(np.linspace(0.5, 2.0, 3000), dtype=torch.float64, device="cuda")
    ref = rbd.compress(X, 0.0, 32, weights=w)
    _times_out(rbd, lambda: rbd.compress(X, 0.0, 32, weights=w))
    _same(rbd.compress(X, 0.0, 32, weights=w), ref)


def test_set_wait_limit_returns_previous(rbd):
    prev = rbd.set_wait_limit(12345)
    try:
        assert rbd.set_wait_limit(777) == 12345
    finally:
        rbd.set_wait_limit(prev)
    assert rbd.set_wait_limit(prev) == prev


def test_batched_run_wait_runs_out(rbd):
    items = []
    for i, (m, n) in enumerate([(2048, 700), (1500, 300), (3000, 1100), (800, 256)] * 6):
        X = to_device(gen.lowrank_haar(m, n, np.exp(-0.2 * np.arange(min(m, n))), seed=40 + i), torch.float32)
        items.append({"X": X, "tol": 1e-5, "d_max": 40, "tol_mode": "maxcol_rel", "d_hint": 40})
    plan = rbd.BatchPlan(items)
    plan.run()
    good = plan.results()
    assert all(r["status"] == 0 for r in good)
    ref = [plan.compressed(i, good[i]) for i in range(len(items))]
    ref = [(c.d, c.pivots.clone(), c.Y.clone(), c.T.clone()) for c in ref]
    prev = rbd.set_wait_limit(100)
    try:
        plan.run()
        bad = plan.results()  # synchronises: the run ended
    finally:
        rbd.set_wait_limit(prev)
    assert any(r["status"] == ETIMEOUT for r in bad)
    plan.run()
    again = plan.results()
    assert all(r["status"] == 0 for r in again)
    for i in range(len(items)):
        c = plan.compressed(i, again[i])
        d, piv, Y, T = ref[i]
        assert c.d == d and torch.equal(c.pivots, piv) and torch.equal(c.Y, Y) and torch.equal(c.T, T)
