"""The differentiation form on the GPU: rbd_grad (the hand-written adjoint, through the C ABI) and
its torch.autograd binding, against the oracle's adjoint and against central finite differences.

* 64 x 32 FP64 subproblem, d = 8 pivots chosen by the CUDA path: the adjoint agrees with FP64
  central differences of L evaluated through numpy's QR of the fixed pivot columns to 1e-6
  relative (the differentiation form's bar).
* The batch of the differentiation workload: 64 FP32 matrices 1024 x 512 (low rank, decay 0.1),
  d = 32, 256 out-of-sample vectors N(0, 1/m) each.  Elementwise against the oracle's adjoint
  evaluated on the same (Y, T, pivots): |dG| <= 1e-10 max |G|, loss to 1e-12 relative.
"""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device, to_numpy
from test_oracle_grad import fd_grad, loss_qr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


def c5_instance(i):
    X = gen.lowrank_haar(1024, 512, np.exp(-0.1 * np.arange(512)), seed=1000 + i)
    Xo = gen.out_of_sample(1024, 256, seed=2000 + i)
    return np.asfortranarray(X.astype(np.float32)), np.asfortranarray(Xo.astype(np.float32))


def test_grad_matches_finite_differences(rbd):
    X = np.asfortranarray(gen.lowrank_haar(64, 32, np.exp(-0.1 * np.arange(32)), seed=21))
    Xo = np.asfortranarray(gen.out_of_sample(64, 16, seed=22))
    Xd, Xod = to_device(X), to_device(Xo)
    r = rbd.compress(Xd, 0.0, 8)
    assert r.d == 8
    piv = list(r.pivots.cpu().numpy())
    for w_rec, w_proj in ((1.0, 1.0), (0.7, 2.5), (1.0, 0.0)):
        G, loss = rbd.grad(Xd, r.Y, r.T, r.pivots, Xod, w_rec, w_proj)
        Gfd = fd_grad(X, piv, Xo, w_rec, w_proj)
        rel = np.linalg.norm(to_numpy(G) - Gfd) / np.linalg.norm(Gfd)
        assert rel <= 1e-6, (w_rec, w_proj, rel)
        ref = loss_qr(X, piv, Xo, w_rec, w_proj)
        assert abs(loss.item() - ref) <= 1e-12 * ref


def test_autograd_backward_matches_adjoint(rbd):
    X = np.asfortranarray(gen.lowrank_haar(64, 32, np.exp(-0.1 * np.arange(32)), seed=21))
    Xo = np.asfortranarray(gen.out_of_sample(64, 16, seed=22))
    Xt = to_device(X).clone().requires_grad_(True)
    Xot = to_device(Xo)
    loss = rbd.rbd_loss(Xt, Xot, 8, 1.0, 1.0)
    loss.backward()
    r = rbd.compress(to_device(X), 0.0, 8)
    G, l2 = rbd.grad(to_device(X), r.Y, r.T, r.pivots, Xot, 1.0, 1.0)
    assert torch.equal(Xt.grad, G)
    assert loss.item() == l2.item()
    Gfd = fd_grad(X, list(r.pivots.cpu().numpy()), Xo, 1.0, 1.0)
    assert np.linalg.norm(to_numpy(Xt.grad) - Gfd) / np.linalg.norm(Gfd) <= 1e-6


def test_loss_only_and_empty_basis(rbd):
    X, Xo = c5_instance(0)
    Xd, Xod = to_device(X, torch.float32), to_device(Xo, torch.float32)
    r = rbd.compress(Xd, 0.0, 32)
    G, l1 = rbd.grad(Xd, r.Y, r.T, r.pivots, Xod, 1.0, 1.0)
    none, l0 = rbd.grad(Xd, r.Y, r.T, r.pivots, Xod, 1.0, 1.0, need_grad=False)
    assert none is None and l0.item() == l1.item()
    G0, loss0 = rbd.grad(Xd, r.Y, r.T, r.pivots[:0], Xod, 1.5, 1.0)
    X64 = X.astype(np.float64)
    assert np.abs(to_numpy(G0) - 3.0 * X64).max() <= 1e-12 * np.abs(X64).max()
    assert abs(loss0.item() - 1.5 * np.sum(X64 * X64)) <= 1e-12 * loss0.item()


def test_differentiation_workload_batch_matches_oracle(rbd, oracle_mod):
    """64 instances of 1024 x 512 FP32, d = 32, 256 out-of-sample vectors each, through the
    autograd binding; each gradient against the oracle's adjoint on the same factors."""
    worst = 0.0
    for i in range(64):
        X, Xo = c5_instance(i)
        Xt = to_device(X, torch.float32).clone().requires_grad_(True)
        Xot = to_device(Xo, torch.float32)
        loss = rbd.rbd_loss(Xt, Xot, 32)
        loss.backward()
        r = rbd.compress(to_device(X, torch.float32), 0.0, 32)
        assert r.d == 32
        G, lg = rbd.grad(to_device(X, torch.float32), r.Y, r.T, r.pivots, Xot, 1.0, 1.0)
        Gref, lref = oracle_mod.grad(X.astype(np.float64), to_numpy(r.Y), to_numpy(r.T), r.pivots.cpu().numpy(),
                                     Xo.astype(np.float64), 1.0, 1.0)
        Gn = to_numpy(G)
        dG = np.abs(Gn - Gref).max() / np.abs(Gref).max()
        worst = max(worst, dG)
        assert dG <= 1e-10, (i, dG)
        assert abs(lg.item() - lref) <= 1e-12 * lref, i
        # the autograd gradient is the adjoint cast to the input dtype
        assert np.abs(to_numpy(Xt.grad) - Gn).max() <= 1e-6 * np.abs(Gn).max()
