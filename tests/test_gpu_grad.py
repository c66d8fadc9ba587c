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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_grad_batched_equals_one_by_one(rbd, dtype):
    """rbd_grad_batched gives each instance rbd_grad's loss and gradient bit for bit, on a ragged
    batch: row counts not multiples of the 32-row block, an instance with d = 0, one without
    out-of-sample data, one with a single out-of-sample vector; and the loss-only form."""
    shapes = [(100, 37, 8, 16), (256, 64, 0, 8), (777, 333, 40, 0), (33, 20, 5, 1), (1024, 512, 32, 256)]
    items = []
    for i, (m, n, d, k) in enumerate(shapes):
        X = to_device(np.asfortranarray(gen.lowrank_haar(m, n, np.exp(-0.1 * np.arange(min(m, n))), seed=300 + i)),
                      dtype)
        Xo = to_device(np.asfortranarray(gen.out_of_sample(m, k, seed=400 + i)), dtype) if k else None
        r = rbd.compress(X, 0.0, max(d, 1))
        items.append({"X": X, "Y": r.Y[:, :d], "T": r.T[:d], "pivots": r.pivots[:d], "Xo": Xo})
    for need in (True, False):
        outs = rbd.grad_batched(items, 1.25, 0.75, need_grad=need)
        for it, (G, loss) in zip(items, outs):
            G1, l1 = rbd.grad(it["X"], it["Y"], it["T"], it["pivots"], it["Xo"], 1.25, 0.75, need_grad=need)
            assert torch.equal(loss, l1)
            assert (G is None and G1 is None) if not need else torch.equal(G, G1)


def test_grad_batched_differentiation_workload(rbd, oracle_mod):
    """The differentiation workload as a batch: the 64 compressions in one batched launch (tol 0,
    d = 32), the 64 adjoints in one rbd_grad_batched call; the pivots equal rbd_compress's, and
    sampled gradients match the oracle's adjoint on the same factors to 1e-10 of max |G|."""
    host = [c5_instance(i) for i in range(64)]
    items = [{"X": to_device(X, torch.float32), "tol": 0.0, "d_max": 32} for X, _ in host]
    plan = rbd.BatchPlan(items)
    plan.run()
    res = plan.results()
    gi = []
    for i, (it, r) in enumerate(zip(items, res)):
        assert r["d"] == 32 and r["status"] == 0, i
        c = plan.compressed(i, r)
        gi.append({"X": it["X"], "Y": c.Y, "T": c.T, "pivots": c.pivots, "Xo": to_device(host[i][1], torch.float32)})
    outs = rbd.grad_batched(gi)
    for i in (0, 21, 63):
        one = rbd.compress(items[i]["X"], 0.0, 32)
        assert torch.equal(one.pivots, gi[i]["pivots"]), i
        X, Xo = host[i]
        Gref, lref = oracle_mod.grad(X.astype(np.float64), to_numpy(gi[i]["Y"]), to_numpy(gi[i]["T"]),
                                     gi[i]["pivots"].cpu().numpy(), Xo.astype(np.float64), 1.0, 1.0)
        G, loss = outs[i]
        assert np.abs(to_numpy(G) - Gref).max() <= 1e-10 * np.abs(Gref).max(), i
        assert abs(loss.item() - lref) <= 1e-12 * lref, i


def test_grad_batched_rejects_mixed_outputs(rbd):
    X = to_device(np.asfortranarray(gen.lowrank_haar(64, 32, np.exp(-0.3 * np.arange(32)), seed=5)))
    r = rbd.compress(X, 0.0, 4)
    it = {"X": X, "Y": r.Y, "T": r.T, "pivots": r.pivots}
    lib = rbd.load()
    from paper_1503_05947_gb300.rbd import _GradItem, _stream_ptr
    G = torch.empty(32, 64, dtype=torch.float64, device=X.device).t()
    loss = torch.empty(2, dtype=torch.float64, device=X.device)
    arr = (_GradItem * 2)()
    for i, g in enumerate((G.data_ptr(), None)):
        arr[i] = _GradItem(X.data_ptr(), 64, 32, 64, it["Y"].data_ptr(), 64, it["T"].data_ptr(), 4,
                           it["pivots"].data_ptr(), 4, None, 0, 64, g, 64, loss[i:].data_ptr())
    assert lib.rbd_grad_batched(arr, 2, 0, 1.0, 1.0, _stream_ptr(X.device)) == 1  # RBD_EINVAL
    assert lib.rbd_grad_batched(arr, 0, 0, 1.0, 1.0, _stream_ptr(X.device)) == 1


def test_batched_autograd_matches_one_by_one(rbd):
    """rbd_loss_batched (batched compression + batched adjoint behind torch.autograd) against
    rbd_loss instance by instance: the same pivots, losses to 1e-12 relative, gradients to 1e-10
    of max |G|; an instance without out-of-sample data and one of another shape in the batch."""
    host = [c5_instance(i) for i in range(3)]
    Xs = [to_device(X, torch.float32).clone().requires_grad_(True) for X, _ in host]
    Xos = [to_device(Xo, torch.float32) for _, Xo in host]
    Xs.append(to_device(np.asfortranarray(gen.lowrank_haar(300, 200, np.exp(-0.2 * np.arange(200)), seed=77)),
                        torch.float32).clone().requires_grad_(True))
    Xos.append(None)
    Xos[1] = None
    w = torch.tensor([1.0, 0.5, 2.0, 1.5], dtype=torch.float32, device="cuda")
    losses = rbd.rbd_loss_batched(Xs, Xos, 24, 1.0, 0.75)
    assert losses.shape == (4,)
    (losses * w).sum().backward()
    for i, (X, Xo) in enumerate(zip(Xs, Xos)):
        Xr = X.detach().clone().requires_grad_(True)
        li = rbd.rbd_loss(Xr, Xo, 24, 1.0, 0.75)
        (li * w[i]).backward()
        assert abs(losses[i].item() - li.item()) <= 1e-6 * abs(li.item()), i  # FP32 outputs
        G, Gr = X.grad.double(), Xr.grad.double()
        assert (G - Gr).abs().max().item() <= 1e-6 * Gr.abs().max().item(), i
