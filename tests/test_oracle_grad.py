"""Pins of the oracle's adjoint (the differentiation form): the closed form in rbd_oracle.c is
checked against what does not depend on it -- central finite differences of the loss evaluated
through numpy's Householder QR of the fixed pivot columns, special cases with known gradients,
invariance to the order of the pivot set -- and planted mistakes must fail those checks."""
import numpy as np
import pytest

import gen


def qr_factors(X, piv):
    """Y = Q, T = Q' X for the pivot columns in the given order, signs fixed so diag(R) > 0
    (what Gram-Schmidt in pivot order produces)."""
    Q, R = np.linalg.qr(X[:, piv])
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    Q = Q * s[None, :]
    return np.asfortranarray(Q), np.asfortranarray(Q.T @ X)


def loss_qr(X, piv, Xo, w_rec, w_proj):
    """L(X) = w_rec ||(I - Q Q') X||_F^2 + w_proj ||Q' Xo||_F^2, Q from QR of X(:, piv)."""
    Q, _ = np.linalg.qr(X[:, piv])
    E = X - Q @ (Q.T @ X)
    return w_rec * np.sum(E * E) + w_proj * np.sum((Q.T @ Xo) ** 2)


def fd_grad(X, piv, Xo, w_rec, w_proj):
    """Central finite differences of loss_qr, entry by entry (FP64)."""
    h = 1e-6 * np.abs(X).max()
    G = np.zeros_like(X)
    for j in range(X.shape[1]):
        for i in range(X.shape[0]):
            Xp = X.copy()
            Xm = X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            G[i, j] = (loss_qr(Xp, piv, Xo, w_rec, w_proj) - loss_qr(Xm, piv, Xo, w_rec, w_proj)) / (2 * h)
    return G


@pytest.fixture(scope="module")
def sub64x32():
    """The 64 x 32 subproblem: low-rank-plus-decay data, d = 8 pivots chosen by Algorithm 1,
    16 out-of-sample vectors."""
    X = np.asfortranarray(gen.lowrank_haar(64, 32, np.exp(-0.1 * np.arange(32)), seed=21))
    Xo = np.asfortranarray(gen.out_of_sample(64, 16, seed=22))
    return X, Xo


def test_grad_matches_central_differences(oracle_mod, sub64x32):
    X, Xo = sub64x32
    r = oracle_mod.compress(X, 0.0, 8)
    assert r["d"] == 8
    for w_rec, w_proj in ((1.0, 1.0), (1.0, 0.0), (0.0, 1.0), (0.7, 2.5)):
        G, loss = oracle_mod.grad(X, r["Y"], r["T"], r["pivots"], Xo, w_rec, w_proj)
        Gfd = fd_grad(X, list(r["pivots"]), Xo, w_rec, w_proj)
        rel = np.linalg.norm(G - Gfd) / np.linalg.norm(Gfd)
        assert rel <= 1e-6, (w_rec, w_proj, rel)
        assert abs(loss - loss_qr(X, list(r["pivots"]), Xo, w_rec, w_proj)) <= 1e-12 * max(loss, 1.0)


def test_grad_no_basis_is_2x(oracle_mod, sub64x32):
    X, Xo = sub64x32
    G, loss = oracle_mod.grad(X, np.zeros((64, 0)), np.zeros((0, 32)), [], Xo, 1.5, 1.0)
    assert np.allclose(G, 3.0 * X, rtol=0, atol=1e-15)
    assert abs(loss - 1.5 * np.sum(X * X)) <= 1e-12 * loss


def test_grad_full_pivot_set_vanishes(oracle_mod):
    X = np.asfortranarray(gen.lowrank_haar(40, 12, np.linspace(1, 0.2, 12), seed=23))
    piv = list(range(12))[::-1]
    Y, T = qr_factors(X, piv)
    G, loss = oracle_mod.grad(X, Y, T, piv, None, 1.0, 0.0)
    assert np.abs(G).max() <= 1e-12 * np.abs(X).max()
    assert loss <= 1e-24 * np.sum(X * X)


def test_grad_invariant_to_pivot_order(oracle_mod, sub64x32):
    X, Xo = sub64x32
    piv = [3, 17, 0, 25, 9, 30]
    Y1, T1 = qr_factors(X, piv)
    Y2, T2 = qr_factors(X, piv[::-1])
    G1, l1 = oracle_mod.grad(X, Y1, T1, piv, Xo, 1.0, 1.0)
    G2, l2 = oracle_mod.grad(X, Y2, T2, piv[::-1], Xo, 1.0, 1.0)
    assert np.abs(G1 - G2).max() <= 1e-10 * np.abs(G1).max()
    assert abs(l1 - l2) <= 1e-12 * l1


@pytest.mark.parametrize("mutant", [11, 12, 13])
def test_grad_mutant_is_caught(oracle_mod, sub64x32, mutant):
    """11: the R^-T solve dropped; 12: the sign of the residual term flipped; 13: the pivot-column
    term dropped."""
    X, Xo = sub64x32
    oracle_mod.build(mutant)
    r = oracle_mod.compress(X, 0.0, 8)
    G, _ = oracle_mod.grad(X, r["Y"], r["T"], r["pivots"], Xo, 1.0, 1.0, mutant=mutant)
    Gfd = fd_grad(X, list(r["pivots"]), Xo, 1.0, 1.0)
    assert np.linalg.norm(G - Gfd) / np.linalg.norm(Gfd) > 1e-3
