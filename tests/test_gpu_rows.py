"""The row-space form (Section 3.1, "or row if we are compressing the row space"): rbd_compress_rows
on X equals rbd_compress on X' bit for bit (the library's transpose moves the values, the path is
the same), and matches the FP64 oracle run on X' at the plain-form bar."""
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


def _colmajor_transpose(X):
    # column-major n x m tensor holding X' (its storage is X in row-major order)
    return X.contiguous().t()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16], ids=["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("m,n", [(333, 777), (1000, 95), (64, 64), (5000, 130)])
def test_rows_equal_compress_of_transpose(rbd, m, n, dtype):
    Xn = gen.lowrank_haar(m, n, 2.0 ** (-0.3 * np.arange(min(m, n))), seed=m + n, noise_sigma=1e-9)
    X = to_device(Xn, dtype)
    d = min(m, n, 40)
    a = rbd.compress_rows(X, 1e-8, d, start=min(m - 1, 7), tol_mode="maxcol_rel")
    b = rbd.compress(_colmajor_transpose(X), 1e-8, d, start=min(m - 1, 7), tol_mode="maxcol_rel")
    assert a.d == b.d and a.d > 0
    assert torch.equal(a.pivots, b.pivots)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T)
    assert torch.equal(a.err, b.err) and torch.equal(a.nu, b.nu)
    assert a.Y.shape == (n, a.d) and a.T.shape == (a.d, m)
    assert int(a.pivots.max()) < m


@pytest.mark.parametrize("m,n", [(1, 9), (9, 1), (2, 3), (129, 130)])
def test_rows_degenerate_shapes(rbd, oracle_mod, m, n):
    """One row, one column, tiny and just-past-a-tile shapes: the transpose's ragged tiles."""
    rng = np.random.default_rng(m * 31 + n)
    Xn = np.asfortranarray(rng.standard_normal((m, n)))
    d = min(m, n)
    r = rbd.compress_rows(to_device(Xn), 0.0, d)
    ref = oracle_mod.compress(np.asfortranarray(Xn.T), 0.0, d, 0)
    assert r.d == ref["d"]
    assert np.array_equal(r.pivots.cpu().numpy(), ref["pivots"])
    if r.d:
        assert np.linalg.norm(to_numpy(r.Y) - ref["Y"], axis=0).max() <= TOL
        scale = np.linalg.norm(Xn, axis=1)
        assert (np.abs(to_numpy(r.T) - ref["T"]) / scale[None, :]).max() <= TOL


def test_rows_match_oracle(rbd, oracle_mod):
    Xn = gen.decay_matrix_c1(seed=3, noise_sigma=1e-5, m=300, n=1100)
    X = to_device(Xn)
    r = rbd.compress_rows(X, 1e-6, 48, start=5)
    ref = oracle_mod.compress(np.asfortranarray(Xn.T), 1e-6, 48, 5)
    assert r.d == ref["d"]
    assert np.array_equal(r.pivots.cpu().numpy(), ref["pivots"])
    scale = np.linalg.norm(Xn, axis=1)
    assert np.linalg.norm(to_numpy(r.Y) - ref["Y"], axis=0).max() <= TOL
    assert (np.abs(to_numpy(r.T) - ref["T"]) / scale[None, :]).max() <= TOL
    assert np.abs(r.err.cpu().numpy() - ref["err"]).max() <= TOL * scale.max()


def test_rows_padded_leading_dimension(rbd):
    Xn = gen.decay_matrix_c1(seed=4, noise_sigma=1e-5, m=200, n=150)
    big = torch.zeros((150, 256), dtype=torch.float64, device="cuda")
    big[:, :200] = torch.from_numpy(np.ascontiguousarray(Xn.T)).cuda()
    Xpad = big.t()[:200, :]                      # 200 x 150 column-major view with ldx = 256
    a = rbd.compress_rows(Xpad, 0.0, 30)
    b = rbd.compress_rows(to_device(Xn), 0.0, 30)
    assert torch.equal(a.Y, b.Y) and torch.equal(a.T, b.T) and torch.equal(a.pivots, b.pivots)
