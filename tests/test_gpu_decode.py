"""Uncompress (Section 3.1, rbd_reconstruct through the C ABI): Xr = Y T against the oracle's FP64
loops, on the CUDA path's own compression outputs.  Bar: |dXr| <= 1e-13 max_j ||x_j|| (the sums
over d bases are float-float, relative error ~2^-47 of sum |y t|).  Also column subsets through a
shifted T pointer, Y c for projected out-of-sample vectors (= the orthogonal projection onto
span Y), ragged sizes, d = 0 and n = 0."""
import numpy as np
import pytest
import torch

import gen
from gpu_util import to_device, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_05947_gb300 as pkg
    pkg.load()
    return pkg


@pytest.mark.parametrize("m,n,d_max", [(1024, 512, 64), (777, 333, 50), (33, 1000, 33), (3001, 97, 97)])
def test_reconstruct_matches_oracle(rbd, oracle_mod, m, n, d_max):
    X = np.asfortranarray(gen.decay_matrix_c1(seed=5, noise_sigma=1e-5, m=m, n=n))
    r = rbd.compress(to_device(X), 0.0, d_max)
    Y, T = to_numpy(r.Y), to_numpy(r.T)
    ref = oracle_mod.reconstruct(Y, T)
    got = to_numpy(rbd.reconstruct(r.Y, r.T))
    scale = np.linalg.norm(X, axis=0).max()
    assert np.abs(got - ref).max() <= 1e-13 * scale
    # the compression error it implies equals the one the compression reported, up to the floor of
    # the running indicator (squared norms downdated in FP64: sqrt(n eps) max_j ||x_j||)
    floor = 4 * np.sqrt(n * 2.0 ** -52) * scale
    assert abs(np.linalg.norm(X - got) - r.fro_last) <= 1e-9 * np.linalg.norm(X) + floor


def test_reconstruct_column_subset_and_vectors(rbd, oracle_mod):
    X = np.asfortranarray(gen.decay_matrix_c1(seed=6, noise_sigma=1e-5))
    r = rbd.compress(to_device(X), 1e-6, 48)
    sub = rbd.reconstruct(r.Y, r.T[:, 100:164])
    full = rbd.reconstruct(r.Y, r.T)
    assert torch.equal(sub, full[:, 100:164])
    V = to_device(np.asfortranarray(gen.out_of_sample(1024, 9, seed=7)))
    C = rbd.project(r.Y, V)
    P = to_numpy(rbd.reconstruct(r.Y, C))
    Yn = to_numpy(r.Y)
    ref = Yn @ (Yn.T @ to_numpy(V))
    assert np.abs(P - ref).max() <= 1e-13 * np.abs(ref).max()
    one = rbd.reconstruct(r.Y, C[:, 3])
    assert torch.equal(one[:, 0], rbd.reconstruct(r.Y, C)[:, 3])


def test_reconstruct_degenerate(rbd):
    Y = torch.zeros((50, 0), dtype=torch.float64, device="cuda")
    T = torch.zeros((0, 7), dtype=torch.float64, device="cuda")
    out = rbd.reconstruct(Y, T)
    assert out.shape == (50, 7) and torch.count_nonzero(out).item() == 0
    Y1 = torch.ones((3, 50), dtype=torch.float64, device="cuda").t()
    T0 = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    assert rbd.reconstruct(Y1, T0).shape == (50, 0)


def test_reconstruct_wide_grid(rbd):
    """More column tiles than a grid's y extent holds (n > 65535 x 64): the kernel walks the
    remaining tiles; sampled columns against numpy."""
    m, d, n = 3, 2, 65535 * 64 + 100
    g = torch.Generator(device="cuda").manual_seed(11)
    Y = torch.randn((d, m), dtype=torch.float64, device="cuda", generator=g).t()
    T = torch.randn((n, d), dtype=torch.float64, device="cuda", generator=g).t()
    out = rbd.reconstruct(Y, T)
    cols = torch.tensor([0, 1, 65535 * 64 - 1, 65535 * 64, n - 1], device="cuda")
    ref = (to_numpy(Y) @ to_numpy(T[:, cols]))
    assert np.abs(to_numpy(out[:, cols]) - ref).max() <= 1e-13 * np.abs(ref).max()
    assert torch.isfinite(out).all()
