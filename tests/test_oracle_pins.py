"""The FP64 CPU oracle against the pins (what the paper and the mathematics fix)."""
import numpy as np
import pytest

import gen
import pins


@pytest.fixture(scope="module")
def compress(oracle_mod):
    return oracle_mod.compress


@pytest.mark.parametrize("pin", pins.FAST_PINS, ids=lambda p: p.__name__)
def test_pin(pin, compress):
    pin(compress)


@pytest.mark.parametrize("pin", pins.W_PINS, ids=lambda p: p.__name__)
def test_weighted_pin(pin, compress):
    pin(compress)


def test_weighted_invalid(oracle_mod):
    X = np.ones((4, 3), order="F")
    for w in (np.array([1.0, 0.0, 1.0, 1.0]), np.array([1.0, -2.0, 1.0, 1.0]), np.array([1.0, np.nan, 1.0, 1.0])):
        with pytest.raises(ValueError, match="status 1"):
            oracle_mod.compress(X, 0.0, 2, weights=w)


def test_paper_rank_functions(compress):
    pins.pin_paper_rank_functions(compress)


@pytest.mark.slow
def test_paper_approx_example(compress):
    pins.pin_paper_approx_example(compress)


def test_rank_function_grid_aliasing(compress):
    """A grid with spacing 0.01 samples sin(100 pi x) only at its zeros, so the rank-3 function
    of Section 4.2.1 looks rank 2 there (why the rank pins use a 1000-point grid)."""
    X = gen.paper_rank_function(201, 3)
    assert compress(X, 1e-10, 10)["d"] == 2


def test_project_and_reconstruct(oracle_mod):
    X = gen.decay_matrix_c1(seed=0, m=128, n=96)
    r = oracle_mod.compress(X, 0.0, 20)
    Y, T = r["Y"], r["T"]
    assert np.abs(oracle_mod.project(Y, Y) - np.eye(20)).max() <= 1e-14
    assert np.abs(oracle_mod.project(Y, X) - T).max() <= 1e-14
    V = gen.out_of_sample(128, 7, seed=3)
    C = oracle_mod.project(Y, V)
    assert np.abs(C - Y.T @ V).max() <= 1e-14
    assert np.abs(oracle_mod.reconstruct(Y, T) - Y @ T).max() <= 1e-14


@pytest.mark.parametrize("r", [1, 5, 17])
def test_reconstruct_exact_recovery(oracle_mod, r):
    """Uncompress (Section 3.1) after Algorithm 1 on a rank-r matrix stops at d = r: Y T is X
    itself, up to rounding (Y spans the column space exactly)."""
    X = gen.lowrank_haar(90, 70, np.linspace(2.0, 0.5, r), seed=100 + r)
    res = oracle_mod.compress(X, 1e-12, 40)
    assert res["d"] == r
    Xr = oracle_mod.reconstruct(res["Y"], res["T"])
    assert np.abs(Xr - X).max() <= 1e-13 * np.abs(X).max()


def test_reconstruct_of_projection_is_identity_on_span(oracle_mod):
    """For v in span(Y), the out-of-sample map followed by uncompress returns v: Y (Y' v) = v."""
    X = gen.decay_matrix_c1(seed=5, m=150, n=80)
    Y = oracle_mod.compress(X, 0.0, 24)["Y"]
    rng = np.random.default_rng(7)
    V = np.asfortranarray(Y @ rng.standard_normal((24, 9)))
    back = oracle_mod.reconstruct(Y, oracle_mod.project(Y, V))
    assert np.abs(back - V).max() <= 1e-13 * np.abs(V).max()
    # and for any v, the residual v - Y Y'v is orthogonal to Y (Galerkin): Y'(v - Y Y' v) = 0
    W = gen.out_of_sample(150, 5, seed=11)
    R = W - oracle_mod.reconstruct(Y, oracle_mod.project(Y, W))
    assert np.abs(oracle_mod.project(Y, R)).max() <= 1e-14 * np.abs(W).max() * 150


def test_invalid_arguments(oracle_mod):
    X = np.ones((4, 3), order="F")
    for kw in (dict(tol=-1.0, d_max=2), dict(tol=0.0, d_max=0), dict(tol=0.0, d_max=4),
               dict(tol=0.0, d_max=2, start=3), dict(tol=0.0, d_max=2, start=-1)):
        with pytest.raises(ValueError):
            oracle_mod.compress(X, **kw)
    Xn = X.copy(order="F")
    Xn[1, 1] = np.nan
    with pytest.raises(ValueError, match="status 4"):
        oracle_mod.compress(Xn, 0.0, 2)
