"""Seeded synthetic input matrices with the shapes and structure of the paper's workloads.

Every generator returns FP64 (or uint8 for the quantised image field) numpy arrays in
COLUMN-MAJOR layout: an m x n matrix X is an ``order='F'`` array, so column j (one data
entry ``X(:, j)`` of Section 3.1) is contiguous in memory, the layout the library expects.

Nothing here implements the compression method; these are only data recipes:

* ``decay_matrix_c1``     U diag(s) V^T + noise with Haar U, V and s_i = 2^(-i/4) (1024 x 512).
* ``image_like_u8``       an 8192 x 8192 grayscale field of Gaussian bumps and plane sinusoids,
                          quantised to uint8; stands in for the paper's test images
                          (Section 4.1), which are not available here.
* ``parametric_snapshots``  columns f(s; mu) = 1/sqrt((s - mu1)^2 + mu2^2) on a uniform grid.
* ``paper_rank_function`` the three tensorial functions of Section 4.2.1 (Table of intrinsic
                          dimensions 1, 2, 3) sampled on a uniform grid of [-1, 1]^2.
* ``paper_approx_function`` the function 0.6 f1 + 0.1 f2 + 0.01 f3 of Section 4.2.2.
* ``orthogonal_columns``  scaled, permuted standard basis vectors (exactly orthogonal columns
                          with exactly known norms), for closed-form checks.
"""
from __future__ import annotations

import numpy as np


def haar_orthonormal(rng: np.random.Generator, m: int, r: int) -> np.ndarray:
    """m x r matrix with orthonormal columns drawn from the Haar measure.

    QR of an i.i.d. standard normal matrix, with each column's sign fixed by the sign of the
    corresponding diagonal entry of R (Mezzadri's recipe), so the law is exactly Haar.
    """
    g = rng.standard_normal((m, r))
    q, rr = np.linalg.qr(g)
    sgn = np.sign(np.diag(rr))
    sgn[sgn == 0] = 1.0
    return np.asfortranarray(q * sgn)


def lowrank_haar(m: int, n: int, s: np.ndarray, seed: int, noise_sigma: float = 0.0) -> np.ndarray:
    """X = U diag(s) V^T + noise, U (m x r) and V (n x r) Haar, r = len(s)."""
    rng = np.random.default_rng(seed)
    r = len(s)
    u = haar_orthonormal(rng, m, r)
    v = haar_orthonormal(rng, n, r)
    x = (u * np.asarray(s, dtype=np.float64)) @ v.T
    if noise_sigma:
        x = x + noise_sigma * rng.standard_normal((m, n))
    return np.asfortranarray(x)


def decay_matrix_c1(seed: int = 0, noise_sigma: float = 1e-5, m: int = 1024, n: int = 512) -> np.ndarray:
    """The small plain-FP64 workload: 1024 x 512, s_i = 2^(-i/4), i = 0..min(m,n)-1, plus
    i.i.d. N(0, noise_sigma^2) noise (the noise is read as a standard deviation of 1e-5)."""
    r = min(m, n)
    s = 2.0 ** (-np.arange(r) / 4.0)
    return lowrank_haar(m, n, s, seed, noise_sigma)


def image_like_factors(npix: int, seed: int, n_bumps: int = 200, n_sin: int = 20):
    """Separable factors (F, G) of the smooth field V = F G^T before quantisation.

    Each isotropic Gaussian bump A exp(-((r-cy)^2 + (c-cx)^2) / (2 sigma^2)) is the product of a
    row factor and a column factor (rank 1); each plane sinusoid A sin(a c + b r + phi) is the
    sum of two such products (rank 2).  Row index r is the image row (matrix row), column index
    c the image column (matrix column).  Parameters:
    centres U[0, npix)^2, sigma U[8, 512] px, amplitude U[-1, 1];
    sinusoid amplitude U[0, 0.1], direction U[0, 2 pi), wavelength log-uniform [16, 4096] px,
    phase U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    pix = np.arange(npix, dtype=np.float64)
    cols_f, cols_g = [], []
    cy = rng.uniform(0, npix, n_bumps)
    cx = rng.uniform(0, npix, n_bumps)
    sig = rng.uniform(8, 512, n_bumps)
    amp = rng.uniform(-1, 1, n_bumps)
    for k in range(n_bumps):
        cols_f.append(amp[k] * np.exp(-((pix - cy[k]) ** 2) / (2 * sig[k] ** 2)))
        cols_g.append(np.exp(-((pix - cx[k]) ** 2) / (2 * sig[k] ** 2)))
    a_s = rng.uniform(0, 0.1, n_sin)
    theta = rng.uniform(0, 2 * np.pi, n_sin)
    lam = np.exp(rng.uniform(np.log(16.0), np.log(4096.0), n_sin))
    phi = rng.uniform(0, 2 * np.pi, n_sin)
    for k in range(n_sin):
        a = 2 * np.pi * np.cos(theta[k]) / lam[k]   # along columns (image x)
        b = 2 * np.pi * np.sin(theta[k]) / lam[k]   # along rows (image y)
        cols_f.append(a_s[k] * np.sin(b * pix + phi[k]))
        cols_g.append(np.cos(a * pix))
        cols_f.append(a_s[k] * np.cos(b * pix + phi[k]))
        cols_g.append(np.sin(a * pix))
    f = np.stack(cols_f, axis=1)
    g = np.stack(cols_g, axis=1)
    return f, g


def image_like_u8(npix: int = 8192, seed: int = 1, n_bumps: int = 200, n_sin: int = 20) -> np.ndarray:
    """npix x npix uint8 field (column-major): V = F G^T min-max scaled to [0, 1], then
    q = round(255 v).  Convert with ``u8_to_unit_f64`` (q / 255) to get the FP64 matrix."""
    f, g = image_like_factors(npix, seed, n_bumps, n_sin)
    # Build column blocks of V = F G^T directly in column-major order.
    v = np.empty((npix, npix), dtype=np.float64, order="F")
    blk = 1024
    for c0 in range(0, npix, blk):
        v[:, c0:c0 + blk] = f @ g[c0:c0 + blk].T
    vmin, vmax = float(v.min()), float(v.max())
    v -= vmin
    v *= 1.0 / (vmax - vmin)
    v *= 255.0
    np.rint(v, out=v)
    q = np.asfortranarray(v.astype(np.uint8))
    return q


def u8_to_unit_f64(q: np.ndarray) -> np.ndarray:
    """uint8 levels -> FP64 values q / 255 in [0, 1], column-major."""
    return np.asfortranarray(q.astype(np.float64) / 255.0)


def parametric_params(m: int, n: int, seed: int = 2):
    """Grid and parameters of the parametric snapshot matrix: s_i = i / (m - 1) (m points),
    mu1 ~ U[-1, -0.01], mu2 ~ U[0.01, 1] (n each, seeded)."""
    rng = np.random.default_rng(seed)
    mu1 = rng.uniform(-1.0, -0.01, n)
    mu2 = rng.uniform(0.01, 1.0, n)
    s = np.arange(m, dtype=np.float64) / max(m - 1, 1)
    return s, mu1, mu2


def parametric_snapshots(m: int, n: int, seed: int = 2) -> np.ndarray:
    """Column j = f(s; mu_j) = 1 / sqrt((s - mu1_j)^2 + mu2_j^2) on s_i = i / (m - 1);
    mu1 ~ U[-1, -0.01], mu2 ~ U[0.01, 1] (seeded)."""
    s, mu1, mu2 = parametric_params(m, n, seed)
    x = 1.0 / np.sqrt((s[:, None] - mu1[None, :]) ** 2 + mu2[None, :] ** 2)
    return np.asfortranarray(x)


def parametric_snapshots_torch(m: int, n: int, seed: int = 2, device="cuda", dtype=None):
    """The same matrix built with torch on `device` (column-major), for sizes too large to build
    on the host: the same seeded parameters, the same formula evaluated elementwise in FP64,
    then cast to `dtype` (round to nearest)."""
    import torch
    s, mu1, mu2 = parametric_params(m, n, seed)
    st = torch.from_numpy(s).to(device)
    m1 = torch.from_numpy(mu1).to(device)
    m2 = torch.from_numpy(mu2).to(device)
    xt = torch.empty((n, m), dtype=dtype or torch.float64, device=device)
    step = max(1, (1 << 27) // max(m, 1))
    for j0 in range(0, n, step):
        j1 = min(n, j0 + step)
        blk = 1.0 / torch.sqrt((st[None, :] - m1[j0:j1, None]) ** 2 + m2[j0:j1, None] ** 2)
        xt[j0:j1] = blk.to(xt.dtype)
    return xt.t()


def paper_rank_function(npts: int, which: int) -> np.ndarray:
    """Section 4.2.1 (Table of three tensorial functions with intrinsic dimension 1, 2, 3):
    X[i, j] = f(x_i, y_j) on a uniform npts x npts grid of [-1, 1]^2.

    which = 1: sin(pi x) cos(pi y)
    which = 2: ... + 0.1 sin(10 pi x) cos(10 pi y)
    which = 3: ... + 0.01 sin(100 pi x) cos(100 pi y)
    A grid whose spacing makes 100 x_i an integer (e.g. npts = 201) samples sin(100 pi x) at its
    zeros and hides the third term; npts = 1000 does not.
    """
    g = np.linspace(-1.0, 1.0, npts)
    x = g[:, None]
    y = g[None, :]
    f = np.sin(np.pi * x) * np.cos(np.pi * y)
    if which >= 2:
        f = f + 0.1 * np.sin(10 * np.pi * x) * np.cos(10 * np.pi * y)
    if which >= 3:
        f = f + 0.01 * np.sin(100 * np.pi * x) * np.cos(100 * np.pi * y)
    return np.asfortranarray(f)


def paper_approx_function(npts: int = 5001) -> np.ndarray:
    """Section 4.2.2: f = 0.6 f1 + 0.1 f2 + 0.01 f3 on a uniform npts x npts grid of [-1, 1]^2,
    f1 = sin(pi (x + 2y)) cos(pi (2x - y)), f2 = sin(10 pi (x - 3y)) cos(10 pi (3x + y)),
    f3 = sin(3 pi x^2 y) cos(6 pi sqrt|x| / (y + 2)).  X[i, j] = f(x_i, y_j)."""
    g = np.linspace(-1.0, 1.0, npts)
    x = g[:, None]
    y = g[None, :]
    f1 = np.sin(np.pi * (x + 2 * y)) * np.cos(np.pi * (2 * x - y))
    f2 = np.sin(10 * np.pi * (x - 3 * y)) * np.cos(10 * np.pi * (3 * x + y))
    f3 = np.sin(3 * np.pi * x * x * y) * np.cos(6 * np.pi * np.sqrt(np.abs(x)) / (y + 2))
    return np.asfortranarray(0.6 * f1 + 0.1 * f2 + 0.01 * f3)


def orthogonal_columns(m: int, norms, seed: int = 0) -> np.ndarray:
    """m x n matrix whose column j is norms[j] * e_{p(j)} for a seeded injective row map p:
    columns are exactly orthogonal and have exactly the given norms (n <= m)."""
    norms = np.asarray(norms, dtype=np.float64)
    n = len(norms)
    if n > m:
        raise ValueError("need n <= m for orthogonal columns")
    rng = np.random.default_rng(seed)
    rows = rng.permutation(m)[:n]
    x = np.zeros((m, n), dtype=np.float64, order="F")
    x[rows, np.arange(n)] = norms
    return x


def row_weights(m: int, seed: int = 0, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """m positive weights for the diagonal A-norm of Section 3.2: a smooth profile (a Gaussian
    bump over a random third of the rows, "part of each entry preserved better") times a seeded
    log-uniform factor per row, clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    r = np.arange(m, dtype=np.float64)
    c = rng.uniform(0.2, 0.8) * m
    width = max(m / 6.0, 1.0)
    smooth = 1.0 + (hi - 1.0) * np.exp(-0.5 * ((r - c) / width) ** 2)
    jitter = np.exp(rng.uniform(np.log(0.5), np.log(2.0), m))
    return np.clip(smooth * jitter, lo, hi)


def out_of_sample(m: int, k: int, seed: int) -> np.ndarray:
    """k i.i.d. N(0, 1/m) vectors of length m, column-major m x k."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, k)) / np.sqrt(m))


def batch_specs(count: int = 2048, seed: int = 3):
    """Sizes and parameters of the batched workload: m log-uniform in [256, 4096] and n
    log-uniform in [64, 2048] (rounded), decay rate r ~ U[0.05, 0.5], tolerance log-uniform in
    [1e-6, 1e-2] (relative max-column mode), d_max = min(m, n, 512)."""
    rng = np.random.default_rng(seed)
    m = np.rint(np.exp(rng.uniform(np.log(256), np.log(4096), count))).astype(np.int64)
    n = np.rint(np.exp(rng.uniform(np.log(64), np.log(2048), count))).astype(np.int64)
    r = rng.uniform(0.05, 0.5, count)
    tol = np.exp(rng.uniform(np.log(1e-6), np.log(1e-2), count))
    # expected number of bases: the tolerance is reached where exp(-r d) ~ tol (a scheduling hint)
    return [{"m": int(m[i]), "n": int(n[i]), "rate": float(r[i]), "tol": float(tol[i]),
             "d_max": int(min(m[i], n[i], 512)), "seed": seed * 100003 + i,
             "d_hint": int(min(min(m[i], n[i], 512), np.ceil(np.log(1.0 / tol[i]) / r[i]) + 1))}
            for i in range(count)]


def decay_spectrum(rate: float, r_max: int) -> np.ndarray:
    """s_i = exp(-rate i), i = 0.., truncated where s_i < 1e-9 (at most r_max values)."""
    r = int(min(r_max, np.floor(np.log(1e9) / rate) + 1))
    return np.exp(-rate * np.arange(r))


def lowrank_torch(m: int, n: int, s: np.ndarray, seed: int, device="cuda", dtype=None):
    """X = U diag(s) V^T with Haar-distributed U (m x r), V (n x r) built with torch on `device`
    (QR of seeded Gaussian matrices, signs fixed), cast to `dtype`; column-major."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    r = len(s)
    A = torch.randn(m, r, generator=g, dtype=torch.float64).to(device)
    B = torch.randn(n, r, generator=g, dtype=torch.float64).to(device)
    qa, ra = torch.linalg.qr(A)
    qb, rb = torch.linalg.qr(B)
    qa = qa * torch.sign(torch.diagonal(ra))[None, :]
    qb = qb * torch.sign(torch.diagonal(rb))[None, :]
    st = torch.from_numpy(np.asarray(s, dtype=np.float64)).to(device)
    X = (qa * st[None, :]) @ qb.t()
    return X.to(dtype or torch.float64).t().contiguous().t()
