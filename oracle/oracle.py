"""ctypes front end of the plain C FP64 oracle (rbd_oracle.c).  Test infrastructure only.

The C file follows Algorithm 1 of the paper step by step (see its header); this module only
builds it with gcc, loads it and marshals numpy arrays.  No arithmetic of the method lives here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

TOL_MODES = {"maxcol_abs": 0, "maxcol_rel": 1, "fro_rel": 2}
# Numerical-rank floor of step 2.2: a pivot whose orthogonalised residual is at most
# RANK_FLOOR * ||X(:, i)|| is treated as already in the span.
RANK_FLOOR = 1e-12

_lock = threading.Lock()
_libs: dict = {}


def _so_path(mutant: int, omp: bool = False) -> str:
    name = "librbd_oracle.so" if mutant == 0 else f"librbd_oracle_mut{mutant}.so"
    if omp:
        name = "librbd_oracle_omp.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False, omp: bool = False) -> str:
    """Compile the oracle (optionally with a planted mistake, for pin tests) with gcc.  omp=True
    builds the same source with OpenMP (its independent column loops on several threads, the
    same arithmetic per column and the same column-order reductions): the all-core CPU baseline."""
    out = _so_path(mutant, omp)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           f"-DRBD_ORACLE_MUTANT={int(mutant)}", _SRC, "-o", tmp, "-lm"]
    if omp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def load(mutant: int = 0, omp: bool = False):
    key = ("omp", 0) if omp else mutant
    with _lock:
        if key in _libs:
            return _libs[key]
        lib = ctypes.CDLL(build(mutant, omp=omp))
        lib.rbd_oracle_set_threads.restype = None
        lib.rbd_oracle_set_threads.argtypes = [ctypes.c_int]
        lib.rbd_oracle_threads.restype = ctypes.c_int
        lib.rbd_oracle_threads.argtypes = []
        i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.rbd_oracle_compress.restype = ctypes.c_int
        lib.rbd_oracle_compress.argtypes = [ptr, i64, i64, i64, dbl, ctypes.c_int, i64, i64, dbl,
                                            ptr, i64, ptr, i64, ptr, ptr, ptr, ptr, ptr, ptr]
        lib.rbd_oracle_compress_weighted.restype = ctypes.c_int
        lib.rbd_oracle_compress_weighted.argtypes = [ptr, i64, i64, i64, ptr, dbl, ctypes.c_int, i64, i64, dbl,
                                                     ptr, i64, ptr, i64, ptr, ptr, ptr, ptr, ptr, ptr]
        lib.rbd_oracle_project.restype = ctypes.c_int
        lib.rbd_oracle_project.argtypes = [ptr, i64, i64, i64, ptr, i64, i64, ptr, i64]
        lib.rbd_oracle_grad.restype = ctypes.c_int
        lib.rbd_oracle_grad.argtypes = [ptr, i64, i64, i64, ptr, i64, ptr, i64, ptr, i64, ptr, i64, i64, dbl, dbl,
                                        ptr, i64, ptr]
        lib.rbd_oracle_reconstruct.restype = ctypes.c_int
        lib.rbd_oracle_reconstruct.argtypes = [ptr, i64, i64, i64, ptr, i64, i64, ptr, i64]
        _libs[key] = lib
        return lib


def _f64_colmajor(a) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return np.asfortranarray(a)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def compress(X, tol: float, d_max: int, start: int = 0, mode: str = "maxcol_abs",
             rank_floor: float = RANK_FLOOR, mutant: int = 0, weights=None, threads: int = 0) -> dict:
    """Run Algorithm 1 on column-major FP64 X (m x n).  Returns a dict with Y (m x d),
    T (d x n), pivots, err, nu, fro (length d), next_pivot and d.  With `weights` (m positive
    values, A = diag(weights)) the error of steps 2.2-2.4 is the A-norm (Section 3.2).
    threads > 0 runs the OpenMP build on that many threads (the same results)."""
    if threads > 0:
        lib = load(omp=True)
        lib.rbd_oracle_set_threads(int(threads))
    else:
        lib = load(mutant)
    X = _f64_colmajor(X)
    m, n = X.shape
    w = None
    if weights is not None:
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
        if w.size != m:
            raise ValueError("weights must have one entry per row of X")
    Y = np.zeros((m, d_max), dtype=np.float64, order="F")
    T = np.zeros((d_max, n), dtype=np.float64, order="F")
    piv = np.zeros(d_max, dtype=np.int64)
    err = np.zeros(d_max)
    nu = np.zeros(d_max)
    fro = np.zeros(d_max)
    nxt = np.zeros(1, dtype=np.int64)
    dout = np.zeros(1, dtype=np.int64)
    if w is None:
        rc = lib.rbd_oracle_compress(_p(X), m, n, m, float(tol), TOL_MODES[mode], int(d_max), int(start),
                                     float(rank_floor), _p(Y), m, _p(T), d_max, _p(piv), _p(err), _p(nu),
                                     _p(fro), _p(nxt), _p(dout))
    else:
        rc = lib.rbd_oracle_compress_weighted(_p(X), m, n, m, _p(w), float(tol), TOL_MODES[mode], int(d_max),
                                              int(start), float(rank_floor), _p(Y), m, _p(T), d_max, _p(piv),
                                              _p(err), _p(nu), _p(fro), _p(nxt), _p(dout))
    if rc != 0:
        raise ValueError(f"rbd_oracle_compress failed with status {rc}")
    d = int(dout[0])
    return {"Y": Y[:, :d].copy(order="F"), "T": T[:d, :].copy(order="F"), "pivots": piv[:d].copy(),
            "err": err[:d].copy(), "nu": nu[:d].copy(), "fro": fro[:d].copy(),
            "next_pivot": int(nxt[0]), "d": d}


def project(Y, V) -> np.ndarray:
    """C = Y' V (the out-of-sample map), FP64 loops."""
    lib = load()
    Y = _f64_colmajor(Y)
    V = _f64_colmajor(V)
    m, d = Y.shape
    if V.shape[0] != m:
        raise ValueError("row mismatch")
    k = V.shape[1]
    C = np.zeros((d, k), dtype=np.float64, order="F")
    rc = lib.rbd_oracle_project(_p(Y), m, d, m, _p(V), k, m, _p(C), max(d, 1))
    if rc != 0:
        raise ValueError(f"rbd_oracle_project failed with status {rc}")
    return C


def reconstruct(Y, T) -> np.ndarray:
    """Xr = Y T (uncompress), FP64 loops."""
    lib = load()
    Y = _f64_colmajor(Y)
    T = _f64_colmajor(T)
    m, d = Y.shape
    n = T.shape[1]
    Xr = np.zeros((m, n), dtype=np.float64, order="F")
    rc = lib.rbd_oracle_reconstruct(_p(Y), m, d, m, _p(T), n, max(d, 1), _p(Xr), m)
    if rc != 0:
        raise ValueError(f"rbd_oracle_reconstruct failed with status {rc}")
    return Xr


def grad(X, Y, T, pivots, Xo=None, w_rec: float = 1.0, w_proj: float = 1.0, mutant: int = 0):
    """Adjoint of L = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2 for the fixed pivot set
    (closed form of rbd_oracle_grad).  Returns (G, loss)."""
    lib = load(mutant)
    X = _f64_colmajor(X)
    m, n = X.shape
    piv = np.ascontiguousarray(np.asarray(pivots, dtype=np.int64).reshape(-1))
    d = piv.size
    Y = _f64_colmajor(np.asarray(Y, dtype=np.float64).reshape(m, d)) if d > 0 else np.zeros((m, 1), order="F")
    T = _f64_colmajor(np.asarray(T, dtype=np.float64).reshape(d, n)) if d > 0 else np.zeros((1, n), order="F")
    if Xo is None:
        Xo = np.zeros((m, 0), order="F")
    Xo = _f64_colmajor(Xo)
    k = Xo.shape[1]
    G = np.zeros((m, n), dtype=np.float64, order="F")
    loss = np.zeros(1)
    rc = lib.rbd_oracle_grad(_p(X), m, n, m, _p(Y), m, _p(T), max(d, 1), _p(piv) if d > 0 else None, d,
                             _p(Xo) if k > 0 else None, k, m, float(w_rec), float(w_proj), _p(G), m, _p(loss))
    if rc != 0:
        raise ValueError(f"rbd_oracle_grad failed with status {rc}")
    return G, float(loss[0])
