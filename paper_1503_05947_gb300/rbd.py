"""Python binding of librbd.so (include/rbd.h): argument marshalling only.

Every step of Reduced Basis Decomposition runs in the library's CUDA kernels; this module only
checks tensor layouts, allocates outputs with PyTorch and passes raw pointers and the current
CUDA stream.  There is no CPU fallback: if the library is missing, every call raises.

Layout: matrices are column-major.  A torch tensor ``X`` of shape (m, n) is column-major when
``X.stride(0) == 1`` (e.g. ``A.t()`` of a contiguous (n, m) tensor); its leading dimension is
``X.stride(1)``.  Outputs are returned as column-major views with the same convention.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import torch

from . import buildlib as _build

_I64, _DBL, _PTR = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p

DTYPES = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
TOL_MODES = {"maxcol_abs": 0, "maxcol_rel": 1, "fro_rel": 2, "none": 3}
STOP_REASONS = {0: "none", 1: "tol", 2: "break", 3: "d_max"}
RANK_FLOOR = 1e-12


class RbdError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class _Result(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("next_pivot", ctypes.c_int64), ("stop_reason", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("err_last", ctypes.c_double), ("fro_last", ctypes.c_double),
                ("x_fro", ctypes.c_double), ("x_maxcol", ctypes.c_double)]


class _Profile(ctypes.Structure):
    _fields_ = [("pass_launches", ctypes.c_int64), ("pass_ms", ctypes.c_double),
                ("orth_launches", ctypes.c_int64), ("orth_ms", ctypes.c_double), ("init_ms", ctypes.c_double),
                ("pass_bytes", ctypes.c_int64), ("loop_launches", ctypes.c_int64), ("loop_ms", ctypes.c_double),
                ("loop_kernel", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _BatchConfig(ctypes.Structure):
    _fields_ = [("cols", ctypes.c_int32), ("tile_rows", ctypes.c_int32), ("team_pct", ctypes.c_int32),
                ("stages", ctypes.c_int32)]


class _GradItem(ctypes.Structure):
    _fields_ = [("X", _PTR), ("m", _I64), ("n", _I64), ("ldx", _I64), ("Y", _PTR), ("ldy", _I64), ("T", _PTR),
                ("ldt", _I64), ("pivots", _PTR), ("d", _I64), ("Xo", _PTR), ("k", _I64), ("ldxo", _I64), ("G", _PTR),
                ("ldg", _I64), ("loss", _PTR)]


class _Instance(ctypes.Structure):
    _fields_ = [("X", _PTR), ("m", _I64), ("n", _I64), ("ldx", _I64), ("tol", _DBL), ("mode", ctypes.c_int32),
                ("d_hint", ctypes.c_int32), ("d_max", _I64), ("start", _I64), ("Y", _PTR), ("ldy", _I64),
                ("T", _PTR), ("ldt", _I64), ("pivots", _PTR), ("err", _PTR), ("nu", _PTR)]


# rbd_batch_result as a numpy record (device results are copied as bytes)
_BATCH_RESULT_BYTES = 56  # sizeof(rbd_batch_result)


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load librbd.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"librbd.so not found at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    lib.rbd_compress_workspace_bytes.restype = ctypes.c_size_t
    lib.rbd_compress_workspace_bytes.argtypes = [_I64, _I64, _I64, ctypes.c_int]
    lib.rbd_compress.restype = ctypes.c_int
    lib.rbd_compress.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _DBL, ctypes.c_int, _I64, _I64,
                                 _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.c_size_t, _PTR,
                                 ctypes.POINTER(_Result)]
    lib.rbd_compress_weighted.restype = ctypes.c_int
    lib.rbd_compress_weighted.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _PTR, _DBL, ctypes.c_int, _I64, _I64,
                                          _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.c_size_t, _PTR,
                                          ctypes.POINTER(_Result)]
    lib.rbd_compress_rows.restype = ctypes.c_int
    lib.rbd_compress_rows.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _DBL, ctypes.c_int, _I64, _I64,
                                      _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.POINTER(_Result)]
    lib.rbd_compress_host.restype = ctypes.c_int
    lib.rbd_compress_host.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _DBL, ctypes.c_int, _I64, _I64,
                                      _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.POINTER(_Result)]
    lib.rbd_compress_resume.restype = ctypes.c_int
    lib.rbd_compress_resume.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _DBL, ctypes.c_int, _I64, _I64, _I64,
                                        _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.c_size_t, _PTR,
                                        ctypes.POINTER(_Result)]
    lib.rbd_compress_noalloc.restype = ctypes.c_int
    lib.rbd_compress_noalloc.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _DBL, ctypes.c_int, _I64, _I64,
                                         _PTR, _I64, _PTR, _I64, _PTR, _PTR, _PTR, _PTR, ctypes.POINTER(_Result)]
    lib.rbd_grad.restype = ctypes.c_int
    lib.rbd_grad.argtypes = [_PTR, ctypes.c_int, _I64, _I64, _I64, _PTR, _I64, _PTR, _I64, _PTR, _I64, _PTR, _I64,
                             _I64, _DBL, _DBL, _PTR, _I64, _PTR, _PTR]
    lib.rbd_grad_batched.restype = ctypes.c_int
    lib.rbd_grad_batched.argtypes = [ctypes.POINTER(_GradItem), _I64, ctypes.c_int, _DBL, _DBL, _PTR]
    lib.rbd_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.rbd_batch_workspace_bytes.argtypes = [ctypes.POINTER(_Instance), _I64, ctypes.c_int]
    lib.rbd_batch_plan_create.restype = ctypes.c_int
    lib.rbd_batch_plan_create.argtypes = [ctypes.POINTER(_PTR), ctypes.POINTER(_Instance), _I64, ctypes.c_int, _PTR,
                                          ctypes.c_size_t, _PTR]
    lib.rbd_batch_run.restype = ctypes.c_int
    lib.rbd_batch_run.argtypes = [_PTR, _PTR, _PTR]
    lib.rbd_batch_tune.restype = ctypes.c_int
    lib.rbd_batch_tune.argtypes = [_PTR, _PTR, _PTR, ctypes.POINTER(_BatchConfig)]
    lib.rbd_batch_plan_config.restype = ctypes.c_int
    lib.rbd_batch_plan_config.argtypes = [_PTR, ctypes.POINTER(_BatchConfig)]
    lib.rbd_batch_plan_set_config.restype = ctypes.c_int
    lib.rbd_batch_plan_set_config.argtypes = [_PTR, ctypes.POINTER(_BatchConfig), _PTR]
    lib.rbd_batch_plan_destroy.restype = ctypes.c_int
    lib.rbd_batch_plan_destroy.argtypes = [_PTR]
    lib.rbd_compress_batched.restype = ctypes.c_int
    lib.rbd_compress_batched.argtypes = [ctypes.POINTER(_Instance), _I64, ctypes.c_int, _PTR, _PTR]
    lib.rbd_reconstruct.restype = ctypes.c_int
    lib.rbd_reconstruct.argtypes = [_PTR, _I64, _I64, _I64, _PTR, _I64, _I64, _PTR, _I64, _PTR]
    lib.rbd_project.restype = ctypes.c_int
    lib.rbd_project.argtypes = [_PTR, _I64, _I64, _I64, _PTR, ctypes.c_int, _I64, _I64, _PTR, _I64, _PTR]
    lib.rbd_set_profiling.restype = None
    lib.rbd_set_profiling.argtypes = [ctypes.c_int]
    lib.rbd_set_wait_limit.restype = ctypes.c_uint64
    lib.rbd_set_wait_limit.argtypes = [ctypes.c_uint64]
    lib.rbd_get_profile.restype = ctypes.c_int
    lib.rbd_get_profile.argtypes = [ctypes.POINTER(_Profile)]
    lib.rbd_status_string.restype = ctypes.c_char_p
    lib.rbd_status_string.argtypes = [ctypes.c_int]
    lib.rbd_version.restype = ctypes.c_int
    lib.rbd_version.argtypes = []
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().rbd_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != 0:
        raise RbdError(status, what)


def _colmajor(x: torch.Tensor, name: str) -> int:
    if x.dim() != 2:
        raise ValueError(f"{name} must be a 2-D (rows x columns) tensor")
    m, n = x.shape
    if x.stride(0) != 1 and m > 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use t().contiguous().t()")
    if n <= 1:
        return max(m, 1)
    if x.stride(1) < m:
        raise ValueError(f"{name}: leading dimension {x.stride(1)} < rows {m}")
    return x.stride(1)


def _stream_ptr(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def colmajor_empty(m: int, n: int, dtype, device) -> torch.Tensor:
    """Uninitialised column-major (m x n) tensor (leading dimension m)."""
    return torch.empty((n, m), dtype=dtype, device=device).t()


def as_colmajor(x: torch.Tensor) -> torch.Tensor:
    """Column-major copy (or view) of a 2-D tensor."""
    return x if x.stride(0) == 1 else x.t().contiguous().t()


@dataclass
class Compressed:
    Y: torch.Tensor        # m x d, column-major, orthonormal columns
    T: torch.Tensor        # d x n, column-major
    pivots: torch.Tensor   # d int64
    err: torch.Tensor      # d FP64, E_cur after each basis
    nu: torch.Tensor       # d FP64, orthogonalised norm of each pivot
    d: int
    next_pivot: int
    stop_reason: str
    err_last: float
    fro_last: float
    x_fro: float
    x_maxcol: float
    launches: int


def workspace_bytes(m: int, n: int, d_max: int, dtype=torch.float64) -> int:
    return int(load().rbd_compress_workspace_bytes(m, n, d_max, DTYPES[dtype]))


def _xt(X: torch.Tensor, accumulate: str) -> int:
    """rbd_dtype of X: its storage type, and for float32 the pass's accumulation ("exact": FP64-grade
    float-float dot products; "fp32": FP32 sums per tile, RBD_F32_ACC32)."""
    if X.dtype not in DTYPES:
        raise ValueError(f"unsupported dtype {X.dtype}")
    if accumulate == "fp32":
        if X.dtype != torch.float32:
            raise ValueError('accumulate="fp32" applies to float32 storage')
        return 3
    if accumulate != "exact":
        raise ValueError(f"unknown accumulate {accumulate!r}")
    return DTYPES[X.dtype]


def compress(X: torch.Tensor, tol: float, d_max: int, start: int = 0, tol_mode: str = "maxcol_abs",
             workspace: Optional[torch.Tensor] = None, weights: Optional[torch.Tensor] = None,
             accumulate: str = "exact") -> Compressed:
    """Algorithm 1 on a column-major CUDA tensor X (m x n) of dtype float64/float32/bfloat16.
    With ``weights`` (m positive float64 values on X's device) the error is measured in the
    A-norm of A = diag(weights) (Section 3.2; rbd_compress_weighted).  ``accumulate="fp32"``
    (float32 X only) sums the pass's products in FP32 per tile (RBD_F32_ACC32)."""
    lib = load()
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor (use compress_host for host arrays)")
    xt = _xt(X, accumulate)
    m, n = X.shape
    ldx = _colmajor(X, "X")
    dev = X.device
    if weights is not None:
        if (not weights.is_cuda or weights.device != dev or weights.dtype != torch.float64
                or weights.numel() != m or not weights.is_contiguous()):
            raise ValueError("weights must be a contiguous float64 CUDA tensor of m entries on X's device")
    Y = colmajor_empty(m, d_max, torch.float64, dev)
    T = colmajor_empty(d_max, n, torch.float64, dev)
    piv = torch.empty(d_max, dtype=torch.int64, device=dev)
    err = torch.empty(d_max, dtype=torch.float64, device=dev)
    nu = torch.empty(d_max, dtype=torch.float64, device=dev)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    res = _Result()
    with torch.cuda.device(dev):
        if weights is None:
            st = lib.rbd_compress(X.data_ptr(), xt, m, n, ldx, float(tol), TOL_MODES[tol_mode],
                                  int(d_max), int(start), Y.data_ptr(), m, T.data_ptr(), d_max, piv.data_ptr(),
                                  err.data_ptr(), nu.data_ptr(), ws_ptr, ws_bytes, _stream_ptr(dev),
                                  ctypes.byref(res))
        else:
            st = lib.rbd_compress_weighted(X.data_ptr(), xt, m, n, ldx, weights.data_ptr(), float(tol),
                                           TOL_MODES[tol_mode], int(d_max), int(start), Y.data_ptr(), m,
                                           T.data_ptr(), d_max, piv.data_ptr(), err.data_ptr(), nu.data_ptr(),
                                           ws_ptr, ws_bytes, _stream_ptr(dev), ctypes.byref(res))
    _check(st, "rbd_compress" if weights is None else "rbd_compress_weighted")
    d = int(res.d)
    return Compressed(Y[:, :d], T[:d, :], piv[:d], err[:d], nu[:d], d, int(res.next_pivot),
                      STOP_REASONS.get(int(res.stop_reason), "?"), float(res.err_last), float(res.fro_last),
                      float(res.x_fro), float(res.x_maxcol), int(res.launches))


def compress_rows(X: torch.Tensor, tol: float, d_max: int, start: int = 0, tol_mode: str = "maxcol_abs") -> Compressed:
    """rbd_compress_rows: Algorithm 1 on the ROWS of the column-major CUDA tensor X (m x n), i.e.
    the compression of X' (the row space of Section 3.1).  Y is n x d, T is d x m, pivots are rows."""
    lib = load()
    if not X.is_cuda or X.dtype not in DTYPES:
        raise ValueError("X must be a CUDA tensor of a supported dtype")
    m, n = X.shape
    ldx = _colmajor(X, "X")
    dev = X.device
    Y = colmajor_empty(n, d_max, torch.float64, dev)
    T = colmajor_empty(d_max, m, torch.float64, dev)
    piv = torch.empty(d_max, dtype=torch.int64, device=dev)
    err = torch.empty(d_max, dtype=torch.float64, device=dev)
    nu = torch.empty(d_max, dtype=torch.float64, device=dev)
    res = _Result()
    with torch.cuda.device(dev):
        st = lib.rbd_compress_rows(X.data_ptr(), DTYPES[X.dtype], m, n, ldx, float(tol), TOL_MODES[tol_mode],
                                   int(d_max), int(start), Y.data_ptr(), n, T.data_ptr(), d_max, piv.data_ptr(),
                                   err.data_ptr(), nu.data_ptr(), _stream_ptr(dev), ctypes.byref(res))
    _check(st, "rbd_compress_rows")
    d = int(res.d)
    return Compressed(Y[:, :d], T[:d, :], piv[:d], err[:d], nu[:d], d, int(res.next_pivot),
                      STOP_REASONS.get(int(res.stop_reason), "?"), float(res.err_last), float(res.fro_last),
                      float(res.x_fro), float(res.x_maxcol), int(res.launches))


def compress_resume(X: torch.Tensor, prev: Compressed, tol: float, d_max: int, tol_mode: str = "maxcol_abs",
                    workspace: Optional[torch.Tensor] = None) -> Compressed:
    """rbd_compress_resume: continue the compression ``prev`` of X (same X, tolerance and mode) to
    a larger d_max; the result equals one compress call with that d_max."""
    lib = load()
    if not X.is_cuda or X.dtype not in DTYPES:
        raise ValueError("X must be a CUDA tensor of a supported dtype")
    m, n = X.shape
    ldx = _colmajor(X, "X")
    d0 = prev.d
    if d0 < 1 or d_max < d0:
        raise ValueError("need 1 <= prev.d <= d_max")
    dev = X.device
    Y = colmajor_empty(m, d_max, torch.float64, dev)
    T = colmajor_empty(d_max, n, torch.float64, dev)
    piv = torch.empty(d_max, dtype=torch.int64, device=dev)
    err = torch.empty(d_max, dtype=torch.float64, device=dev)
    nu = torch.empty(d_max, dtype=torch.float64, device=dev)
    Y[:, :d0].copy_(prev.Y)
    T[:d0, :].copy_(prev.T)
    piv[:d0].copy_(prev.pivots)
    err[:d0].copy_(prev.err)
    nu[:d0].copy_(prev.nu)
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    res = _Result()
    with torch.cuda.device(dev):
        st = lib.rbd_compress_resume(X.data_ptr(), DTYPES[X.dtype], m, n, ldx, float(tol), TOL_MODES[tol_mode], d0,
                                     int(prev.next_pivot), int(d_max), Y.data_ptr(), m, T.data_ptr(), d_max,
                                     piv.data_ptr(), err.data_ptr(), nu.data_ptr(), ws_ptr, ws_bytes,
                                     _stream_ptr(dev), ctypes.byref(res))
    _check(st, "rbd_compress_resume")
    d = int(res.d)
    return Compressed(Y[:, :d], T[:d, :], piv[:d], err[:d], nu[:d], d, int(res.next_pivot),
                      STOP_REASONS.get(int(res.stop_reason), "?"), float(res.err_last), float(res.fro_last),
                      float(res.x_fro), float(res.x_maxcol), int(res.launches))


def compress_noalloc(X: torch.Tensor, tol: float, d_max: int, start: int = 0, tol_mode: str = "maxcol_abs",
                     out: Optional[dict] = None) -> Compressed:
    """rbd_compress_noalloc: ``compress`` with the library's fixed device workspace.  Pass the
    outputs preallocated in ``out`` (column-major CUDA tensors Y, T and vectors pivots, err, nu
    on X's device) to keep the whole call free of allocations."""
    lib = load()
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor")
    if X.dtype not in DTYPES:
        raise ValueError(f"unsupported dtype {X.dtype}")
    m, n = X.shape
    ldx = _colmajor(X, "X")
    dev = X.device
    if out is None:
        out = {"Y": colmajor_empty(m, d_max, torch.float64, dev), "T": colmajor_empty(d_max, n, torch.float64, dev),
               "pivots": torch.empty(d_max, dtype=torch.int64, device=dev),
               "err": torch.empty(d_max, dtype=torch.float64, device=dev),
               "nu": torch.empty(d_max, dtype=torch.float64, device=dev)}
    Y, T, piv, err, nu = out["Y"], out["T"], out["pivots"], out["err"], out["nu"]
    res = _Result()
    with torch.cuda.device(dev):
        st = lib.rbd_compress_noalloc(X.data_ptr(), DTYPES[X.dtype], m, n, ldx, float(tol), TOL_MODES[tol_mode],
                                      int(d_max), int(start), Y.data_ptr(), _colmajor(Y, "Y"), T.data_ptr(),
                                      _colmajor(T, "T"), piv.data_ptr(), err.data_ptr(), nu.data_ptr(),
                                      _stream_ptr(dev), ctypes.byref(res))
    _check(st, "rbd_compress_noalloc")
    d = int(res.d)
    return Compressed(Y[:, :d], T[:d, :], piv[:d], err[:d], nu[:d], d, int(res.next_pivot),
                      STOP_REASONS.get(int(res.stop_reason), "?"), float(res.err_last), float(res.fro_last),
                      float(res.x_fro), float(res.x_maxcol), int(res.launches))


def compress_host(X: torch.Tensor, tol: float, d_max: int, start: int = 0, tol_mode: str = "maxcol_abs",
                  device: Optional[torch.device] = None, out: Optional[dict] = None) -> Compressed:
    """rbd_compress_host on a column-major CPU tensor (pinned memory makes the copies DMA).
    ``out`` may hold preallocated (pinned) CPU outputs Y, T, pivots, err, nu."""
    lib = load()
    if X.is_cuda:
        raise ValueError("compress_host takes a CPU tensor")
    m, n = X.shape
    ldx = _colmajor(X, "X")
    if out is None:
        out = {"Y": colmajor_empty(m, d_max, torch.float64, "cpu"),
               "T": colmajor_empty(d_max, n, torch.float64, "cpu"),
               "pivots": torch.empty(d_max, dtype=torch.int64), "err": torch.empty(d_max, dtype=torch.float64),
               "nu": torch.empty(d_max, dtype=torch.float64)}
    Y, T, piv, err, nu = out["Y"], out["T"], out["pivots"], out["err"], out["nu"]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    res = _Result()
    with torch.cuda.device(dev):
        st = lib.rbd_compress_host(X.data_ptr(), DTYPES[X.dtype], m, n, ldx, float(tol), TOL_MODES[tol_mode],
                                   int(d_max), int(start), Y.data_ptr(), Y.stride(1), T.data_ptr(), T.stride(1),
                                   piv.data_ptr(), err.data_ptr(), nu.data_ptr(), _stream_ptr(dev),
                                   ctypes.byref(res))
    _check(st, "rbd_compress_host")
    d = int(res.d)
    return Compressed(Y[:, :d], T[:d, :], piv[:d], err[:d], nu[:d], d, int(res.next_pivot),
                      STOP_REASONS.get(int(res.stop_reason), "?"), float(res.err_last), float(res.fro_last),
                      float(res.x_fro), float(res.x_maxcol), int(res.launches))


def grad(X: torch.Tensor, Y: torch.Tensor, T: torch.Tensor, pivots: torch.Tensor, Xo: Optional[torch.Tensor] = None,
         w_rec: float = 1.0, w_proj: float = 1.0, need_grad: bool = True):
    """rbd_grad: L = w_rec ||X - Y T||_F^2 + w_proj ||Y' Xo||_F^2 for the fixed pivot set of a
    compression, and (need_grad) its gradient with respect to X.  Returns (G or None, loss) with
    G an m x n column-major FP64 CUDA tensor and loss a 0-dim FP64 CUDA tensor."""
    lib = load()
    if not X.is_cuda or X.dtype not in DTYPES:
        raise ValueError("X must be a CUDA tensor of a supported dtype")
    m, n = X.shape
    ldx = _colmajor(X, "X")
    d = int(pivots.numel())
    dev = X.device
    if d > 0:
        if Y.dtype != torch.float64 or T.dtype != torch.float64:
            raise ValueError("Y and T must be float64")
        ldy, ldt = _colmajor(Y, "Y"), _colmajor(T, "T")
        piv = pivots.to(device=dev, dtype=torch.int64).contiguous()
    else:
        ldy, ldt, piv = m, 1, None
    k, ldxo, xo_ptr = 0, m, None
    if Xo is not None and Xo.numel() > 0:
        if Xo.dtype != X.dtype:
            raise ValueError("Xo must have the dtype of X")
        if Xo.dim() == 1:
            Xo = Xo[:, None]
        k = Xo.shape[1]
        ldxo = _colmajor(Xo, "Xo")
        xo_ptr = Xo.data_ptr()
    G = colmajor_empty(m, n, torch.float64, dev) if need_grad else None
    loss = torch.empty((), dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        st = lib.rbd_grad(X.data_ptr(), DTYPES[X.dtype], m, n, ldx, Y.data_ptr() if d > 0 else None, ldy,
                          T.data_ptr() if d > 0 else None, ldt, piv.data_ptr() if d > 0 else None, d, xo_ptr, k,
                          ldxo, float(w_rec), float(w_proj), G.data_ptr() if G is not None else None, m,
                          loss.data_ptr(), _stream_ptr(dev))
    _check(st, "rbd_grad")
    return G, loss


def grad_batched(items, w_rec: float = 1.0, w_proj: float = 1.0, need_grad: bool = True):
    """rbd_grad_batched: ``grad`` for a list of instances in one set of launches.  Each item is a dict
    with X, Y, T, pivots and optionally Xo (all CUDA tensors on one device, X and Xo of one storage
    type); returns a list of (G or None, loss) as ``grad`` would for each item."""
    lib = load()
    if not items:
        return []
    dev = items[0]["X"].device
    xdt = items[0]["X"].dtype
    arr = (_GradItem * len(items))()
    keep, outs = [], []
    for i, it in enumerate(items):
        X = it["X"]
        if not X.is_cuda or X.dtype != xdt or X.device != dev:
            raise ValueError("every X must be a CUDA tensor of one dtype on one device")
        m, n = X.shape
        ldx = _colmajor(X, "X")
        d = int(it["pivots"].numel())
        Y, T = it["Y"], it["T"]
        if d > 0:
            if Y.dtype != torch.float64 or T.dtype != torch.float64:
                raise ValueError("Y and T must be float64")
            ldy, ldt = _colmajor(Y, "Y"), _colmajor(T, "T")
            piv = it["pivots"].to(device=dev, dtype=torch.int64).contiguous()
        else:
            ldy, ldt, piv = m, 1, None
        Xo = it.get("Xo")
        k, ldxo, xo_ptr = 0, m, None
        if Xo is not None and Xo.numel() > 0:
            if Xo.dtype != xdt:
                raise ValueError("Xo must have the dtype of X")
            if Xo.dim() == 1:
                Xo = Xo[:, None]
            k, ldxo, xo_ptr = Xo.shape[1], _colmajor(Xo, "Xo"), Xo.data_ptr()
        G = colmajor_empty(m, n, torch.float64, dev) if need_grad else None
        loss = torch.empty((), dtype=torch.float64, device=dev)
        keep += [piv, Xo]
        outs.append((G, loss))
        arr[i] = _GradItem(X.data_ptr(), m, n, ldx, Y.data_ptr() if d > 0 else None, ldy,
                           T.data_ptr() if d > 0 else None, ldt, piv.data_ptr() if d > 0 else None, d, xo_ptr, k, ldxo,
                           G.data_ptr() if G is not None else None, m, loss.data_ptr())
    with torch.cuda.device(dev):
        st = lib.rbd_grad_batched(arr, len(items), DTYPES[xdt], float(w_rec), float(w_proj), _stream_ptr(dev))
    _check(st, "rbd_grad_batched")
    return outs


def reconstruct(Y: torch.Tensor, T: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Uncompress (Section 3.1): Xr = Y T for column-major FP64 CUDA tensors Y (m x d) and T (d x n),
    or Y c for a vector c."""
    lib = load()
    if Y.dtype != torch.float64 or T.dtype != torch.float64 or not Y.is_cuda or not T.is_cuda:
        raise ValueError("Y and T must be CUDA float64 tensors")
    if T.dim() == 1:
        T = T[:, None]
    m, d = Y.shape
    if T.shape[0] != d:
        raise ValueError("T must have d rows")
    n = T.shape[1]
    ldy = _colmajor(Y, "Y") if d > 0 else m
    ldt = _colmajor(T, "T") if d > 0 else 1
    Xr = colmajor_empty(m, n, torch.float64, Y.device) if out is None else out
    with torch.cuda.device(Y.device):
        st = lib.rbd_reconstruct(Y.data_ptr() if d > 0 else None, m, d, ldy, T.data_ptr() if d > 0 else None, n,
                                 ldt, Xr.data_ptr(), _colmajor(Xr, "out"), _stream_ptr(Y.device))
    _check(st, "rbd_reconstruct")
    return Xr


def project(Y: torch.Tensor, V: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Out-of-sample map C = Y' V (Section 3.1) for column-major CUDA tensors Y (m x d, FP64)
    and V (m x k)."""
    lib = load()
    if Y.dtype != torch.float64 or not Y.is_cuda or not V.is_cuda:
        raise ValueError("Y must be a CUDA float64 tensor and V a CUDA tensor")
    if V.dim() == 1:
        V = V[:, None]
    m, d = Y.shape
    if V.shape[0] != m:
        raise ValueError("Y and V must have the same number of rows")
    k = V.shape[1]
    ldy = _colmajor(Y, "Y")
    ldv = _colmajor(V, "V")
    C = colmajor_empty(d, k, torch.float64, Y.device) if out is None else out
    ldc = _colmajor(C, "out") if d > 0 and k > 0 else max(d, 1)
    with torch.cuda.device(Y.device):
        st = lib.rbd_project(Y.data_ptr(), m, d, ldy, V.data_ptr(), DTYPES[V.dtype], k, ldv, C.data_ptr(),
                             ldc, _stream_ptr(Y.device))
    _check(st, "rbd_project")
    return C


def set_profiling(enabled: bool):
    load().rbd_set_profiling(1 if enabled else 0)


def set_wait_limit(ns: int) -> int:
    """Bound (nanoseconds) on every device-side wait of the persistent kernels launched from now
    on; 0 restores the defaults.  Returns the previous setting."""
    return int(load().rbd_set_wait_limit(int(ns)))


def get_profile() -> dict:
    p = _Profile()
    _check(load().rbd_get_profile(ctypes.byref(p)), "rbd_get_profile")
    return {f: getattr(p, f) for f, _ in _Profile._fields_}


def version() -> int:
    return int(load().rbd_version())


class BatchPlan:
    """The batched form: many column-major CUDA matrices of one dtype (float64 or float32), each
    with its own tolerance, mode, d_max and start column, compressed in one persistent launch.

    ``items`` is a list of dicts {X, tol, d_max, tol_mode="maxcol_abs", start=0, d_hint=0}; d_hint,
    the expected number of bases, only orders the queue and sizes teams of CTAs.  The plan owns the
    outputs (per matrix Y, T, pivots, err, nu), the workspace and the device result array.
    ``run()`` only enqueues work on the current stream (capturable in a CUDA graph);
    ``results()`` synchronises and returns the per-matrix summaries; ``compressed(i)`` the outputs
    of matrix i trimmed to its d."""

    def __init__(self, items, device=None):
        lib = load()
        if not items:
            raise ValueError("empty batch")
        X0 = items[0]["X"]
        self.dtype = X0.dtype
        if self.dtype not in (torch.float64, torch.float32):
            raise ValueError("the batched form takes float64 or float32 matrices")
        self.device = torch.device(device) if device is not None else X0.device
        self.items = items
        self.out = []
        inst = (_Instance * len(items))()
        for i, it in enumerate(items):
            X = it["X"]
            if X.dtype != self.dtype or X.device != self.device:
                raise ValueError("all matrices must share dtype and device")
            m, n = X.shape
            ldx = _colmajor(X, "X")
            d_max = int(it["d_max"])
            o = {"Y": colmajor_empty(m, d_max, torch.float64, self.device),
                 "T": colmajor_empty(d_max, n, torch.float64, self.device),
                 "pivots": torch.empty(d_max, dtype=torch.int64, device=self.device),
                 "err": torch.empty(d_max, dtype=torch.float64, device=self.device),
                 "nu": torch.empty(d_max, dtype=torch.float64, device=self.device)}
            self.out.append(o)
            inst[i] = _Instance(X.data_ptr(), m, n, ldx, float(it.get("tol", 0.0)),
                                TOL_MODES[it.get("tol_mode", "maxcol_abs")], int(it.get("d_hint", 0)), d_max,
                                int(it.get("start", 0)),
                                o["Y"].data_ptr(), m, o["T"].data_ptr(), d_max, o["pivots"].data_ptr(),
                                o["err"].data_ptr(), o["nu"].data_ptr())
        self._inst = inst
        count = len(items)
        nbytes = int(lib.rbd_batch_workspace_bytes(inst, count, DTYPES[self.dtype]))
        if nbytes == 0:
            # an invalid or unsupported descriptor: plan creation reports which
            plan = _PTR()
            _check(lib.rbd_batch_plan_create(ctypes.byref(plan), inst, count, DTYPES[self.dtype], None, 0,
                                             _stream_ptr(self.device)), "rbd_batch_plan_create")
            raise RbdError(1, "rbd_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = self.workspace.data_ptr() + off
        self._ws_bytes = nbytes
        self.res = torch.zeros(count * _BATCH_RESULT_BYTES, dtype=torch.uint8, device=self.device)
        plan = _PTR()
        with torch.cuda.device(self.device):
            st = lib.rbd_batch_plan_create(ctypes.byref(plan), inst, count, DTYPES[self.dtype], self._ws_ptr,
                                           self._ws_bytes, _stream_ptr(self.device))
        _check(st, "rbd_batch_plan_create")
        self._plan = plan

    def run(self):
        with torch.cuda.device(self.device):
            _check(load().rbd_batch_run(self._plan, self.res.data_ptr(), _stream_ptr(self.device)), "rbd_batch_run")

    def tune(self, cache: Optional[str] = None) -> dict:
        """Autotune the launch shape (rbd_batch_tune) and keep it in the plan; returns the choice
        {cols, tile_rows, team_pct, stages} plus "cached": whether it came from `cache`.

        ``cache``: a JSON file of earlier choices keyed by ``bucket()``.  A batch whose bucket is
        there takes the stored shape without timing anything; otherwise the tuner runs and the
        choice is added to the file."""
        import json
        key = self.bucket()
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                cfg = dict(table[key])
                self.set_config(cfg)
                return dict(cfg, cached=True)
        c = _BatchConfig()
        with torch.cuda.device(self.device):
            _check(load().rbd_batch_tune(self._plan, self.res.data_ptr(), _stream_ptr(self.device), ctypes.byref(c)),
                   "rbd_batch_tune")
        cfg = {f: int(getattr(c, f)) for f, _ in _BatchConfig._fields_}
        if cache:
            table = {}
            if os.path.exists(cache):
                with open(cache) as f:
                    table = json.load(f)
            table[key] = cfg
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(cfg, cached=False)

    def config(self) -> dict:
        c = _BatchConfig()
        _check(load().rbd_batch_plan_config(self._plan, ctypes.byref(c)), "rbd_batch_plan_config")
        return {f: int(getattr(c, f)) for f, _ in _BatchConfig._fields_}

    def set_config(self, cfg: dict) -> None:
        c = _BatchConfig(int(cfg["cols"]), int(cfg["tile_rows"]), int(cfg["team_pct"]), int(cfg.get("stages", 0)))
        with torch.cuda.device(self.device):
            _check(load().rbd_batch_plan_set_config(self._plan, ctypes.byref(c), _stream_ptr(self.device)),
                   "rbd_batch_plan_set_config")

    def bucket(self) -> str:
        """The tuning cache's key for this batch: storage type, the GPU's SM count, the batch size
        and the quartiles of rows, columns and d_max (each rounded to a power of two)."""
        import numpy as np

        def q(v):
            return [int(2 ** round(np.log2(max(1, x)))) for x in np.percentile(v, [25, 50, 75])]
        ms = [it["X"].shape[0] for it in self.items]
        ns = [it["X"].shape[1] for it in self.items]
        ds = [int(it.get("d_hint") or it["d_max"]) for it in self.items]
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        return (f"{'f64' if self.dtype == torch.float64 else 'f32'}/sm{sms}/count{2 ** round(np.log2(len(ms)))}"
                f"/m{q(ms)}/n{q(ns)}/d{q(ds)}").replace(" ", "")

    def results(self) -> list:
        import numpy as np
        raw = self.res.cpu().numpy()
        rec = np.dtype([("d", "<i8"), ("next_pivot", "<i8"), ("stop_reason", "<i4"), ("status", "<i4"),
                        ("err_last", "<f8"), ("fro_last", "<f8"), ("x_fro", "<f8"), ("x_maxcol", "<f8")])
        arr = raw.view(rec)
        return [{k: arr[i][k].item() for k in rec.names} for i in range(len(self.items))]

    def compressed(self, i: int, res: Optional[dict] = None) -> Compressed:
        r = res if res is not None else self.results()[i]
        o = self.out[i]
        d = int(r["d"])
        return Compressed(o["Y"][:, :d], o["T"][:d, :], o["pivots"][:d], o["err"][:d], o["nu"][:d], d,
                          int(r["next_pivot"]), STOP_REASONS.get(int(r["stop_reason"]), "?"), float(r["err_last"]),
                          float(r["fro_last"]), float(r["x_fro"]), float(r["x_maxcol"]), 2)

    def __del__(self):
        try:
            if getattr(self, "_plan", None):
                load().rbd_batch_plan_destroy(self._plan)
                self._plan = None
        except Exception:
            pass
