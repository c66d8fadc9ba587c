"""The C-ABI library: it builds, loads and exports every entry point include/rbd.h declares;
argument validation returns status codes without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_1503_05947_gb300 as rbd
from paper_1503_05947_gb300 import rbd as rbd_binding
from paper_1503_05947_gb300 import buildlib as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rbd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(rbd_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return rbd.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("rbd_compress", "rbd_compress_host", "rbd_compress_weighted", "rbd_project", "rbd_compress_workspace_bytes",
              "rbd_status_string", "rbd_version", "rbd_set_profiling", "rbd_get_profile"):
        assert f in names, f


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"librbd.so does not export {name}"


def test_library_is_built_for_sm103a(lib):
    # the build passes exactly one -gencode for sm_103a
    assert pkg_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(pkg_build.LIB)


def test_status_strings(lib):
    assert rbd.status_string(0) == "ok"
    assert "NaN" in rbd.status_string(4)
    assert rbd.version() >= 100


def test_workspace_bytes(lib):
    assert lib.rbd_compress_workspace_bytes(0, 5, 1, 0) == 0
    assert lib.rbd_compress_workspace_bytes(5, 5, 6, 0) == 0
    small = lib.rbd_compress_workspace_bytes(1024, 512, 64, 0)
    f32 = lib.rbd_compress_workspace_bytes(1024, 512, 64, 1)
    # FP64 input keeps two FP32 planes (8 bytes/element), FP32 one plane
    assert small >= 1024 * 512 * 8 and f32 >= 1024 * 512 * 4 and small > f32
    assert lib.rbd_compress_workspace_bytes(8192, 8192, 512, 0) >= 8192 * 8192 * 8


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    P = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    res = rbd_binding._Result()

    def call(**kw):
        a = dict(X=P, xt=0, m=8, n=6, ldx=8, tol=0.0, mode=0, d_max=4, start=0, Y=P, ldy=8, T=P, ldt=4,
                 piv=P, err=P)
        a.update(kw)
        return lib.rbd_compress(a["X"], a["xt"], a["m"], a["n"], a["ldx"], a["tol"], a["mode"], a["d_max"],
                                a["start"], a["Y"], a["ldy"], a["T"], a["ldt"], a["piv"], a["err"], None, None, 0,
                                None, ctypes.byref(res))

    assert call(X=None) == 1
    assert call(m=0) == 1
    assert call(ldx=7) == 1
    assert call(d_max=7) == 1          # d_max > min(m, n)
    assert call(d_max=0) == 1
    assert call(start=6) == 1
    assert call(start=-1) == 1
    assert call(tol=-1.0) == 1
    assert call(tol=float("nan")) == 1
    assert call(mode=4) == 1
    assert call(xt=7) == 1
    assert call(ldt=3) == 1
    # the A-norm form: the same checks, plus a NULL or misaligned weight vector
    def wcall(w, **kw):
        a = dict(X=P, m=8, n=6, ldx=8, d_max=4)
        a.update(kw)
        return lib.rbd_compress_weighted(a["X"], 0, a["m"], a["n"], a["ldx"], w, 0.0, 0, a["d_max"], 0, P, 8, P, 4,
                                         P, P, None, None, 0, None, ctypes.byref(res))

    assert wcall(None) == 1
    assert wcall(ctypes.c_void_p(20)) == 1   # not 8-byte aligned
    assert wcall(P, X=None) == 1
    assert wcall(P, d_max=9) == 1
    # the row-space form: start indexes rows, Y is n x d (ldy >= n), T is d x m
    def rcall(**kw):
        a = dict(X=P, m=8, n=6, ldx=8, d_max=4, start=0, ldy=6, ldt=4)
        a.update(kw)
        return lib.rbd_compress_rows(a["X"], 0, a["m"], a["n"], a["ldx"], 0.0, 0, a["d_max"], a["start"], P, a["ldy"],
                                     P, a["ldt"], P, P, None, None, ctypes.byref(res))

    assert rcall(X=None) == 1
    assert rcall(ldx=7) == 1
    assert rcall(start=8) == 1       # start < m (a row)
    assert rcall(ldy=5) == 1         # ldy >= n
    assert rcall(d_max=7) == 1       # d_max <= min(m, n)
    assert lib.rbd_project(P, 0, 2, 1, P, 0, 1, 1, P, 2, None) == 1
    assert lib.rbd_project(P, 4, 2, 3, P, 0, 1, 4, P, 2, None) == 1   # ldy < m
    assert lib.rbd_project(P, 4, 0, 4, P, 0, 1, 4, P, 1, None) == 0   # d = 0: no-op


def test_no_cpu_fallback_in_product_path():
    """The product package never imports the oracle (test infrastructure) or numpy math of
    the method; its only compute entry points go through librbd.so."""
    pkg = os.path.join(ROOT, "paper_1503_05947_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            txt = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, fn


def test_wait_limit_setting_round_trips(lib):
    # host-only: the bound on device-side waits is a process-wide setting (0 = the defaults)
    prev = rbd.set_wait_limit(5000)
    try:
        assert rbd.set_wait_limit(0) == 5000
    finally:
        rbd.set_wait_limit(prev)


def _inst(m, n, d_max, tol=1e-3, mode=1, start=0):
    P = 64  # never dereferenced
    return rbd_binding._Instance(P, m, n, m, tol, mode, 0, d_max, start, P, m, P, d_max, P, P, None)


def test_batched_workspace_and_descriptor_checks(lib):
    """The batched form's workspace query validates every descriptor on the host: an invalid or
    out-of-limit matrix gives 0; the size covers every launch shape and grows with d_max."""
    def ws(*insts, xt=1):
        arr = (rbd_binding._Instance * len(insts))(*insts)
        return lib.rbd_batch_workspace_bytes(arr, len(insts), xt)

    small = ws(_inst(300, 200, 20), _inst(1000, 64, 64))
    assert small >= 4 * (300 * 200 + 1000 * 64)
    assert ws(_inst(300, 200, 40), _inst(1000, 64, 64)) > small
    assert ws(_inst(300, 200, 20), xt=0) > ws(_inst(300, 200, 20), xt=1)   # FP64: two planes
    assert ws(_inst(4097, 64, 8)) == 0       # more than 4096 rows
    assert ws(_inst(600, 600, 513)) == 0     # d_max above 512
    assert ws(_inst(300, 200, 201)) == 0     # d_max > min(m, n)
    assert ws(_inst(300, 200, 20, start=200)) == 0
    assert ws(_inst(300, 200, 20, tol=-1.0)) == 0
    assert ws(_inst(300, 200, 20, mode=7)) == 0
    assert ws(_inst(300, 200, 20), xt=2) == 0  # BF16 is not a batched storage type
    assert lib.rbd_batch_workspace_bytes(None, 1, 1) == 0


def test_adjoint_and_decode_argument_checks(lib):
    P = ctypes.c_void_p(64)
    loss = ctypes.c_void_p(128)
    # rbd_grad: X, m, n, ldx, Y, ldy, T, ldt, pivots, d, Xo, k, ldxo, w_rec, w_proj, G, ldg, loss
    def g(**kw):
        a = dict(X=P, m=8, n=6, ldx=8, ldy=8, ldt=4, d=4, wp=1.0)
        a.update(kw)
        return lib.rbd_grad(a["X"], 0, a["m"], a["n"], a["ldx"], P, a["ldy"], P, a["ldt"], P, a["d"], None, 0,
                            a["m"], 1.0, a["wp"], P, a["m"], loss, None)

    assert g(X=None) == 1
    assert g(ldx=7) == 1
    assert g(d=7) == 1                 # d > min(m, n)
    assert g(ldt=3) == 1               # ldt < d
    assert g(wp=float("nan")) == 1
    assert g(m=300, n=300, ldx=300, ldy=300, ldt=257, d=257) == 6   # d above 256: unsupported
    # rbd_grad_batched: count range and a mix of gradient / loss-only outputs, before device work
    items = (rbd_binding._GradItem * 2)()
    for i, G in enumerate((P, None)):
        items[i] = rbd_binding._GradItem(P, 8, 6, 8, P, 8, P, 4, P, 4, None, 0, 8, G, 8, loss)
    assert lib.rbd_grad_batched(items, 2, 0, 1.0, 1.0, None) == 1
    assert lib.rbd_grad_batched(items, 0, 0, 1.0, 1.0, None) == 1
    assert lib.rbd_grad_batched(items, 70000, 0, 1.0, 1.0, None) == 1
    items[1] = rbd_binding._GradItem(P, 8, 6, 8, P, 8, P, 4, P, 7, None, 0, 8, P, 8, loss)   # d > min(m, n)
    assert lib.rbd_grad_batched(items, 2, 0, 1.0, 1.0, None) == 1
    # rbd_reconstruct: n = 0 is a no-op; bad sizes are rejected
    assert lib.rbd_reconstruct(P, 8, 4, 8, P, 0, 4, P, 8, None) == 0
    assert lib.rbd_reconstruct(P, 0, 4, 8, P, 5, 4, P, 8, None) == 1
    assert lib.rbd_reconstruct(P, 8, 4, 7, P, 5, 4, P, 8, None) == 1   # ldy < m
    assert lib.rbd_reconstruct(P, 8, 4, 8, P, 5, 3, P, 8, None) == 1   # ldt < d
