"""C-ABI checks that need no GPU: the library loads, exports every function
that include/qbx.h declares, and its host-only functions behave."""
import ctypes
import os
import re

import numpy as np

import paper_1207_4461_gb300 as qbx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(qbx_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    L = qbx.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_version_and_error_string():
    L = qbx.lib()
    assert L.qbx_version() == 1
    assert isinstance(L.qbx_last_error(), bytes)


def test_host_gauss_legendre_matches_numpy():
    for q in (1, 3, 16, 64, 128):
        x, w = qbx.qbx_gauss_legendre(q)
        xn, wn = np.polynomial.legendre.leggauss(q)
        assert np.abs(x - xn).max() < 1e-15
        assert np.abs(w - wn).max() < 1e-14
        assert abs(w.sum() - 2.0) < 1e-14


def test_host_argument_errors_need_no_device():
    L = qbx.lib()
    x = np.zeros(4)
    assert L.qbx_gauss_legendre(0, x.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p)) == 1
    assert L.qbx_gauss_legendre(qbx.MAX_P * 10, None, None) == 1
    h = ctypes.c_void_p()
    assert L.qbx_plan_create(ctypes.byref(h), 0, 0, 64, 0) == 1
    assert b"q_tgt" in L.qbx_last_error()
    assert L.qbx_apply(None, None, 0, 0, 0, qbx.c64(1.0, 0.0), 4, None, 1, 0, None, None, None, None) == 1
    assert b"plan" in L.qbx_last_error()
    assert L.qbx_apply_cfie(None, None, qbx.c64(1.0, 0.0), qbx.c64(1.0, 0.0), 4, None, 1, None, None) == 1
    assert b"plan" in L.qbx_last_error()


def test_workspace_bytes_formula():
    b = qbx.qbx_workspace_bytes(16384, 8192, 2, 1)
    assert b >= 16384 * 16 + 64 * 8192 * 2 * 16
    assert qbx.qbx_workspace_bytes(-1, 1, 1, 1) == 0


def test_shape_adjoint_workspace_bytes():
    """Holds the oversampled density, the centre gradients, coefficient
    columns and 64 splits of both sweeps; 0 for bad arguments."""
    M, p, nrhs = 128, 10, 1
    b = qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, nrhs)
    n_t, n_s = M * 16, M * 64
    assert b >= n_s * 16 + 64 * (2 * n_t) * 4 * 16 + 64 * n_s * 3 * 16
    assert qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, p, 2) > b
    assert qbx.qbx_shape_adjoint_workspace_bytes(0, 16, 64, p, 1) == 0
    assert qbx.qbx_shape_adjoint_workspace_bytes(M, 16, 64, -1, 1) == 0
