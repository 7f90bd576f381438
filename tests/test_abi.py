"""C-ABI checks that need no GPU: the library builds, loads, and exports
every entry point include/*.h declares; argument errors that are caught on
the host before any CUDA call come back as status codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(inc, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(esmf_\w+)\s*\(", txt, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2002_00322_gb300 import build as b
    from paper_2002_00322_gb300 import fock
    b.build()
    return fock.load()


def test_header_lists_the_entry_points():
    names = declared_functions()
    from paper_2002_00322_gb300 import fock
    assert set(fock.EXPORTS) | set(fock.SERVER_EXPORTS) | set(fock.ENERGY_EXPORTS) == set(names)
    assert "esmf_fock_create" in names and "esmf_fock_build" in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_host_side_argument_errors(lib):
    from paper_2002_00322_gb300 import fock
    assert fock.esmf_strerror(0) == "ok"
    assert fock.esmf_strerror(fock.ESMF_ERR_TIMEOUT) == "timed out"
    h = C.c_void_p()
    # NULL basis / NULL out are rejected before touching CUDA
    assert lib.esmf_fock_create(None, 0.0, 0, 0, 0, 0, C.byref(h)) == fock.ESMF_ERR_INVALID_ARG
    b = fock.esmf_basis_t(0, None, None, None, None)
    assert lib.esmf_fock_create(C.byref(b), 0.0, 0, 0, 0, 0, None) == fock.ESMF_ERR_INVALID_ARG
    assert lib.esmf_fock_build(None, 1, None, None, None, None, None, None) == fock.ESMF_ERR_INVALID_ARG
    bb = fock.esmf_basis_t(0, None, None, None, None)
    assert lib.esmf_fock_create_screened(C.byref(bb), 0.0, 7, 0, 0, 0, 0, C.byref(h)) == fock.ESMF_ERR_INVALID_ARG
    assert lib.esmf_energy_gradient(None, 1, 1.0, None, None, None, None, None, None, None) == \
        fock.ESMF_ERR_INVALID_ARG
    assert lib.esmf_gvp_gradient(None, 1, 1.0, None, None, None, 0.0, 0.5, 1.0, None, None, None, None) == \
        fock.ESMF_ERR_INVALID_ARG
    st = fock.esmf_stats_t()
    assert lib.esmf_fock_stats(None, C.byref(st)) == fock.ESMF_ERR_INVALID_ARG
    lib.esmf_fock_destroy(None)
    # server: unknown flag bits, bad slot count and budget are rejected before any CUDA call
    from paper_2002_00322_gb300 import server
    server._lib()
    for args in ((0, 1 << 30, 4, 2, 8), (0, 1 << 30, 0, 2, server.SERVER_BATCH), (0, 0, 4, 2, 1)):
        assert lib.esmf_server_create(*args, C.byref(h)) == fock.ESMF_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", ["exp", "nprim", "coef", "tol", "mode", "prec", "direct_f32x2"])
def test_invalid_basis_rejected(lib, bad):
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W
    w = W.small_random(6, 1, 1)
    b = w.basis
    exps, nprim, coefs = b.exps.copy(), b.nprim.copy(), b.coefs.copy()
    tol, mode, prec = 0.0, 0, 0
    if bad == "exp":
        exps[2] = -1.0
    elif bad == "nprim":
        nprim[1] = fock.MAX_PRIM + 1
    elif bad == "coef":
        coefs[0] = np.nan
    elif bad == "tol":
        tol = -1.0
    elif bad == "mode":
        mode = 7
    elif bad == "prec":
        prec = 9
    elif bad == "direct_f32x2":
        mode, prec = 1, 4
    center = np.ascontiguousarray(b.center)
    cb = fock.esmf_basis_t(b.n, center.ctypes.data_as(C.POINTER(C.c_double)),
                           nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                           exps.ctypes.data_as(C.POINTER(C.c_double)),
                           coefs.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    rc = lib.esmf_fock_create(C.byref(cb), tol, mode, prec, 0, 0, C.byref(h))
    expect = fock.ESMF_ERR_UNSUPPORTED if bad == "direct_f32x2" else fock.ESMF_ERR_INVALID_ARG
    assert rc == expect, (bad, rc, fock.esmf_last_error())
    assert not h.value


@pytest.mark.parametrize("label", [-1, 10])
def test_cartesian_label_outside_s_p_d_rejected(lib, label):
    """esmf_fock_create_cart takes labels 0..9 (s, p_x..p_z, d_xx..d_yz) and
    rejects any other on the host, before any device work."""
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W
    w = W.spd_random(1, 1, 0)
    b = w.basis
    cart = np.ascontiguousarray(b.cart, dtype=np.int32).copy()
    cart[3] = label
    center = np.ascontiguousarray(b.center)
    nprim, exps, coefs = (np.ascontiguousarray(x) for x in (b.nprim, b.exps, b.coefs))
    cb = fock.esmf_basis_t(b.n, center.ctypes.data_as(C.POINTER(C.c_double)),
                           nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                           exps.ctypes.data_as(C.POINTER(C.c_double)),
                           coefs.ctypes.data_as(C.POINTER(C.c_double)))
    h = C.c_void_p()
    rc = lib.esmf_fock_create_cart(C.byref(cb), cart.ctypes.data_as(C.POINTER(C.c_int32)), 0.0, 0, 0, 0, 0,
                                   C.byref(h))
    assert rc == fock.ESMF_ERR_INVALID_ARG, (label, rc)
    assert not h.value


@pytest.mark.parametrize("bad", ["empty", "too_many", "nan_point", "null_points", "ridge_neg", "ridge_nan",
                                 "tol_neg", "budget_neg", "prec", "split"])
def test_thc_arguments_rejected_on_the_host(lib, bad):
    """esmf_fock_create_thc checks the grid, tolerance, ridge, budget and
    precision before any device work: INVALID_ARG, or UNSUPPORTED for the
    split 16-bit precisions."""
    from paper_2002_00322_gb300 import fock
    from paper_2002_00322_gb300 import workloads as W
    w = W.small_random(6, 1, 1)
    b = w.basis
    pts = np.ascontiguousarray(W.thc_grid(b))
    G, tol, ridge, budget, prec = pts.shape[0], 0.0, 1e-8, 0, 0
    ptr = pts.ctypes.data_as(C.POINTER(C.c_double))
    if bad == "empty":
        G = 0
    elif bad == "too_many":
        G = 8193
    elif bad == "nan_point":
        pts[3, 1] = np.nan
    elif bad == "null_points":
        ptr = None
    elif bad == "ridge_neg":
        ridge = -1e-8
    elif bad == "ridge_nan":
        ridge = float("nan")
    elif bad == "tol_neg":
        tol = -1.0
    elif bad == "budget_neg":
        budget = -1
    elif bad == "prec":
        prec = 9
    elif bad == "split":
        prec = 2
    center, nprim, exps, coefs = (np.ascontiguousarray(x) for x in (b.center, b.nprim, b.exps, b.coefs))
    cb = fock.esmf_basis_t(b.n, center.ctypes.data_as(C.POINTER(C.c_double)),
                           nprim.ctypes.data_as(C.POINTER(C.c_int32)),
                           exps.ctypes.data_as(C.POINTER(C.c_double)),
                           coefs.ctypes.data_as(C.POINTER(C.c_double)))
    g = fock.esmf_grid_t(G, ptr)
    h = C.c_void_p()
    rc = lib.esmf_fock_create_thc(C.byref(cb), C.byref(g), tol, ridge, prec, 0, budget, C.byref(h))
    expect = fock.ESMF_ERR_UNSUPPORTED if bad == "split" else fock.ESMF_ERR_INVALID_ARG
    assert rc == expect, (bad, rc, fock.esmf_last_error())
    assert not h.value
