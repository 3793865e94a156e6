"""The C ABI library builds (nvcc cross-compiles for sm_103a without a GPU), loads,
exports every entry point include/lagp.h declares, and rejects bad arguments on the
host before touching a GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1303_0383_gb300 import lagp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(lagp_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_library_loads_and_exports_every_declared_symbol():
    L = lagp.load()
    names = declared_functions()
    assert len(names) >= 12, names
    for name in names:
        assert hasattr(L, name), "missing export %s" % name


def test_version_and_error_strings():
    assert lagp.lagp_version() >= 100
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10):
        assert lagp.strerror(code) and lagp.strerror(code) != "unknown error code"
    assert lagp.strerror(-99) == "unknown error code"


def _pred_dev(**kw):
    a = dict(X=1, Z=1, N=100, p=2, XX=1, T=10, n0=6, n=20, M=50, theta=0.5, g=1e-6, method=0,
             prec=0, mean=1, s2=1, ws=256, wsb=1 << 20)
    a.update(kw)
    P = ctypes.c_void_p
    return lagp.load().lagp_predict_dev(P(a["X"]), P(a["Z"]), a["N"], a["p"], P(a["XX"]), a["T"],
                                        a["n0"], a["n"], a["M"], a["theta"], a["g"], a["method"],
                                        a["prec"], P(a["mean"]), P(a["s2"]), None, None, None,
                                        P(a["ws"]), a["wsb"], None)


@pytest.mark.parametrize("bad", [
    dict(n=2), dict(n0=0), dict(n0=21), dict(M=19), dict(M=101), dict(p=0), dict(p=9),
    dict(theta=0.0), dict(theta=-1.0), dict(theta=float("nan")), dict(g=-1e-9),
    dict(method=7), dict(prec=5), dict(method=1, n0=2), dict(T=-1), dict(n=300, M=300, N=400),
    dict(M=9000, N=10000), dict(X=0), dict(ws=0), dict(ws=8),
])
def test_invalid_arguments_are_rejected_on_the_host(bad):
    assert _pred_dev(**bad) == lagp.LAGP_ERR_INVALID_ARG


def test_null_design_and_bad_knn_args():
    L = lagp.load()
    P = ctypes.c_void_p
    assert L.lagp_predict(None, None, 1, 6, 20, 50, 0.5, 1e-6, 0, 0, None, None, None, None,
                          None) == lagp.LAGP_ERR_INVALID_ARG
    assert L.lagp_design_destroy(None) == lagp.LAGP_ERR_INVALID_ARG
    out = P()
    assert L.lagp_design_create(None, None, 10, 2, ctypes.byref(out)) == lagp.LAGP_ERR_INVALID_ARG
    assert L.lagp_knn_dev(P(1), 10, 2, P(1), 3, 11, P(1), P(256), 1 << 20, None) == \
        lagp.LAGP_ERR_INVALID_ARG            # ncand > N
    assert L.lagp_knn_dev(P(1), 10, 2, P(1), 3, 5, P(1), P(8), 1 << 20, None) == \
        lagp.LAGP_ERR_INVALID_ARG            # misaligned workspace


def test_batch_arguments_are_checked_on_the_host():
    import ctypes as C
    L = lagp.load()
    designs = (lagp.DesignDesc * 2)(lagp.DesignDesc(1, 1, 1000, 2, 4, 0.5, 1e-6),
                                    lagp.DesignDesc(1, 1, 500, 8, 6, 1.0, 1e-4))
    def call(do, n, m, method=0, precision=0, ldxx=8):
        do, n, m = (np.ascontiguousarray(x, dtype=np.int32) for x in (do, n, m))
        P = C.c_void_p
        return L.lagp_predict_batch_dev(designs, 2, P(1), ldxx, len(n), lagp._hp(do), lagp._hp(n),
                                        lagp._hp(m), method, precision, P(1), P(1), None, None,
                                        None, 0, P(256), 1 << 30, None)
    assert call([0, 1], [10, 5], [50, 40]) == lagp.LAGP_ERR_INVALID_ARG      # n < n0 of design 1
    assert call([0, 2], [10, 10], [50, 40]) == lagp.LAGP_ERR_INVALID_ARG     # design index
    assert call([0, 1], [10, 10], [9, 40]) == lagp.LAGP_ERR_INVALID_ARG      # ncand < n
    assert call([0, 1], [10, 10], [50, 501]) == lagp.LAGP_ERR_INVALID_ARG    # ncand > N
    assert call([0, 1], [10, 300], [50, 400]) == lagp.LAGP_ERR_INVALID_ARG   # n > 256
    assert call([0, 1], [10, 10], [50, 40], ldxx=4) == lagp.LAGP_ERR_INVALID_ARG  # ldxx < p
    assert call([0, 1], [10, 10], [50, 40], method=3) == lagp.LAGP_ERR_INVALID_ARG  # method
    assert call([0, 1], [10, 10], [50, 40], precision=2) == lagp.LAGP_ERR_INVALID_ARG  # precision


def test_server_arguments_are_checked_on_the_host():
    import ctypes as C
    L = lagp.load()
    designs = (lagp.DesignDesc * 1)(lagp.DesignDesc(1, 1, 1000, 2, 4, 0.5, 1e-6))
    out = C.c_void_p()
    bad = [dict(nd=0), dict(nmax=2), dict(nmax=300), dict(ncand=10, nmax=20), dict(ncand=9000),
           dict(max_batch=0), dict(max_slots=0)]
    for b in bad:
        a = dict(nd=1, method=0, precision=1, nmax=64, ncand=400, max_batch=1024, budget=1 << 30,
                 max_slots=2)
        a.update(b)
        assert L.lagp_server_create(designs, a["nd"], a["method"], a["precision"], a["nmax"],
                                    a["ncand"], a["max_batch"], a["budget"], a["max_slots"],
                                    C.byref(out)) == lagp.LAGP_ERR_INVALID_ARG, b
    assert L.lagp_server_destroy(None) == lagp.LAGP_ERR_INVALID_ARG


def test_mle_and_stagewise_entry_points_reject_bad_arguments():
    L = lagp.load()
    P = ctypes.c_void_p
    dummy = ctypes.c_double(0.0)
    d = ctypes.cast(ctypes.pointer(dummy), P)
    bad = [
        # N, p, T, n, theta0, g, tmin, tmax, maxit, tol
        (0, 2, 1, 10, 0.5, 0.0, 0.01, 1.0, 10, 1e-8),
        (100, 9, 1, 10, 0.5, 0.0, 0.01, 1.0, 10, 1e-8),
        (100, 2, 1, 1, 0.5, 0.0, 0.01, 1.0, 10, 1e-8),
        (100, 2, 1, 10, 0.5, 0.0, 0.0, 1.0, 10, 1e-8),
        (100, 2, 1, 10, 0.5, 0.0, 1.0, 1.0, 10, 1e-8),
        (100, 2, 1, 10, 0.5, 0.0, 0.01, 1.0, 0, 1e-8),
        (100, 2, 1, 10, 0.5, 0.0, 0.01, 1.0, 10, 0.0),
        (100, 2, 1, 10, -1.0, 0.0, 0.01, 1.0, 10, 1e-8),
        (100, 2, 1, 10, 0.5, -1.0, 0.01, 1.0, 10, 1e-8),
    ]
    for N, p, T, n, th0, g, tmin, tmax, maxit, tol in bad:
        assert L.lagp_mle_dev(d, d, N, p, T, d, n, th0, None, g, tmin, tmax, maxit, tol, d, None,
                              None, d, 1 << 20, None) == lagp.LAGP_ERR_INVALID_ARG
    # T = 0 is a no-op even without buffers
    assert L.lagp_mle_dev(None, None, 100, 2, 0, None, 10, 0.5, None, 0.0, 0.01, 1.0, 10, 1e-8,
                          None, None, None, None, 0, None) == lagp.LAGP_OK
    # kernel (c) alone: n >= 3, theta > 0
    assert L.lagp_design_predict_dev(d, d, 100, 2, d, 1, d, 2, 0.5, None, 0.0, d, d, None, None, d,
                                     1 << 20, None) == lagp.LAGP_ERR_INVALID_ARG
    assert L.lagp_design_predict_dev(d, d, 100, 2, d, 1, d, 10, 0.0, None, 0.0, d, d, None, None,
                                     d, 1 << 20, None) == lagp.LAGP_ERR_INVALID_ARG
    # per-location theta select: the theta array is required
    assert L.lagp_select_theta_dev(d, d, 100, 2, d, 1, d, 20, 6, 10, None, 0.0, 0, 0, d, d, None,
                                   None, None, d, 1 << 20, None) == lagp.LAGP_ERR_INVALID_ARG
    assert lagp.strerror(-9).startswith("iteration limit")


def test_rescore_count_arguments_on_the_host():
    # the FP64 and NN forms have no screen to re-score: 0, without touching a workspace;
    # the mixed screens need the workspace of their call; bad arguments are refused
    L = lagp.load()
    out = ctypes.c_int64(-1)
    assert L.lagp_select_rescore_count(None, 0, 0, 0, ctypes.byref(out), None) == 0 and out.value == 0
    out.value = -1
    assert L.lagp_select_rescore_count(None, 0, 2, 1, ctypes.byref(out), None) == 0 and out.value == 0
    bad = lagp.LAGP_ERR_INVALID_ARG
    assert L.lagp_select_rescore_count(None, 0, 0, 1, ctypes.byref(out), None) == bad
    assert L.lagp_select_rescore_count(None, 0, 1, 1, ctypes.byref(out), None) == bad
    assert L.lagp_select_rescore_count(None, 0, 7, 0, ctypes.byref(out), None) == bad
    assert L.lagp_select_rescore_count(None, 0, 0, 3, ctypes.byref(out), None) == bad
    assert L.lagp_select_rescore_count(None, 4096, 0, 0, None, None) == bad


def test_dense_form_arguments_on_the_host():
    # the paper's explicit-inverse form shares lagp_select_dev's rules, keeps K_j^{-1} in
    # shared memory (n <= 128) and needs a 256-byte aligned workspace
    L = lagp.load()
    P = ctypes.c_void_p
    d = P(256)

    def call(**kw):
        a = dict(N=100, p=2, T=4, M=50, n0=6, n=20, theta=0.5, g=1e-6, X=d, ws=d)
        a.update(kw)
        return L.lagp_select_dense_dev(a["X"], d, a["N"], a["p"], d, a["T"], d, a["M"], a["n0"],
                                       a["n"], a["theta"], a["g"], d, d, None, None, None,
                                       a["ws"], 1 << 20, None)
    bad = lagp.LAGP_ERR_INVALID_ARG
    assert call(n0=0) == bad and call(n=2) == bad and call(M=19) == bad and call(p=9) == bad
    assert call(theta=0.0) == bad and call(g=-1.0) == bad and call(X=None) == bad
    assert call(ws=P(8)) == bad
    assert call(n=129, M=200, N=300) == lagp.LAGP_ERR_UNSUPPORTED
    # T = 0 does nothing and needs no buffers
    assert L.lagp_select_dense_dev(None, None, 100, 2, None, 0, None, 50, 6, 20, 0.5, 1e-6, None,
                                   None, None, None, None, None, 0, None) == 0


def test_checked_build_compiles_and_identifies_itself():
    # the bounds-checked build (nvcc cross-compiles it here) reports checked = 1, the normal
    # build 0; both before any GPU work (the flag is set before the device is touched)
    from paper_1303_0383_gb300 import build
    for checked, want in ((True, 1), (False, 0)):
        L = ctypes.CDLL(build.build(checked=checked))
        flag = ctypes.c_int32(-1)
        L.lagp_check_take.argtypes = [ctypes.c_void_p] * 5
        L.lagp_check_take(ctypes.byref(flag), None, None, None, None)
        assert flag.value == want
