"""CPU oracle for local approximate GP prediction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or calls it, and it shares no code with them.

The arithmetic lives in ``lagp_oracle.c`` (plain C, FP64, no fused multiply-add),
built here with gcc into two shared libraries: the FP64 oracle and the same source
in long double (an adjudicating reference for rounding questions).  Each wrapper
below cites the passage of Gramacy & Apley (arXiv:1303.0383) that its C function
follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lagp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

ALC, MSPE, NN, MSPE_NODERIV = 0, 1, 2, 3
METHODS = {"alc": ALC, "mspe": MSPE, "nn": NN}
TRACE_W = 7
OK, INVALID, OOM, NOT_PD = 0, -1, -2, -5

_lock = threading.Lock()
_libs: dict = {}


def _lib_path(long_double: bool) -> str:
    return os.path.join(_BUILD, "liblagp_oracle_ld.so" if long_double else "liblagp_oracle.so")


def _gcc(src: str, out: str, long_double: bool) -> list:
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wl,-Bsymbolic", "-o", out, src, "-lm"]
    if long_double:
        cmd.insert(1, "-DLAGP_ORACLE_LONG")
    return cmd


def build(force: bool = False) -> None:
    """Compile both oracle libraries with gcc (FP64 and long double)."""
    os.makedirs(_BUILD, exist_ok=True)
    for ld in (False, True):
        out = _lib_path(ld)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        subprocess.run(_gcc(_SRC, out + ".tmp", ld), check=True)
        os.replace(out + ".tmp", out)


def build_variant(source: str, outdir: str) -> tuple:
    """Compile another version of the oracle source (a test plants mistakes in a copy
    this way) into outdir; returns the FP64 and long-double library paths.  Load them
    with load_variant."""
    os.makedirs(outdir, exist_ok=True)
    src = os.path.join(outdir, "lagp_oracle_variant.c")
    with open(src, "w") as f:
        f.write(source)
    outs = (os.path.join(outdir, "variant.so"), os.path.join(outdir, "variant_ld.so"))
    procs = [subprocess.Popen(_gcc(src, o, ld), stderr=subprocess.PIPE)
             for o, ld in zip(outs, (False, True))]
    for pr in procs:
        _, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("gcc failed on the variant: %s" % err.decode(errors="replace"))
    return outs


def load_variant(path: str):
    """ctypes handle of a library built by build_variant, with the oracle's signatures."""
    return _bind(ctypes.CDLL(path))


def _bind(L):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.orc_knn.argtypes = [P, i64, i32, P, i64, i32, P, P, i32]
    L.orc_local_design.argtypes = [P, P, i64, i32, P, P, i32, i32, i32, f64, f64, i32,
                                   P, P, P, P, P, P]
    L.orc_local_design_adaptive.argtypes = [P, P, i64, i32, P, P, i32, i32, i32, f64, f64,
                                            f64, P, P, P, P, P, P, P]
    L.orc_local_design_start.argtypes = [P, P, i64, i32, P, P, i32, P, i32, i32, f64, f64,
                                         i32, P, P, P, P, P, P]
    L.orc_predict.argtypes = [P, P, i64, i32, P, i64, i32, i32, i32, f64, f64, i32,
                              P, P, P, P, P, P, i32]
    L.orc_full_gp.argtypes = [P, P, i64, i32, P, f64, f64, P, P]
    L.orc_design_predict.argtypes = [P, P, i64, i32, P, P, i32, f64, f64, P]
    L.orc_chol.argtypes = [P, i32, P]
    L.orc_inverse.argtypes = [P, i32, P]
    L.orc_pinv_update.argtypes = [P, i32, P, f64, P]
    L.orc_loglik.argtypes = [P, P, i32, i32, f64, f64, P]
    L.orc_pred_derivs.argtypes = [P, P, i32, i32, P, f64, f64, P]
    L.orc_d2l_conditional.argtypes = [P, f64, i32]
    L.orc_d2l_conditional.restype = f64
    L.orc_alc_forms.argtypes = [P, i32, i32, P, P, f64, f64, P]
    L.orc_corr.argtypes = [P, P, i32, f64]
    L.orc_corr.restype = f64
    L.orc_mle.argtypes = [P, P, i64, i32, P, i32, f64, f64, f64, f64, i32, f64, P, P]
    L.orc_mle_batch.argtypes = [P, P, i64, i32, i64, P, i32, P, f64, f64, f64, i32, f64,
                                P, P, P, i32]
    return L


def _lib(long_double: bool = False):
    with _lock:
        if long_double not in _libs:
            build()
            _libs[long_double] = _bind(ctypes.CDLL(_lib_path(long_double)))
        return _libs[long_double]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str) -> None:
    if st != OK:
        raise RuntimeError("oracle %s failed with status %d" % (what, st))


def knn(X, XX, M: int, nthreads: int = 0, with_d2: bool = False):
    """M nearest design points per location, (d2, index) order (Sec. 3; Sec. 6)."""
    X, XX = _f64(X), _f64(XX)
    N, p = X.shape
    T = XX.shape[0]
    cand = np.empty((T, M), np.int32)
    d2 = np.empty((T, M), np.float64) if with_d2 else None
    _check(_lib().orc_knn(_p(X), N, p, _p(XX), T, M, _p(cand), _p(d2) if with_d2 else None,
                          nthreads), "knn")
    return (cand, d2) if with_d2 else cand


def local_design(X, Z, x, cand, n0: int, n: int, d: float, g: float, method="alc",
                 forced=None, long_double: bool = False, start=None, r_min=None):
    """Greedy local design and predictive equations at one location (Sec. 3; Eqs.
    dxy, mspe, predgp, preds2).  With start (n0 design indices) the design grows from
    that saved design instead of the n0 nearest (Sec. 6).  Returns dict(idx, mean, s2,
    var, trace)."""
    X, Z, x, cand = _f64(X), _f64(Z), _f64(x), _i32(cand)
    if start is not None:
        sz = _i32(start)
        n0 = sz.shape[0]
    N, p = X.shape
    M = cand.shape[0]
    m = METHODS.get(method, method) if isinstance(method, str) else int(method)
    idx = np.empty(n, np.int32)
    out = np.empty(3, np.float64)
    trace = np.full((max(n - n0, 1), TRACE_W), np.nan)
    fz = _i32(forced) if forced is not None else None
    if r_min is not None:  # ALC with the stopping rule of Sec. 6
        n_out = ctypes.c_int32()
        st = _lib(long_double).orc_local_design_adaptive(
            _p(X), _p(Z), N, p, _p(x), _p(cand), M, n0, n, d, g, r_min,
            _p(fz) if fz is not None else None, _p(idx), _p(out[0:]), _p(out[1:]), _p(out[2:]),
            _p(trace), ctypes.byref(n_out))
        k = n_out.value
        return dict(status=st, idx=idx, mean=out[0], s2=out[1], var=out[2], n_out=k,
                    trace=trace[: max(k - n0 + 1, 0)])
    if start is not None:
        st = _lib(long_double).orc_local_design_start(
            _p(X), _p(Z), N, p, _p(x), _p(cand), M, _p(sz), n0, n, d, g, m,
            _p(fz) if fz is not None else None, _p(idx), _p(out[0:]), _p(out[1:]), _p(out[2:]),
            _p(trace))
    else:
        st = _lib(long_double).orc_local_design(
            _p(X), _p(Z), N, p, _p(x), _p(cand), M, n0, n, d, g, m,
            _p(fz) if fz is not None else None, _p(idx), _p(out[0:]), _p(out[1:]), _p(out[2:]),
            _p(trace))
    return dict(status=st, idx=idx, mean=out[0], s2=out[1], var=out[2], trace=trace[: n - n0])


def predict(X, Z, XX, n0: int, n: int, ncand: int, d: float, g: float, method="alc",
            nthreads: int = 0, long_double: bool = False):
    """kNN + local design + predictive equations for every location (Sec. 4)."""
    X, Z, XX = _f64(X), _f64(Z), _f64(XX)
    N, p = X.shape
    T = XX.shape[0]
    m = METHODS[method] if isinstance(method, str) else int(method)
    idx = np.empty((T, n), np.int32)
    mean, s2, var = (np.empty(T) for _ in range(3))
    status = np.empty(T, np.int32)
    cand = np.empty((T, ncand), np.int32)
    _check(_lib(long_double).orc_predict(_p(X), _p(Z), N, p, _p(XX), T, n0, n, ncand, d, g, m,
                                         _p(idx), _p(mean), _p(s2), _p(var), _p(status),
                                         _p(cand), nthreads), "predict")
    return dict(idx=idx, mean=mean, s2=s2, var=var, status=status, cand=cand)


def design_predict(X, Z, x, idx, d: float, g: float, long_double: bool = False):
    """Predictive equations (Eqs. predgp, preds2) at x on the given design indices;
    returns (mean, s2, var)."""
    X, Z, x, idx = _f64(X), _f64(Z), _f64(x), _i32(idx)
    out = np.empty(3)
    _check(_lib(long_double).orc_design_predict(_p(X), _p(Z), X.shape[0], X.shape[1], _p(x),
                                                _p(idx), idx.shape[0], d, g, _p(out)),
           "design_predict")
    return float(out[0]), float(out[1]), float(out[2])


NO_CONV = -9


def mle(X, Z, idx, theta0: float, g: float, tmin: float, tmax: float, maxit: int = 100,
        tol: float = 1e-8, long_double: bool = False):
    """Local maximum-likelihood lengthscale of the design idx (Sec. 4.2 step 3; safeguarded
    Newton on Eqs. dl, d2l); returns (theta, iterations, status)."""
    X, Z, idx = _f64(X), _f64(Z), _i32(idx)
    th, it = ctypes.c_double(), ctypes.c_int32()
    st = _lib(long_double).orc_mle(_p(X), _p(Z), X.shape[0], X.shape[1], _p(idx), idx.shape[0],
                                   theta0, g, tmin, tmax, maxit, tol, ctypes.byref(th),
                                   ctypes.byref(it))
    if st not in (OK, NOT_PD, NO_CONV):
        _check(st, "mle")
    return th.value, it.value, st


def mle_batch(X, Z, idx, theta0, g: float, tmin: float, tmax: float, maxit: int = 100,
              tol: float = 1e-8, nthreads: int = 0):
    """orc_mle for every row of idx (T x n); theta0 scalar or length T.
    Returns dict(theta, iters, status)."""
    X, Z, idx = _f64(X), _f64(Z), _i32(idx)
    T, n = idx.shape
    th0 = _f64(np.broadcast_to(np.asarray(theta0, dtype=np.float64), (T,)))
    th, it, st = np.empty(T), np.empty(T, np.int32), np.empty(T, np.int32)
    _check(_lib().orc_mle_batch(_p(X), _p(Z), X.shape[0], X.shape[1], T, _p(idx), n, _p(th0), g,
                                tmin, tmax, maxit, tol, _p(th), _p(it), _p(st), nthreads),
           "mle_batch")
    return {"theta": th, "iters": it, "status": st}


def full_gp(X, Z, x, d: float, g: float):
    """Full-design GP prediction (Eqs. predgp, preds2 with all N points)."""
    X, Z, x = _f64(X), _f64(Z), _f64(x)
    mean, s2 = np.empty(1), np.empty(1)
    _check(_lib().orc_full_gp(_p(X), _p(Z), X.shape[0], X.shape[1], _p(x), d, g, _p(mean),
                              _p(s2)), "full_gp")
    return float(mean[0]), float(s2[0])


def chol(K):
    K = _f64(K)
    L = np.empty_like(K)
    st = _lib().orc_chol(_p(K), K.shape[0], _p(L))
    return st, L


def inverse(K):
    K = _f64(K)
    Ki = np.empty_like(K)
    _check(_lib().orc_inverse(_p(K), K.shape[0], _p(Ki)), "inverse")
    return Ki


def pinv_update(Kinv, k, kss: float):
    """Partitioned inverse (SM Sec. 1)."""
    Kinv, k = _f64(Kinv), _f64(k)
    j = Kinv.shape[0]
    out = np.empty((j + 1, j + 1))
    _check(_lib().orc_pinv_update(_p(Kinv), j, _p(k), kss, _p(out)), "pinv_update")
    return out


def loglik(Xd, Y, d: float, g: float):
    """(l, l', l'') of Eqs. gpk, dl, d2l (l without its theta-free constant)."""
    Xd, Y = _f64(Xd), _f64(Y)
    out = np.empty(3)
    _check(_lib().orc_loglik(_p(Xd), _p(Y), Xd.shape[0], Xd.shape[1], d, g, _p(out)), "loglik")
    return out


def pred_derivs(Xd, Y, xs, d: float, g: float):
    """mu, dmu, d2mu, V, dV, d2V, v, psi at xs (SM Eqs. dz, d2z, dmu, dV, d2V)."""
    Xd, Y, xs = _f64(Xd), _f64(Y), _f64(xs)
    out = np.empty(8)
    _check(_lib().orc_pred_derivs(_p(Xd), _p(Y), Xd.shape[0], Xd.shape[1], _p(xs), d, g,
                                  _p(out)), "pred_derivs")
    return out


def d2l_conditional(pd, y: float, j: int) -> float:
    """SM Eq. d2lx from the predictive quantities returned by pred_derivs."""
    pd = _f64(pd)
    return float(_lib().orc_d2l_conditional(_p(pd), y, j))


def alc_forms(Xd, x, xc, d: float, g: float):
    """(cov^2/v, Eq. dxy expanded, brute-force v_j(x) - v_{j+1}(x))."""
    Xd, x, xc = _f64(Xd), _f64(x), _f64(xc)
    out = np.empty(3)
    _check(_lib().orc_alc_forms(_p(Xd), Xd.shape[0], Xd.shape[1], _p(x), _p(xc), d, g, _p(out)),
           "alc_forms")
    return out


def corr(a, b, d: float) -> float:
    a, b = _f64(a), _f64(b)
    return float(_lib().orc_corr(_p(a), _p(b), a.shape[0], d))
