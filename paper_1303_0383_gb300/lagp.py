"""Thin ctypes binding of liblagp (include/lagp.h): the same entry points, argument
marshalling only.  Every step of the method runs in the library's CUDA kernels; this
module never computes any of it and has no CPU fallback -- if the library cannot be
loaded, importing or calling it raises.

Device entry points take torch CUDA tensors (used only as device memory and for
their stream); host entry points take numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LAGP_OK = 0
LAGP_ERR_INVALID_ARG = -1
LAGP_ERR_OOM = -2
LAGP_ERR_CUDA = -3
LAGP_ERR_TIMEOUT = -4
LAGP_ERR_NOT_PD = -5
LAGP_ERR_NO_DEVICE = -6
LAGP_ERR_UNSUPPORTED = -7
LAGP_ERR_SCRATCH_LIMIT = -8
LAGP_ERR_CANCELLED = -10

LAGP_ALC, LAGP_MSPE, LAGP_NN = 0, 1, 2
LAGP_FP64, LAGP_MIXED = 0, 1
METHODS = {"alc": LAGP_ALC, "mspe": LAGP_MSPE, "nn": LAGP_NN}
PRECISIONS = {"fp64": LAGP_FP64, "mixed": LAGP_MIXED}

_lib = None


class LagpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (code %d)" % (what, strerror(code) if _lib else "?", code))
        self.code = code


def load(path: str | None = None):
    """Load liblagp.so (building it first if it is missing or stale); with the environment
    variable LAGP_CHECKED=1, the checked build liblagp_checked.so instead."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build(checked=os.environ.get("LAGP_CHECKED") == "1")
    if not os.path.exists(path):
        raise ImportError("liblagp.so not found at %s" % path)
    L = ctypes.CDLL(path)
    P, i32, i64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                            ctypes.c_size_t)
    L.lagp_strerror.argtypes = [ctypes.c_int]
    L.lagp_strerror.restype = ctypes.c_char_p
    L.lagp_version.restype = ctypes.c_int
    L.lagp_launch_count.restype = i64
    L.lagp_design_create.argtypes = [P, P, i64, i32, ctypes.POINTER(P)]
    L.lagp_design_destroy.argtypes = [P]
    L.lagp_predict.argtypes = [P, P, i64, i32, i32, i32, f64, f64, i32, i32, P, P, P, P, P]
    L.lagp_knn_workspace_bytes.argtypes = [i64, i64, i32]
    L.lagp_knn_workspace_bytes.restype = sz
    L.lagp_knn_dev.argtypes = [P, i64, i32, P, i64, i32, P, P, sz, P]
    L.lagp_select_workspace_bytes.argtypes = [i64, i32, i32, i32, i32, i32]
    L.lagp_select_workspace_bytes.restype = sz
    L.lagp_select_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, i32, i32, f64, f64, i32, i32,
                                  P, P, P, P, P, P, sz, P]
    L.lagp_check_take.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                  ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.lagp_select_dense_workspace_bytes.argtypes = [i64, i32, i32, i32]
    L.lagp_select_dense_workspace_bytes.restype = sz
    L.lagp_select_dense_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, i32, i32, f64, f64, P, P,
                                        P, P, P, P, sz, P]
    L.lagp_select_rescore_count.argtypes = [P, sz, i32, i32, ctypes.POINTER(i64), P]
    L.lagp_predict_workspace_bytes.argtypes = [i64, i64, i32, i32, i32, i32, i32]
    L.lagp_predict_workspace_bytes.restype = sz
    L.lagp_predict_dev.argtypes = [P, P, i64, i32, P, i64, i32, i32, i32, f64, f64, i32, i32,
                                   P, P, P, P, P, P, sz, P]
    L.lagp_exp_dev.argtypes = [P, P, i64, P]
    L.lagp_server_create.argtypes = [P, i32, i32, i32, i32, i32, i64, sz, i32, ctypes.POINTER(P)]
    L.lagp_server_submit.argtypes = [P, i32, P, i64, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    L.lagp_server_wait.argtypes = [P, ctypes.c_uint64, i32, ctypes.POINTER(i32)]
    L.lagp_server_results.argtypes = [P, ctypes.c_uint64, P, P, P, P, P, ctypes.POINTER(f64)]
    L.lagp_server_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                    ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.lagp_server_destroy.argtypes = [P]
    L.lagp_server_slot_bytes.argtypes = [P, i32, i32, i32, i32, i32, i64]
    L.lagp_server_slot_bytes.restype = sz
    L.lagp_server_cancel.argtypes = [P, ctypes.c_uint64]
    L.lagp_server_inject_error.argtypes = [P, ctypes.c_uint64, i32]
    L.lagp_predict_batch_workspace_bytes.argtypes = [P, i32, i64, P, P, P, i32, i32]
    L.lagp_predict_batch_workspace_bytes.restype = sz
    L.lagp_predict_batch_dev.argtypes = [P, i32, P, i32, i64, P, P, P, i32, i32, P, P, P, P, P,
                                         ctypes.c_uint32, P, sz, P]
    L.lagp_select_dev_noalloc.argtypes = [P, P, i64, i32, P, i64, P, i32, i32, i32, f64, f64,
                                          i32, i32, P, P, P, P, P, P]
    L.lagp_select_adaptive_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, i32, i32, f64, f64,
                                           i32, f64, P, P, P, P, P, P, P, sz, P]
    L.lagp_select_augment_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, P, i32, i32, f64, f64,
                                          i32, i32, P, P, P, P, P, P, sz, P]
    L.lagp_select_theta_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, i32, i32, P, f64, i32,
                                        i32, P, P, P, P, P, P, sz, P]
    L.lagp_mle_workspace_bytes.argtypes = [i64, i32]
    L.lagp_mle_workspace_bytes.restype = sz
    L.lagp_mle_dev.argtypes = [P, P, i64, i32, i64, P, i32, f64, P, f64, f64, f64, i32, f64, P, P,
                               P, P, sz, P]
    L.lagp_design_predict_workspace_bytes.argtypes = [i64, i32]
    L.lagp_design_predict_workspace_bytes.restype = sz
    L.lagp_design_predict_dev.argtypes = [P, P, i64, i32, P, i64, P, i32, f64, P, f64, P, P, P, P,
                                          P, sz, P]
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().lagp_strerror(code).decode()


def _chk(code: int, what: str) -> None:
    if code != LAGP_OK:
        raise LagpError(code, what)


def _m(method) -> int:
    return METHODS[method] if isinstance(method, str) else int(method)


def _pr(precision) -> int:
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def lagp_version() -> int:
    return int(load().lagp_version())


def lagp_launch_count() -> int:
    return int(load().lagp_launch_count())


# ----------------------------------------------------------------- device-buffer API

def _dp(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def lagp_knn_workspace_bytes(N: int, T: int, ncand: int) -> int:
    return int(load().lagp_knn_workspace_bytes(N, T, ncand))


def lagp_select_workspace_bytes(T, p, n, ncand, method="alc", precision="fp64") -> int:
    return int(load().lagp_select_workspace_bytes(T, p, n, ncand, _m(method), _pr(precision)))


def lagp_predict_workspace_bytes(N, T, p, n, ncand, method="alc", precision="fp64") -> int:
    return int(load().lagp_predict_workspace_bytes(N, T, p, n, ncand, _m(method), _pr(precision)))


def workspace(nbytes: int, device=None):
    """A uint8 CUDA tensor usable as library scratch (256-byte aligned by the allocator)."""
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def lagp_knn_dev(X, XX, ncand: int, cand, ws, stream=None) -> None:
    """Kernel (a) on device tensors: X (N,p) f64, XX (T,p) f64 -> cand (T,ncand) int32."""
    N, p = X.shape
    T = XX.shape[0]
    _chk(load().lagp_knn_dev(_dp(X), N, p, _dp(XX), T, ncand, _dp(cand), _dp(ws), ws.numel(),
                             _stream(stream)), "lagp_knn_dev")


def lagp_select_dev(X, Z, XX, cand, n0, n, theta, g, method, precision, mean, s2, var=None,
                    idx=None, status=None, ws=None, stream=None) -> None:
    """Kernels (b)+(c) on device tensors, candidate lists given."""
    N, p = X.shape
    T, M = cand.shape
    _chk(load().lagp_select_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, n0, n, theta, g,
                                _m(method), _pr(precision), _dp(mean), _dp(s2), _dp(var), _dp(idx),
                                _dp(status), _dp(ws), ws.numel(), _stream(stream)),
         "lagp_select_dev")


def lagp_check_take() -> dict:
    """Bounds-check violations recorded since the last call (checked build; zeros otherwise):
    {"checked": 0/1, "count", "site", "index", "bound"} -- waits for the device."""
    c, n, st, i, b = (ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(),
                      ctypes.c_int64())
    _chk(load().lagp_check_take(ctypes.byref(c), ctypes.byref(n), ctypes.byref(st), ctypes.byref(i),
                                ctypes.byref(b)), "lagp_check_take")
    return {"checked": int(c.value), "count": int(n.value), "site": int(st.value),
            "index": int(i.value), "bound": int(b.value)}


def lagp_select_dense_workspace_bytes(T, p, n, ncand) -> int:
    return int(load().lagp_select_dense_workspace_bytes(T, p, n, ncand))


def lagp_select_dense_dev(X, Z, XX, cand, n0, n, theta, g, mean, s2, var=None, idx=None,
                          status=None, ws=None, stream=None) -> None:
    """ALC in the paper's own form (explicit K_j^{-1}, O(j^2) per candidate), FP64, on
    device tensors, candidate lists given; outputs as lagp_select_dev."""
    N, p = X.shape
    T, M = cand.shape
    _chk(load().lagp_select_dense_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, n0, n,
                                      theta, g, _dp(mean), _dp(s2), _dp(var), _dp(idx),
                                      _dp(status), _dp(ws), ws.numel(), _stream(stream)),
         "lagp_select_dense_dev")


def lagp_select_rescore_count(ws, method="alc", precision="mixed", stream=None) -> int:
    """FP64 re-score passes made by the last selection call on workspace ws (mixed screens;
    0 for FP64 and NN)."""
    out = ctypes.c_int64()
    _chk(load().lagp_select_rescore_count(_dp(ws), ws.numel() * ws.element_size(), _m(method),
                                          _pr(precision), ctypes.byref(out), _stream(stream)),
         "lagp_select_rescore_count")
    return int(out.value)


def lagp_exp_dev(x, y, stream=None) -> None:
    """The library's FP64 exponential elementwise (device tensors, float64)."""
    _chk(load().lagp_exp_dev(_dp(x), _dp(y), x.numel(), _stream(stream)), "lagp_exp_dev")


LAGP_BATCH_TUNE, LAGP_BATCH_GRAPH = 1, 2


class DesignDesc(ctypes.Structure):
    """lagp_design_desc: one resident design of a batch (device X, Z)."""
    _fields_ = [("X", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("p", ctypes.c_int32), ("n0", ctypes.c_int32), ("theta", ctypes.c_double),
                ("g", ctypes.c_double)]


def _descs(designs):
    """designs: sequence of dicts with X, Z (CUDA tensors), n0, theta, g."""
    arr = (DesignDesc * len(designs))()
    for i, d in enumerate(designs):
        X, Z = d["X"], d["Z"]
        if not (X.is_cuda and Z.is_cuda and X.is_contiguous() and Z.is_contiguous()):
            raise ValueError("design tensors must be contiguous CUDA tensors")
        arr[i] = DesignDesc(X.data_ptr(), Z.data_ptr(), X.shape[0], X.shape[1], int(d["n0"]),
                            float(d["theta"]), float(d["g"]))
    return arr


def lagp_predict_batch_workspace_bytes(designs, design_of, n, ncand, method="alc",
                                       precision="fp64") -> int:
    a = _descs(designs)
    do, nn, nc = (np.ascontiguousarray(x, dtype=np.int32) for x in (design_of, n, ncand))
    return int(load().lagp_predict_batch_workspace_bytes(a, len(designs), do.shape[0], _hp(do),
                                                         _hp(nn), _hp(nc), _m(method),
                                                         _pr(precision)))


def lagp_predict_batch_dev(designs, XX, design_of, n, ncand, method, precision, mean, s2,
                           var=None, idx=None, status=None, flags=0, ws=None, stream=None) -> None:
    """Batched path: XX is a (T, ldxx) CUDA tensor, design_of/n/ncand host int arrays."""
    a = _descs(designs)
    do, nn, nc = (np.ascontiguousarray(x, dtype=np.int32) for x in (design_of, n, ncand))
    T, ldxx = XX.shape
    _chk(load().lagp_predict_batch_dev(a, len(designs), _dp(XX), ldxx, T, _hp(do), _hp(nn),
                                       _hp(nc), _m(method), _pr(precision), _dp(mean), _dp(s2),
                                       _dp(var), _dp(idx), _dp(status), flags, _dp(ws),
                                       ws.numel(), _stream(stream)), "lagp_predict_batch_dev")


def lagp_server_slot_bytes(designs, method="alc", precision="mixed", nmax=128, ncand_max=2048,
                           max_batch=16384) -> int:
    """Device bytes of one slot of a server created with these arguments."""
    return int(load().lagp_server_slot_bytes(_descs(designs), len(designs), _m(method), _pr(precision),
                                             nmax, ncand_max, max_batch))


class Server:
    """lagp_server_*: continuous-batching serving loop over resident designs."""

    def __init__(self, designs, method="alc", precision="mixed", nmax=128, ncand_max=2048,
                 max_batch=16384, memory_budget=8 << 30, max_slots=4):
        self._designs = designs          # keeps the device tensors alive
        self._descs = _descs(designs)
        self._p = [int(d["X"].shape[1]) for d in designs]
        h = ctypes.c_void_p()
        _chk(load().lagp_server_create(self._descs, len(designs), _m(method), _pr(precision), nmax,
                                       ncand_max, max_batch, memory_budget, max_slots,
                                       ctypes.byref(h)), "lagp_server_create")
        self._h = h
        self._n = {}

    def submit(self, design, XX, n, ncand) -> int:
        XX = np.ascontiguousarray(XX, dtype=np.float64)
        rid = ctypes.c_uint64()
        _chk(load().lagp_server_submit(self._h, design, _hp(XX), XX.shape[0], n, ncand,
                                       ctypes.byref(rid)), "lagp_server_submit")
        self._n[rid.value] = (XX.shape[0], n)
        return rid.value

    def wait(self, rid, timeout_ms=-1) -> bool:
        done = ctypes.c_int32()
        _chk(load().lagp_server_wait(self._h, rid, timeout_ms, ctypes.byref(done)), "lagp_server_wait")
        return bool(done.value)

    def results(self, rid):
        L, n = self._n.pop(rid)
        out = dict(mean=np.empty(L), s2=np.empty(L), var=np.empty(L),
                   idx=np.empty((L, n), np.int32), status=np.empty(L, np.int8))
        lat = ctypes.c_double()
        _chk(load().lagp_server_results(self._h, rid, _hp(out["mean"]), _hp(out["s2"]),
                                        _hp(out["var"]), _hp(out["idx"]), _hp(out["status"]),
                                        ctypes.byref(lat)), "lagp_server_results")
        out["latency_ms"] = lat.value
        return out

    def cancel(self, rid) -> int:
        """Cancels a request (lagp_server_cancel); returns the library's code."""
        return int(load().lagp_server_cancel(self._h, rid))

    def inject_error(self, rid, code) -> int:
        """Test hook: the queued request's batch fails on the host with code."""
        return int(load().lagp_server_inject_error(self._h, rid, code))

    def try_results(self, rid):
        """results(), but a failed or cancelled request gives (code, None) instead of raising."""
        try:
            return 0, self.results(rid)
        except LagpError as e:
            self._n.pop(rid, None)
            return e.code, None

    def stats(self):
        b, l, s, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        code = load().lagp_server_stats(self._h, ctypes.byref(b), ctypes.byref(l), ctypes.byref(s),
                                        ctypes.byref(m))
        return dict(batches=b.value, locations=l.value, slots=s.value, max_inflight=m.value,
                    last_error=code)

    def close(self):
        if self._h is not None and self._h.value:
            _chk(load().lagp_server_destroy(self._h), "lagp_server_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lagp_select_dev_noalloc(X, Z, XX, cand, n0, n, theta, g, method, precision, mean, s2,
                            var=None, idx=None, status=None, stream=None) -> int:
    """Kernels (b)+(c) with the library's static scratch (no workspace, no allocation).
    Returns the library's status code instead of raising, so callers can see
    LAGP_ERR_SCRATCH_LIMIT."""
    N, p = X.shape
    T, M = cand.shape
    return int(load().lagp_select_dev_noalloc(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, n0,
                                              n, theta, g, _m(method), _pr(precision), _dp(mean),
                                              _dp(s2), _dp(var), _dp(idx), _dp(status),
                                              _stream(stream)))


def lagp_predict_dev(X, Z, XX, n0, n, ncand, theta, g, method, precision, mean, s2, var=None,
                     idx=None, status=None, ws=None, stream=None) -> None:
    """The whole path on device tensors."""
    N, p = X.shape
    T = XX.shape[0]
    _chk(load().lagp_predict_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, n0, n, ncand, theta, g,
                                 _m(method), _pr(precision), _dp(mean), _dp(s2), _dp(var), _dp(idx),
                                 _dp(status), _dp(ws), ws.numel(), _stream(stream)),
         "lagp_predict_dev")


# ----------------------------------------------------------------- host-buffer API

def _hp(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Design:
    """A resident design (lagp_design_create / lagp_design_destroy)."""

    def __init__(self, X, Z):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.Z = np.ascontiguousarray(Z, dtype=np.float64)
        self.N, self.p = self.X.shape
        h = ctypes.c_void_p()
        _chk(load().lagp_design_create(_hp(self.X), _hp(self.Z), self.N, self.p, ctypes.byref(h)),
             "lagp_design_create")
        self._h = h

    def close(self):
        if self._h is not None and self._h.value:
            _chk(load().lagp_design_destroy(self._h), "lagp_design_destroy")
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def predict(self, XX, n0, n, ncand, theta, g, method="alc", precision="fp64", out=None):
        """lagp_predict on host arrays; returns dict(mean, s2, var, idx, status)."""
        XX = np.ascontiguousarray(XX, dtype=np.float64)
        T = XX.shape[0]
        if out is None:
            out = dict(mean=np.empty(T), s2=np.empty(T), var=np.empty(T),
                       idx=np.empty((T, n), np.int32), status=np.empty(T, np.int8))
        _chk(load().lagp_predict(self._h, _hp(XX), T, n0, n, ncand, theta, g, _m(method),
                                 _pr(precision), _hp(out["mean"]), _hp(out["s2"]),
                                 _hp(out.get("var")), _hp(out.get("idx")), _hp(out.get("status"))),
             "lagp_predict")
        return out


def predict_torch(X, Z, XX, n0, n, ncand, theta, g, method="alc", precision="fp64"):
    """Convenience: allocate outputs and workspace as torch tensors, run lagp_predict_dev."""
    import torch
    dev = X.device
    T = XX.shape[0]
    mean = torch.empty(T, dtype=torch.float64, device=dev)
    s2 = torch.empty_like(mean)
    var = torch.empty_like(mean)
    idx = torch.empty((T, n), dtype=torch.int32, device=dev)
    status = torch.empty(T, dtype=torch.int8, device=dev)
    ws = workspace(lagp_predict_workspace_bytes(X.shape[0], T, X.shape[1], n, ncand, method,
                                                precision), dev)
    lagp_predict_dev(X, Z, XX, n0, n, ncand, theta, g, method, precision, mean, s2, var, idx,
                     status, ws)
    return dict(mean=mean, s2=s2, var=var, idx=idx, status=status)


# ------------------------------------------------ stagewise scheme (Sec. 4.2), device API

def lagp_select_theta_dev(X, Z, XX, cand, n0, n, theta, g, method, precision, mean, s2, var=None,
                          idx=None, status=None, ws=None, stream=None) -> None:
    """Kernels (b)+(c) with a lengthscale per location: theta is a (T,) float64 tensor."""
    N, p = X.shape
    T, M = cand.shape
    _chk(load().lagp_select_theta_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, n0, n,
                                      _dp(theta), g, _m(method), _pr(precision), _dp(mean),
                                      _dp(s2), _dp(var), _dp(idx), _dp(status), _dp(ws),
                                      ws.numel(), _stream(stream)), "lagp_select_theta_dev")


def lagp_mle_workspace_bytes(T: int, n: int) -> int:
    return int(load().lagp_mle_workspace_bytes(T, n))


def lagp_mle_dev(X, Z, idx, theta0, g, tmin, tmax, theta_out, iters=None, status=None,
                 maxit: int = 100, tol: float = 1e-8, ws=None, stream=None) -> None:
    """Local maximum-likelihood lengthscale of each design (idx (T,n) int32); theta0 a float
    or a (T,) float64 tensor of starting values."""
    N, p = X.shape
    T, n = idx.shape
    th_loc = theta0 if not isinstance(theta0, (int, float)) else None
    th_s = float(theta0) if th_loc is None else 1.0
    _chk(load().lagp_mle_dev(_dp(X), _dp(Z), N, p, T, _dp(idx), n, th_s, _dp(th_loc), g, tmin,
                             tmax, maxit, tol, _dp(theta_out), _dp(iters), _dp(status), _dp(ws),
                             ws.numel(), _stream(stream)), "lagp_mle_dev")


def lagp_design_predict_workspace_bytes(T: int, n: int) -> int:
    return int(load().lagp_design_predict_workspace_bytes(T, n))


def lagp_design_predict_dev(X, Z, XX, idx, theta, g, mean, s2, var=None, status=None, ws=None,
                            stream=None) -> None:
    """Kernel (c) on given designs idx (T,n); theta a float or a (T,) float64 tensor."""
    N, p = X.shape
    T, n = idx.shape
    th_loc = theta if not isinstance(theta, (int, float)) else None
    th_s = float(theta) if th_loc is None else 1.0
    _chk(load().lagp_design_predict_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(idx), n, th_s,
                                        _dp(th_loc), g, _dp(mean), _dp(s2), _dp(var), _dp(status),
                                        _dp(ws), ws.numel(), _stream(stream)),
         "lagp_design_predict_dev")


def predict_stagewise(X, Z, XX, n0, n, ncand, theta0, g, method="alc", precision="fp64",
                      stages: int = 2, tmin=None, tmax=None, maxit: int = 100, tol: float = 1e-8,
                      stream=None):
    """The stagewise scheme of Sec. 4.2 on device tensors, every step in the library's
    kernels: candidates (kernel (a)); design with theta0 (kernels (b)+(c)); local MLE;
    then stages - 1 times: design with the per-location estimates and a fresh MLE; finally
    the predictive equations on the last design with the last estimates.  stages = 1 gives
    the one-stage scheme with local MLE ("alc"/"mspe" rows); stages = 2 the two-stage
    ("alc2"/"mspe2").  tmin/tmax default to theta0/100 and 100 theta0.
    Returns dict(mean, s2, var, idx, theta, iters, status)."""
    import torch
    dev = X.device
    N, p = X.shape
    T = XX.shape[0]
    tmin = theta0 / 100.0 if tmin is None else tmin
    tmax = theta0 * 100.0 if tmax is None else tmax
    f64, i32 = torch.float64, torch.int32
    cand = torch.empty((T, ncand), dtype=i32, device=dev)
    lagp_knn_dev(X, XX, ncand, cand, workspace(lagp_knn_workspace_bytes(N, T, ncand), dev), stream)
    mean = torch.empty(T, dtype=f64, device=dev)
    s2, var = torch.empty_like(mean), torch.empty_like(mean)
    idx = torch.empty((T, n), dtype=i32, device=dev)
    status = torch.empty(T, dtype=torch.int8, device=dev)
    mstatus = torch.empty(T, dtype=torch.int8, device=dev)
    theta = torch.empty(T, dtype=f64, device=dev)
    iters = torch.empty(T, dtype=i32, device=dev)
    ws_sel = workspace(lagp_select_workspace_bytes(T, p, n, ncand, method, precision), dev)
    ws_mle = workspace(lagp_mle_workspace_bytes(T, n), dev)
    lagp_select_dev(X, Z, XX, cand, n0, n, theta0, g, method, precision, mean, s2, var, idx,
                    status, ws_sel, stream)
    lagp_mle_dev(X, Z, idx, theta0, g, tmin, tmax, theta, iters, mstatus, maxit, tol, ws_mle,
                 stream)
    for _ in range(stages - 1):
        # a location without an estimate (its screen failed) keeps theta0
        th1 = torch.where(torch.isfinite(theta), theta, torch.full_like(theta, theta0))
        lagp_select_theta_dev(X, Z, XX, cand, n0, n, th1, g, method, precision, mean, s2, var,
                              idx, status, ws_sel, stream)
        lagp_mle_dev(X, Z, idx, th1, g, tmin, tmax, theta, iters, mstatus, maxit, tol, ws_mle,
                     stream)
    ws_pr = workspace(lagp_design_predict_workspace_bytes(T, n), dev)
    lagp_design_predict_dev(X, Z, XX, idx, theta, g, mean, s2, var, status, ws_pr, stream)
    return dict(mean=mean, s2=s2, var=var, idx=idx, theta=theta, iters=iters, status=status,
                mle_status=mstatus)


def lagp_select_augment_dev(X, Z, XX, cand, start, n, theta, g, method, precision, mean, s2,
                            var=None, idx=None, status=None, ws=None, stream=None) -> None:
    """Kernels (b)+(c) growing saved designs start (T, n1) int32 to n points."""
    N, p = X.shape
    T, M = cand.shape
    n1 = start.shape[1]
    _chk(load().lagp_select_augment_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, _dp(start),
                                        n1, n, theta, g, _m(method), _pr(precision), _dp(mean),
                                        _dp(s2), _dp(var), _dp(idx), _dp(status), _dp(ws),
                                        ws.numel(), _stream(stream)), "lagp_select_augment_dev")


def lagp_select_adaptive_dev(X, Z, XX, cand, n0, n, theta, g, precision, r_min, mean, s2, n_out,
                             var=None, idx=None, status=None, ws=None, stream=None) -> None:
    """ALC designs with the stopping rule of Sec. 6 (sizes into n_out (T,) int32)."""
    N, p = X.shape
    T, M = cand.shape
    _chk(load().lagp_select_adaptive_dev(_dp(X), _dp(Z), N, p, _dp(XX), T, _dp(cand), M, n0, n,
                                         theta, g, _pr(precision), r_min, _dp(mean), _dp(s2),
                                         _dp(var), _dp(idx), _dp(n_out), _dp(status), _dp(ws),
                                         ws.numel(), _stream(stream)), "lagp_select_adaptive_dev")
