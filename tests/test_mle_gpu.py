"""Local maximum-likelihood lengthscales and the stagewise scheme of Sec. 4.2 on the GPU,
against the CPU oracle: each GPU stage is checked with the oracle fed the same inputs
(needs a GPU)."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import cancellation_bound, check_location
from tests.test_parity_gpu import dev

pytestmark = pytest.mark.gpu

THETA_RTOL = 1e-9


def _torch():
    import torch
    return torch


def gpu_mle(w, idx, theta0, tmin, tmax, maxit=100, tol=1e-8):
    torch = _torch()
    T, n = idx.shape
    th = torch.empty(T, dtype=torch.float64, device="cuda")
    it = torch.empty(T, dtype=torch.int32, device="cuda")
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    t0 = theta0 if np.isscalar(theta0) else dev(theta0, torch.float64)
    lagp.lagp_mle_dev(dev(w.X, torch.float64), dev(w.Z, torch.float64), dev(idx, torch.int32), t0,
                      w.g, tmin, tmax, th, it, st, maxit, tol,
                      lagp.workspace(lagp.lagp_mle_workspace_bytes(T, n)))
    torch.cuda.synchronize()
    return th.cpu().numpy(), it.cpu().numpy(), st.cpu().numpy()


def _designs(w, T):
    r = oracle.predict(w.X, w.Z, w.XX[:T], w.n0, w.n, w.ncand, w.d, w.g, "alc")
    assert (r["status"] == 0).all()
    return r["idx"]


@pytest.mark.parametrize("maker", [inputs.tiny_2d, lambda: inputs.random_case(31, 900, 3, 12, 6, 24, 80, d=0.4, g=1e-4)])
def test_mle_matches_oracle(maker):
    w = maker()
    T = min(w.T, 40)
    idx = _designs(w, T)
    th, it, st = gpu_mle(w, idx, w.d, w.d / 100, w.d * 100)
    ref = oracle.mle_batch(w.X, w.Z, idx, w.d, w.g, w.d / 100, w.d * 100)
    assert np.array_equal(st, ref["status"])
    ok = st == 0
    assert ok.all()
    rel = np.abs(th - ref["theta"]) / ref["theta"]
    assert rel.max() <= THETA_RTOL, rel.max()
    assert np.abs(it.astype(int) - ref["iters"]).max() <= 1


def test_mle_boundary_and_per_location_start():
    w = inputs.tiny_2d()
    idx = _designs(w, 16)
    ref = oracle.mle_batch(w.X, w.Z, idx, w.d, w.g, w.d / 100, w.d * 100)
    # an interval ending below every interior maximum: the estimate is its upper end
    tmax = 0.5 * ref["theta"].min()
    th, it, st = gpu_mle(w, idx, 0.5 * tmax, 1e-3, tmax)
    assert (st == 0).all() and (th == tmax).all()
    # per-location starting values converge to the same estimates
    starts = np.linspace(0.1, 3.0, 16)
    th2, it2, st2 = gpu_mle(w, idx, starts, w.d / 100, w.d * 100)
    assert (st2 == 0).all()
    assert (np.abs(th2 - ref["theta"]) / ref["theta"]).max() <= 1e-7


@pytest.mark.parametrize("method", ["alc", "mspe"])
def test_select_with_per_location_theta_matches_oracle(method):
    torch = _torch()
    w = inputs.tiny_2d()
    T = w.T
    thetas = np.random.default_rng(3).uniform(0.2, 1.5, size=T)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    out = {k: torch.empty(T, dtype=torch.float64, device="cuda") for k in ("mean", "s2", "var")}
    idx = torch.empty((T, w.n), dtype=torch.int32, device="cuda")
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    for precision in ("fp64", "mixed"):
        ws = lagp.workspace(lagp.lagp_select_workspace_bytes(T, w.p, w.n, w.ncand, method, precision))
        lagp.lagp_select_theta_dev(dev(w.X, torch.float64), dev(w.Z, torch.float64),
                                   dev(w.XX, torch.float64), dev(cand, torch.int32), w.n0, w.n,
                                   dev(thetas, torch.float64), w.g, method, precision, out["mean"],
                                   out["s2"], out["var"], idx, st, ws)
        torch.cuda.synchronize()
        assert int(st.abs().sum()) == 0
        g = {k: v.cpu().numpy() for k, v in out.items()}
        gi = idx.cpu().numpy()
        for t in range(0, T, 5):
            wt = dataclasses.replace(w, d=float(thetas[t]))
            info = check_location(wt, t, cand[t], gi[t], g["mean"][t], g["s2"][t], method,
                                  gpu_var=g["var"][t])
            assert info["ok_vals"], (precision, info)


def test_design_predict_matches_oracle():
    torch = _torch()
    w = inputs.tiny_2d()
    T = w.T
    idx = _designs(w, T)
    thetas = np.random.default_rng(4).uniform(0.3, 1.2, size=T)
    mean = torch.empty(T, dtype=torch.float64, device="cuda")
    s2, var = torch.empty_like(mean), torch.empty_like(mean)
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    lagp.lagp_design_predict_dev(dev(w.X, torch.float64), dev(w.Z, torch.float64),
                                 dev(w.XX, torch.float64), dev(idx, torch.int32),
                                 dev(thetas, torch.float64), w.g, mean, s2, var, st,
                                 lagp.workspace(lagp.lagp_design_predict_workspace_bytes(T, w.n)))
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    m, s, v = mean.cpu().numpy(), s2.cpu().numpy(), var.cpu().numpy()
    for t in range(T):
        rm, rs, rv = oracle.design_predict(w.X, w.Z, w.XX[t], idx[t], thetas[t], w.g)
        ok = abs(m[t] - rm) <= 1e-10 * abs(rm) and abs(s[t] - rs) <= 1e-10 * rs
        if not ok:  # the cancellation in v_n(x): adjudicate against the long-double oracle
            lm, ls, lv = oracle.design_predict(w.X, w.Z, w.XX[t], idx[t], thetas[t], w.g,
                                               long_double=True)
            e_g, e_o = abs(s[t] - ls) / ls, abs(rs - ls) / ls
            wt = dataclasses.replace(w, d=float(thetas[t]))
            ok = abs(m[t] - lm) <= 1e-10 * abs(lm) and (
                e_g <= 1e-10 or e_g <= 8 * max(e_o, 1e-14) or
                e_g <= cancellation_bound(wt, w.XX[t], idx[t]))
        assert ok, t


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "mixed")])
def test_two_stage_scheme_stage_by_stage(method, precision):
    torch = _torch()
    w = inputs.tiny_2d()
    T, n = w.T, w.n
    tmin, tmax = w.d / 100, w.d * 100
    Xd, Zd, XXd = dev(w.X, torch.float64), dev(w.Z, torch.float64), dev(w.XX, torch.float64)
    r = lagp.predict_stagewise(Xd, Zd, XXd, w.n0, n, w.ncand, w.d, w.g, method, precision, stages=2)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in r.items()}
    assert (g["status"] == 0).all() and (g["mle_status"] == 0).all()
    # the same stages one call at a time, each checked against the oracle on its inputs
    cand = oracle.knn(w.X, w.XX, w.ncand)
    cd = dev(cand, torch.int32)
    mean = torch.empty(T, dtype=torch.float64, device="cuda")
    s2, var = torch.empty_like(mean), torch.empty_like(mean)
    idx = torch.empty((T, n), dtype=torch.int32, device="cuda")
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    ws = lagp.workspace(lagp.lagp_select_workspace_bytes(T, w.p, n, w.ncand, method, precision))
    lagp.lagp_select_dev(Xd, Zd, XXd, cd, w.n0, n, w.d, w.g, method, precision, mean, s2, var, idx,
                         st, ws)
    idx1 = idx.cpu().numpy()
    th1, _, st1 = gpu_mle(w, idx1, w.d, tmin, tmax)
    assert (st1 == 0).all()
    ref1 = oracle.mle_batch(w.X, w.Z, idx1, w.d, w.g, tmin, tmax)
    assert (np.abs(th1 - ref1["theta"]) / ref1["theta"]).max() <= THETA_RTOL
    lagp.lagp_select_theta_dev(Xd, Zd, XXd, cd, w.n0, n, dev(th1, torch.float64), w.g, method,
                               precision, mean, s2, var, idx, st, ws)
    torch.cuda.synchronize()
    idx2 = idx.cpu().numpy()
    assert np.array_equal(idx2, g["idx"])
    for t in range(0, T, 4):  # stage-2 designs: the greedy path at theta = the estimate
        wt = dataclasses.replace(w, d=float(th1[t]))
        info = check_location(wt, t, cand[t], idx2[t], mean[t].item(), s2[t].item(), method)
        assert info["ok_vals"], info
    th2, _, st2 = gpu_mle(w, idx2, th1, tmin, tmax)
    assert np.array_equal(th2, g["theta"])
    ref2 = oracle.mle_batch(w.X, w.Z, idx2, th1, w.g, tmin, tmax)
    assert (np.abs(th2 - ref2["theta"]) / ref2["theta"]).max() <= THETA_RTOL
    for t in range(T):  # the output: predictive equations on the final design at theta2
        rm, rs, rv = oracle.design_predict(w.X, w.Z, w.XX[t], idx2[t], th2[t], w.g)
        assert abs(g["mean"][t] - rm) <= 1e-8 * abs(rm) and abs(g["s2"][t] - rs) <= 1e-7 * rs, t


def test_mle_is_deterministic():
    # every location's arithmetic depends only on its own inputs: two runs over a few
    # thousand locations (designs from the mixed screen) give bitwise-identical estimates
    torch = _torch()
    w = inputs.paper_2d()
    w.XX = np.ascontiguousarray(w.XX[:3000])
    X, Z, XX = dev(w.X, torch.float64), dev(w.Z, torch.float64), dev(w.XX, torch.float64)
    idx = lagp.predict_torch(X, Z, XX, w.n0, w.n, w.ncand, w.d, w.g, "alc", "mixed")["idx"]
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    a = gpu_mle(w, idx, w.d, w.d / 100, w.d * 100)
    b = gpu_mle(w, idx, w.d, w.d / 100, w.d * 100)
    assert (a[2] == 0).all()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
