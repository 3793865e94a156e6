"""Batched uneven problems (lagp_predict_batch_dev) through the C ABI (needs a GPU).

Each location's arithmetic depends only on its own inputs, so every location of a batch
must come out bitwise identical to a uniform call for that location alone."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import check_location

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def make_batch(seed=0, T=60, nmin=5, nmax=40, mmax=300):
    rng = np.random.default_rng(seed)
    ws = [inputs.random_case(seed + 1, 3000, 2, 1, 4, 10, 10, d=0.3, g=1e-6),
          inputs.random_case(seed + 2, 5000, 4, 1, 4, 10, 10, d=0.6, g=1e-6),
          inputs.random_case(seed + 3, 4000, 8, 1, 5, 10, 10, d=1.2, g=1e-4)]
    design_of = rng.integers(0, 3, size=T).astype(np.int32)
    n = np.empty(T, np.int32)
    M = np.empty(T, np.int32)
    XX = np.zeros((T, 8))
    for t in range(T):
        w = ws[design_of[t]]
        n[t] = rng.integers(max(nmin, w.n0), nmax + 1)
        M[t] = rng.integers(n[t], mmax + 1)
        XX[t, : w.p] = rng.uniform(0, 1, size=w.p)
    return ws, design_of, n, M, XX


def run_batch(ws, design_of, n, M, XX, method, precision, flags=0, out=None, XXd=None, wsbuf=None):
    torch = _torch()
    dev = "cuda"
    designs = [dict(X=torch.as_tensor(w.X, device=dev), Z=torch.as_tensor(w.Z, device=dev),
                    n0=w.n0, theta=w.d, g=w.g) for w in ws]
    T = len(n)
    if XXd is None:
        XXd = torch.as_tensor(XX, device=dev)
    if out is None:
        out = dict(mean=torch.empty(T, dtype=torch.float64, device=dev),
                   s2=torch.empty(T, dtype=torch.float64, device=dev),
                   var=torch.empty(T, dtype=torch.float64, device=dev),
                   idx=torch.empty(int(n.sum()), dtype=torch.int32, device=dev),
                   status=torch.empty(T, dtype=torch.int8, device=dev))
    if wsbuf is None:
        wsbuf = lagp.workspace(lagp.lagp_predict_batch_workspace_bytes(designs, design_of, n, M, method,
                                                                       precision))
    lagp.lagp_predict_batch_dev(designs, XXd, design_of, n, M, method, precision, out["mean"],
                                out["s2"], out["var"], out["idx"], out["status"], flags, wsbuf)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return res, designs, out, XXd, wsbuf


def split_idx(idx, n):
    off = np.concatenate([[0], np.cumsum(n)])
    return [idx[off[t]:off[t + 1]] for t in range(len(n))]


def uniform_one(designs, w, x, n, M, method, precision):
    torch = _torch()
    return {k: v.cpu().numpy() for k, v in lagp.predict_torch(
        designs["X"], designs["Z"], torch.as_tensor(x[None, :w.p], device="cuda").contiguous(),
        w.n0, int(n), int(M), w.d, w.g, method, precision).items()}


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed"), ("nn", "fp64")])
def test_batch_equals_uniform_calls_bitwise(method, precision):
    ws, design_of, n, M, XX = make_batch(seed=10, T=45)
    res, designs, _, _, _ = run_batch(ws, design_of, n, M, XX, method, precision)
    assert (res["status"] == 0).all()
    idxs = split_idx(res["idx"], n)
    for t in range(len(n)):
        d = design_of[t]
        u = uniform_one(designs[d], ws[d], XX[t], n[t], M[t], method, precision)
        assert np.array_equal(u["idx"][0], idxs[t]), t
        for k in ("mean", "s2", "var"):
            assert u[k][0] == res[k][t], (t, k)


def test_batch_against_oracle_sample():
    ws, design_of, n, M, XX = make_batch(seed=20, T=30)
    res, _, _, _, _ = run_batch(ws, design_of, n, M, XX, "alc", "mixed")
    idxs = split_idx(res["idx"], n)
    for t in range(0, len(n), 3):
        w = ws[design_of[t]]
        w2 = inputs.Workload(w.name, w.X, w.Z, XX[t:t + 1, : w.p], n0=w.n0, n=int(n[t]),
                             ncand=int(M[t]), d=w.d, g=w.g)
        cand = oracle.knn(w2.X, w2.XX, w2.ncand)[0]
        info = check_location(w2, 0, cand, idxs[t], res["mean"][t], res["s2"][t], "alc",
                              gpu_var=res["var"][t])
        assert info["ok_vals"], info


def test_batch_graph_replay_with_new_inputs_and_tuning():
    torch = _torch()
    ws, design_of, n, M, XX = make_batch(seed=30, T=40)
    ref1, designs, out, XXd, wsbuf = run_batch(ws, design_of, n, M, XX, "alc", "mixed")
    # graph path: first call captures, second replays after the inputs changed in place
    g1, _, _, _, _ = run_batch(ws, design_of, n, M, XX, "alc", "mixed", flags=lagp.LAGP_BATCH_GRAPH,
                               out=out, XXd=XXd, wsbuf=wsbuf)
    for k in ref1:
        assert np.array_equal(g1[k], ref1[k]), k
    XX2 = XX.copy()
    XX2[:, :8] = np.clip(XX2[:, :8] + 0.01, 0, 1)
    XXd.copy_(torch.as_tensor(XX2, device="cuda"))
    g2, _, _, _, _ = run_batch(ws, design_of, n, M, XX2, "alc", "mixed", flags=lagp.LAGP_BATCH_GRAPH,
                               out=out, XXd=XXd, wsbuf=wsbuf)
    ref2, _, _, _, _ = run_batch(ws, design_of, n, M, XX2, "alc", "mixed")
    for k in ref2:
        assert np.array_equal(g2[k], ref2[k]), k
    assert not np.array_equal(ref1["mean"], ref2["mean"])
    # tuning picks a launch shape; outputs are the same whatever it picks
    t1, _, _, _, _ = run_batch(ws, design_of, n, M, XX2, "alc", "mixed", flags=lagp.LAGP_BATCH_TUNE)
    t2, _, _, _, _ = run_batch(ws, design_of, n, M, XX2, "alc", "mixed", flags=lagp.LAGP_BATCH_TUNE)
    for k in ref2:
        assert np.array_equal(t1[k], ref2[k]) and np.array_equal(t2[k], ref2[k]), k
