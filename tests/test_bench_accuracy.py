"""The benchmark's error-against-the-oracle reports for the batched and served workloads
(bench.batched_accuracy, bench.served_accuracy), on the CPU: the oracle's own answers put in
place of the device's pass with every design the oracle's, and an answer perturbed past the
tolerance is reported as failed (not raised), so the default benchmark line cannot be lost to
its accuracy report."""
from __future__ import annotations

import numpy as np

import bench
import oracle
from paper_1303_0383_gb300 import inputs


def _fill(B, locs, answers, s2_scale=1.0):
    off = np.concatenate([[0], np.cumsum(B.n)])
    idx = np.full(int(B.n.sum()), -1, np.int32)
    mean, s2, var = np.zeros(B.T), np.ones(B.T), np.ones(B.T)
    for t, (_, ora) in zip(locs, answers):
        idx[off[t]:off[t + 1]] = ora["idx"]
        mean[t], s2[t], var[t] = ora["mean"], ora["s2"] * s2_scale, ora["var"]
    return idx, mean, s2, var


def test_batched_accuracy_report():
    B = inputs.batched_uneven(3000)
    empty = _fill(B, [], [])
    first = bench.batched_accuracy(B, *empty)        # every sampled location fails, none raises
    assert first["failed"] == first["locations"] > 0
    key = [k for k in bench._BATCH_ORACLE if k[1] == B.T][0]
    locs, answers = key[2], bench._BATCH_ORACLE[key]
    good = bench.batched_accuracy(B, *_fill(B, locs, answers))
    assert good["failed"] == 0 and good["selection_match_rate"] == 1.0
    assert good["max_rel_err_s2"] == 0.0 and good["adjudicated"] == {}
    bad = bench.batched_accuracy(B, *_fill(B, locs, answers, s2_scale=1.0 + 1e-6))
    assert bad["failed"] == bad["locations"]


def test_served_accuracy_report():
    B = inputs.batched_uneven(1)
    ncand = [1000, 2000, 2000]
    lo, hi = [-2.0, 0.0, 0.0], [2.0, 1.0, 1.0]
    rng = np.random.default_rng(1)
    picked = []
    for k in range(4):
        d, n = k % 3, (50, 100)[k % 2]
        x = rng.uniform(lo[d], hi[d], size=B.designs[d].p)
        W = B.designs[d]
        cand = oracle.knn(W.X, x[None, :], ncand[d])[0]
        o = oracle.local_design(W.X, W.Z, x, cand, W.n0, n, W.d, W.g, "alc")
        picked.append((d, x, n, {q: o[q] for q in ("idx", "mean", "s2", "var")}))
    good = bench.served_accuracy(B.designs, ncand, picked)
    assert good["locations"] == 4 and good["failed"] == 0 and good["selection_match_rate"] == 1.0
    wrong = [(d, x, n, dict(r, idx=r["idx"][::-1].copy())) for d, x, n, r in picked]
    assert bench.served_accuracy(B.designs, ncand, wrong)["failed"] == 4
