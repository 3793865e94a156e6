"""Parity protocol between the CUDA path and the CPU oracle (test helper).

Selections: the GPU's index sequence is compared with the oracle's step by step.  Where
they differ, the oracle replays the GPU's choices ("forced path"); at every step where
the GPU's pick is not the oracle's own best, the oracle's score of the GPU's pick must
be within SEL_RTOL (relative) of the oracle's best score -- a near-tie that rounding may
decide either way.  Means and variances are then compared along the same path.
"""
from __future__ import annotations

import numpy as np

import oracle

SEL_RTOL = 1e-9      # near-tie margin for selections
VAL_RTOL = 1e-10     # FP64 form: relative tolerance for mean and s2
ADJ_FACTOR = 8.0     # adjudication: GPU error vs long double <= this x the oracle's own
EPS64 = 2.0 ** -53


def cancellation_bound(w, x, idx):
    """Rounding scale of v_n(x) = K(x,x) + g - k^T K^{-1} k (Eq. preds2) in FP64: each
    of its n-term inner products carries errors growing like sqrt(n) eps times the size
    of the terms (about 1 + g), and v_n(x) can be far smaller than that, so the relative
    error of s2 and var is of order sqrt(n) eps (1 + g) / v_n(x)."""
    Xd, Yd = w.X[idx], w.Z[idx]
    v = oracle.pred_derivs(Xd, Yd, x, w.d, w.g)[6]
    return float(np.sqrt(len(idx)) * EPS64 * (1.0 + w.g) / v)


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.maximum(np.abs(b), 1e-300)
    return np.abs(a - b) / den


def check_location(w, t, cand_t, gpu_idx, gpu_mean, gpu_s2, method="alc", val_rtol=VAL_RTOL,
                   sel_rtol=SEL_RTOL, gpu_var=None, start=None):
    """Check one location; returns a dict with the path used and the errors.  With start
    (saved design indices) the design grows from it instead of the n0 nearest."""
    x = w.XX[t]
    ora = oracle.local_design(w.X, w.Z, x, cand_t, w.n0, w.n, w.d, w.g, method, start=start)
    assert ora["status"] == 0, "oracle failed at location %d" % t
    # start design: the n0 nearest in order, or the saved design
    first = cand_t[: w.n0] if start is None else np.asarray(start)
    assert np.array_equal(gpu_idx[: len(first)], first), "start design differs at %d" % t
    info = dict(t=t, forced=False, near_ties=0)
    ref = ora
    if not np.array_equal(ora["idx"], gpu_idx):
        f = oracle.local_design(w.X, w.Z, x, cand_t, w.n0, w.n, w.d, w.g, method, forced=gpu_idx,
                                start=start)
        assert f["status"] == 0, "forced replay failed at location %d" % t
        tr = f["trace"]
        for k in range(tr.shape[0]):
            best_rank, best_s, chosen, chosen_s = tr[k, 0], tr[k, 1], tr[k, 2], tr[k, 3]
            if best_rank != chosen:
                gap = abs(best_s - chosen_s)
                assert gap <= sel_rtol * abs(best_s), (
                    "location %d step %d: GPU chose rank %d (score %.17g), oracle best rank %d "
                    "(score %.17g), relative gap %.3g > %.1g" %
                    (t, k + w.n0, chosen, chosen_s, best_rank, best_s, gap / abs(best_s), sel_rtol))
                info["near_ties"] += 1
        ref = f
        info["forced"] = True
    em = float(rel_err(gpu_mean, ref["mean"]))
    es = float(rel_err(gpu_s2, ref["s2"]))
    info.update(err_mean=em, err_s2=es, ref_mean=ref["mean"], ref_s2=ref["s2"])
    if gpu_var is not None:
        info["err_var"] = float(rel_err(gpu_var, ref["var"]))
    info["ok_vals"] = em <= val_rtol and es <= val_rtol and info.get("err_var", 0.0) <= val_rtol
    info["adjudicated"] = False
    if not info["ok_vals"]:
        # v_n(x) = K(x,x) - k^T K^{-1} k is a cancellation whose sensitivity to one-ulp
        # differences in the correlations grows like |K^{-1}k|^2 eps, so two correct FP64
        # evaluations can differ by more than val_rtol.  Adjudicate against the long-double
        # oracle on the same design: the GPU must be within val_rtol of it, or no less
        # accurate than ADJ_FACTOR times the FP64 oracle's own error, or (s2, var) within
        # the rounding scale of the cancellation itself (cancellation_bound).
        ld = oracle.design_predict(w.X, w.Z, x, gpu_idx, w.d, w.g, long_double=True)
        ok = True
        cb = None
        for k, gv in ((0, gpu_mean), (1, gpu_s2)) + (((2, gpu_var),) if gpu_var is not None else ()):
            rv = (ref["mean"], ref["s2"], ref["var"])[k]
            e_gpu = float(rel_err(gv, ld[k]))
            e_ora = float(rel_err(rv, ld[k]))
            info["adj_%d" % k] = (e_gpu, e_ora)
            good = e_gpu <= val_rtol or e_gpu <= ADJ_FACTOR * max(e_ora, 1e-14)
            if not good and k > 0:
                cb = cancellation_bound(w, x, gpu_idx) if cb is None else cb
                info["cancel_bound"] = cb
                good = e_gpu <= cb
            ok = ok and good
        info["ok_vals"] = ok
        info["adjudicated"] = True
    return info
