"""Parity protocol between the CUDA path and the CPU oracle -- TEST INFRASTRUCTURE ONLY.

Used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``;
the product path never imports it.  One protocol for all three:

Selections.  The GPU's index sequence is compared with the oracle's step by step.  Where
they differ, the oracle replays the GPU's choices ("forced path"); at every step where
the GPU's pick is not the oracle's own best, the oracle's score of the GPU's pick must be
within SEL_RTOL (relative) of the oracle's best score -- a near-tie that rounding may
decide either way (Sec. 3.3 decides ties only by the order of the candidates).  Means and
variances are then compared along the same path.

Values.  mean, s2 and var within VAL_RTOL (relative) of the FP64 oracle.  A value beyond
that is adjudicated against the long-double oracle on the same design; it passes by the
first clause that holds, and the clause is recorded:

  1  within VAL_RTOL of the long-double value;
  2  no less accurate than ADJ_FACTOR times the FP64 oracle's own error (against the long
     double value);
  3  s2 and var only: within the rounding scale of the cancellation in
     v_n(x) = K(x,x) + g - k^T K^{-1} k (Eq. preds2), sqrt(n) eps (1 + g) / v_n(x), capped
     at CANCEL_CAP.

Every clause used is counted in TALLY (with the largest error it admitted), so a run can
print how many values needed each loosening past VAL_RTOL.
"""
from __future__ import annotations

import threading

import numpy as np

from . import design_predict, local_design, pred_derivs

SEL_RTOL = 1e-9      # near-tie margin for selections
VAL_RTOL = 1e-10     # relative tolerance for mean, s2 and var (both precisions)
ADJ_FACTOR = 8.0     # clause 2: GPU error vs long double <= this x the oracle's own
CANCEL_CAP = 1e-9    # clause 3 never admits more than this relative error (v_n(x) >= g, so
                     # at g = 1e-6 the bound itself stays below it for n <= 80)
EPS64 = 2.0 ** -53

CLAUSES = {0: "within 1e-10 of the FP64 oracle", 1: "within 1e-10 of the long-double oracle",
           2: "at most 8x the FP64 oracle's own error", 3: "within the cancellation bound"}

_tally_lock = threading.Lock()
TALLY: dict = {}


def _record(clause: int, err: float) -> None:
    with _tally_lock:
        c, m = TALLY.get(clause, (0, 0.0))
        TALLY[clause] = (c + 1, max(m, err))


def tally_reset() -> None:
    with _tally_lock:
        TALLY.clear()


def tally_summary() -> dict:
    """{clause: {"values": count, "max_rel_err": largest error admitted}} for clauses 1-3."""
    with _tally_lock:
        return {k: {"values": c, "max_rel_err": m} for k, (c, m) in sorted(TALLY.items()) if k}


def cancellation_bound(w, x, idx):
    """Rounding scale of v_n(x) = K(x,x) + g - k^T K^{-1} k (Eq. preds2) in FP64: each of
    its n-term inner products carries errors growing like sqrt(n) eps times the size of the
    terms (about 1 + g), and v_n(x) can be far smaller than that, so the relative error of
    s2 and var is of order sqrt(n) eps (1 + g) / v_n(x).  Capped at CANCEL_CAP."""
    Xd, Yd = w.X[idx], w.Z[idx]
    v = pred_derivs(Xd, Yd, x, w.d, w.g)[6]
    return float(min(np.sqrt(len(idx)) * EPS64 * (1.0 + w.g) / v, CANCEL_CAP))


def rel_err(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = np.maximum(np.abs(b), 1e-300)
    return np.abs(a - b) / den


def check_location(w, t, cand_t, gpu_idx, gpu_mean, gpu_s2, method="alc", val_rtol=VAL_RTOL,
                   sel_rtol=SEL_RTOL, gpu_var=None, start=None, ora=None):
    """Check one location; returns a dict with the path used, the errors and the clause
    that admitted each value.  With start (saved design indices) the design grows from it
    instead of the n0 nearest.  ora: the oracle's own result for this location (a dict
    with idx, mean, s2, var), when the caller already has it."""
    x = w.XX[t]
    if ora is None:
        ora = local_design(w.X, w.Z, x, cand_t, w.n0, w.n, w.d, w.g, method, start=start)
        assert ora["status"] == 0, "oracle failed at location %d" % t
    # start design: the n0 nearest in order, or the saved design
    first = cand_t[: w.n0] if start is None else np.asarray(start)
    assert np.array_equal(gpu_idx[: len(first)], first), "start design differs at %d" % t
    info = dict(t=t, forced=False, near_ties=0)
    ref = ora
    if not np.array_equal(ora["idx"], gpu_idx):
        f = local_design(w.X, w.Z, x, cand_t, w.n0, w.n, w.d, w.g, method, forced=gpu_idx,
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
    gvals = [gpu_mean, gpu_s2] + ([gpu_var] if gpu_var is not None else [])
    rvals = [ref["mean"], ref["s2"], ref["var"]]
    errs = [float(rel_err(g, r)) for g, r in zip(gvals, rvals)]
    info.update(err_mean=errs[0], err_s2=errs[1], ref_mean=ref["mean"], ref_s2=ref["s2"],
                ref_var=ref["var"])
    if gpu_var is not None:
        info["err_var"] = errs[2]
    clauses = [0 if e <= val_rtol else None for e in errs]
    info["adjudicated"] = any(c is None for c in clauses)
    if info["adjudicated"]:
        # v_n(x) = K(x,x) - k^T K^{-1} k is a cancellation whose sensitivity to one-ulp
        # differences in the correlations grows like |K^{-1}k|^2 eps, so two correct FP64
        # evaluations can differ by more than val_rtol: the long-double oracle on the same
        # design decides (clauses 1-3 of the module docstring).
        ld = design_predict(w.X, w.Z, x, gpu_idx, w.d, w.g, long_double=True)
        cb = None
        for k in range(len(errs)):
            if clauses[k] is not None:
                continue
            e_gpu = float(rel_err(gvals[k], ld[k]))
            e_ora = float(rel_err(rvals[k], ld[k]))
            info["adj_%d" % k] = (e_gpu, e_ora)
            if e_gpu <= val_rtol:
                clauses[k] = 1
            elif e_gpu <= ADJ_FACTOR * max(e_ora, 1e-14):
                clauses[k] = 2
            elif k > 0:
                cb = cancellation_bound(w, x, gpu_idx) if cb is None else cb
                info["cancel_bound"] = cb
                if e_gpu <= cb:
                    clauses[k] = 3
            if clauses[k] is not None:
                _record(clauses[k], e_gpu)
    info["clauses"] = clauses
    info["ok_vals"] = all(c is not None for c in clauses)
    return info


def check_sample(w, locs, ora, gpu, method="alc"):
    """The protocol on a sample of locations, with the oracle's results for them already
    computed (ora: dict of arrays idx, mean, s2, var, cand indexed like locs) and the GPU's
    for every location (gpu: dict of arrays idx, mean, s2, var indexed by t).  Returns a
    summary: the largest and median relative error of mean, s2 and var against the FP64
    oracle along the path the GPU took, the selection match rate, forced-path locations and
    near-tie steps, the values admitted by each adjudication clause (with the largest error
    each admitted) and the number of locations that failed."""
    errs = {"mean": [], "s2": [], "var": []}
    same = forced = near = failed = 0
    by_clause: dict = {}
    first_failure = None
    for k, t in enumerate(locs):
        o = {key: ora[key][k] for key in ("idx", "mean", "s2", "var")}
        try:
            info = check_location(w, t, ora["cand"][k], gpu["idx"][t], gpu["mean"][t],
                                  gpu["s2"][t], method, gpu_var=gpu["var"][t], ora=o)
        except AssertionError as e:   # a selection beyond the near-tie margin
            failed += 1
            first_failure = first_failure or str(e)
            continue
        same += not info["forced"]
        forced += info["forced"]
        near += info["near_ties"]
        for name, key in (("mean", "err_mean"), ("s2", "err_s2"), ("var", "err_var")):
            errs[name].append(info[key])
        for k2, c in enumerate(info["clauses"]):
            if c:
                e = info["adj_%d" % k2][0]
                n, m = by_clause.get(c, (0, 0.0))
                by_clause[c] = (n + 1, max(m, e))
        if not info["ok_vals"]:
            failed += 1
            first_failure = first_failure or "values at location %d: %s" % (
                t, {kk: info.get(kk) for kk in ("err_mean", "err_s2", "err_var", "adj_0",
                                                "adj_1", "adj_2", "cancel_bound")})
    out = {"locations": len(locs), "selection_match_rate": same / max(len(locs), 1),
           "forced_path_locations": forced, "near_tie_steps": near, "failed": failed}
    for name, v in errs.items():
        v = np.asarray(v) if v else np.zeros(1)
        out["max_rel_err_" + name] = float(v.max())
        out["median_rel_err_" + name] = float(np.median(v))
    out["adjudicated"] = {CLAUSES[c]: {"values": n, "max_rel_err": m}
                          for c, (n, m) in sorted(by_clause.items())}
    if first_failure:
        out["first_failure"] = first_failure[:400]
    return out
