"""Adaptive local design size by the stopping rule of Sec. 6 on the GPU (needs a GPU).

The rule compares the chosen point's ratio v_j(x) / v_{j+1}(x) with r_min; where the
oracle's ratio lies within STOP_RTOL * (r_min - 1) of the threshold, either decision is
accepted (the same idea as the near-tie protocol for selections)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import cancellation_bound
from tests.test_parity_gpu import dev

pytestmark = pytest.mark.gpu

STOP_RTOL = 1e-6


def gpu_adaptive(w, cand, precision, r_min):
    import torch
    T = w.T
    out = {k: torch.empty(T, dtype=torch.float64, device="cuda") for k in ("mean", "s2", "var")}
    idx = torch.empty((T, w.n), dtype=torch.int32, device="cuda")
    n_out = torch.empty(T, dtype=torch.int32, device="cuda")
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    ws = lagp.workspace(lagp.lagp_select_workspace_bytes(T, w.p, w.n, w.ncand, "alc", precision))
    lagp.lagp_select_adaptive_dev(dev(w.X, torch.float64), dev(w.Z, torch.float64),
                                  dev(w.XX, torch.float64), dev(cand, torch.int32), w.n0, w.n, w.d,
                                  w.g, precision, r_min, out["mean"], out["s2"], n_out, out["var"],
                                  idx, st, ws)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r.update(idx=idx.cpu().numpy(), n_out=n_out.cpu().numpy(), status=st.cpu().numpy())
    return r


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("r_min", [1.001, 1.01, 1.1])
def test_adaptive_designs_match_oracle(precision, r_min):
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    g = gpu_adaptive(w, cand, precision, r_min)
    assert (g["status"] == 0).all()
    agree = 0
    for t in range(w.T):
        o = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc",
                                r_min=r_min)
        assert o["status"] == 0
        kg, ko = int(g["n_out"][t]), o["n_out"]
        assert w.n0 <= kg <= w.n and (g["idx"][t][kg:] == -1).all()
        k = min(kg, ko)
        assert np.array_equal(g["idx"][t][:k], o["idx"][:k]), t  # no near-ties on tiny-2d
        if kg != ko:
            # the oracle's ratio at the step where the two decisions differ is at the threshold
            ratio = o["trace"][k - w.n0, 6]
            assert abs(ratio - r_min) <= STOP_RTOL * (r_min - 1), (t, kg, ko, ratio)
            continue
        agree += 1
        em = abs(g["mean"][t] - o["mean"]) / abs(o["mean"])
        es = abs(g["s2"][t] - o["s2"]) / o["s2"]
        if em > 1e-10 or es > 1e-10:
            ld = oracle.design_predict(w.X, w.Z, w.XX[t], o["idx"][:k], w.d, w.g, long_double=True)
            e_g = abs(g["s2"][t] - ld[1]) / ld[1]
            e_o = abs(o["s2"] - ld[1]) / ld[1]
            assert abs(g["mean"][t] - ld[0]) <= 1e-10 * abs(ld[0]) + 1e-15, t
            assert e_g <= 1e-10 or e_g <= 8 * max(e_o, 1e-14) or \
                e_g <= cancellation_bound(w, w.XX[t], o["idx"][:k]), (t, e_g, e_o)
    assert agree >= w.T - 2
    # the design sizes vary across locations
    assert len(set(g["n_out"].tolist())) > 3


def test_adaptive_sizes_shrink_as_the_threshold_grows():
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    prev = None
    for r_min in (1.0005, 1.005, 1.05, 1.5):
        g = gpu_adaptive(w, cand, "mixed", r_min)
        if prev is not None:
            assert (g["n_out"] <= prev).all()
        prev = g["n_out"]
