"""Design augmentation from saved start designs (Sec. 6) on the GPU (needs a GPU)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import check_location
from tests.test_parity_gpu import dev, gpu_predict

pytestmark = pytest.mark.gpu


def gpu_augment(w, cand, start, method="alc", precision="fp64", n=None):
    import torch
    n = n or w.n
    T = start.shape[0]
    out = {k: torch.empty(T, dtype=torch.float64, device="cuda") for k in ("mean", "s2", "var")}
    idx = torch.empty((T, n), dtype=torch.int32, device="cuda")
    st = torch.empty(T, dtype=torch.int8, device="cuda")
    ws = lagp.workspace(lagp.lagp_select_workspace_bytes(T, w.p, n, w.ncand, method, precision))
    lagp.lagp_select_augment_dev(dev(w.X, torch.float64), dev(w.Z, torch.float64),
                                 dev(w.XX, torch.float64), dev(cand, torch.int32),
                                 dev(start, torch.int32), n, w.d, w.g, method, precision,
                                 out["mean"], out["s2"], out["var"], idx, st, ws)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r.update(idx=idx.cpu().numpy(), status=st.cpu().numpy())
    return r


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed")])
def test_augmenting_a_prefix_reproduces_the_design(method, precision):
    w = inputs.tiny_2d()
    full = gpu_predict(w, method, precision)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for n1 in (w.n0, 20, w.n - 1):
        a = gpu_augment(w, cand, np.ascontiguousarray(full["idx"][:, :n1]), method, precision)
        assert (a["status"] == 0).all()
        assert np.array_equal(a["idx"], full["idx"]), n1
        assert np.array_equal(a["mean"], full["mean"]) and np.array_equal(a["s2"], full["s2"]), n1


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed")])
def test_augmenting_a_design_chosen_at_another_lengthscale(method, precision):
    # saved designs of 20 points chosen at theta = 0.25, grown to 50 at theta = 0.5
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    r = oracle.predict(w.X, w.Z, w.XX, w.n0, 20, w.ncand, 0.25, w.g, "alc")
    start = np.ascontiguousarray(r["idx"])
    a = gpu_augment(w, cand, start, method, precision)
    assert (a["status"] == 0).all()
    bad = []
    for t in range(0, w.T, 3):
        info = check_location(w, t, cand[t], a["idx"][t], a["mean"][t], a["s2"][t], method,
                              gpu_var=a["var"][t], start=start[t])
        if not info["ok_vals"]:
            bad.append(info)
    assert not bad, bad[:3]


def test_augmenting_flags_a_start_point_outside_the_candidates():
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    full = gpu_predict(w)
    start = np.ascontiguousarray(full["idx"][:, :10])
    outside = np.setdiff1d(np.arange(w.N), cand[3])[0]
    start[3, 5] = outside
    a = gpu_augment(w, cand, start)
    assert a["status"][3] == lagp.LAGP_ERR_NOT_PD and np.isnan(a["mean"][3])
    ok = np.arange(w.T) != 3
    assert (a["status"][ok] == 0).all()
    assert np.array_equal(a["idx"][ok], full["idx"][ok])
