"""The no-allocation entry point lagp_select_dev_noalloc, checked through the C ABI.

Some callers cannot allocate device memory (a plugin inside a host application that
owns all device allocations, a real-time loop that cannot take cudaMalloc's
synchronisation, a process with no allocation budget left).  For them the library
offers the greedy-design kernels with scratch taken from a static device array instead
of a workspace.  These tests compare it with the workspace entry point lagp_select_dev
on the same inputs, twice in a row (the array keeps the previous call's contents), and
check that a problem too large for the array is refused.  This file is collected last
so that a failure here stops a -x run only after every other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import VAL_RTOL

pytestmark = pytest.mark.gpu


def _case(w):
    import torch
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    X, Z, XX = d(w.X), d(w.Z), d(w.XX)
    cand = torch.empty((w.T, w.ncand), dtype=torch.int32, device="cuda")
    lagp.lagp_knn_dev(X, XX, w.ncand, cand,
                      lagp.workspace(lagp.lagp_knn_workspace_bytes(w.N, w.T, w.ncand)))
    return X, Z, XX, cand


def _outs(T, n):
    import torch
    mean = torch.full((T,), float("nan"), dtype=torch.float64, device="cuda")
    return dict(mean=mean, s2=torch.full_like(mean, float("nan")),
                var=torch.full_like(mean, float("nan")),
                idx=torch.full((T, n), -7, dtype=torch.int32, device="cuda"),
                status=torch.full((T,), 9, dtype=torch.int8, device="cuda"))


@pytest.mark.parametrize("make", [inputs.tiny_2d,
                                  lambda: inputs.random_case(77, 3000, 3, 700, 5, 40, 300, d=0.4)])
def test_noalloc_matches_workspace_entry_point_on_two_calls(make):
    import torch
    w = make()
    X, Z, XX, cand = _case(w)
    ref = _outs(w.T, w.n)
    ws = lagp.workspace(lagp.lagp_select_workspace_bytes(w.T, w.p, w.n, w.ncand))
    lagp.lagp_select_dev(X, Z, XX, cand, w.n0, w.n, w.d, w.g, "alc", "fp64", ref["mean"],
                         ref["s2"], ref["var"], ref["idx"], ref["status"], ws)
    torch.cuda.synchronize()
    for call in range(2):
        got = _outs(w.T, w.n)
        code = lagp.lagp_select_dev_noalloc(X, Z, XX, cand, w.n0, w.n, w.d, w.g, "alc", "fp64",
                                            got["mean"], got["s2"], got["var"], got["idx"],
                                            got["status"])
        torch.cuda.synchronize()
        assert code == lagp.LAGP_OK, lagp.strerror(code)
        assert torch.equal(got["status"], ref["status"]), call
        assert torch.equal(got["idx"], ref["idx"]), call
        for k in ("mean", "s2", "var"):
            a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
            rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
            assert np.all(rel <= VAL_RTOL), (call, k, rel.max())


def test_noalloc_refuses_problems_larger_than_its_scratch():
    import torch
    w = inputs.random_case(78, 9000, 2, 2, 6, 256, 8192, d=0.3)
    X, Z, XX, cand = _case(w)
    out = _outs(w.T, w.n)
    code = lagp.lagp_select_dev_noalloc(X, Z, XX, cand, w.n0, w.n, w.d, w.g, "alc", "fp64",
                                        out["mean"], out["s2"], out["var"], out["idx"],
                                        out["status"])
    torch.cuda.synchronize()
    assert code == lagp.LAGP_ERR_SCRATCH_LIMIT
    assert "static scratch" in lagp.strerror(code)
