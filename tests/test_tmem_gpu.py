"""Factor rows in tensor memory: the mixed ALC kernel's instance without the row ring keeps
rows R .. R + RT - 1 of every candidate also in its CTA's tensor memory and reads them from
there.  Against the same instance reading them from global memory (LAGP_MIX_TMEM=0, a
launch-shape override that changes no result) the designs and outputs must be bitwise
identical -- the same values summed in the same order -- for 1 to 4 candidate pairs per
thread (16, 8 and 4 rows in tensor memory), and they must pass the oracle protocol (needs a
GPU)."""
from __future__ import annotations

import contextlib
import os

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs
from tests.parity import check_location
from tests.test_parity_gpu import gpu_predict

pytestmark = pytest.mark.gpu


@contextlib.contextmanager
def tmem(on: bool):
    old = os.environ.get("LAGP_MIX_TMEM")
    try:
        if on:
            os.environ.pop("LAGP_MIX_TMEM", None)
        else:
            os.environ["LAGP_MIX_TMEM"] = "0"
        yield
    finally:
        if old is None:
            os.environ.pop("LAGP_MIX_TMEM", None)
        else:
            os.environ["LAGP_MIX_TMEM"] = old


def _same(a, b, what):
    for k in ("idx", "mean", "s2", "var", "status"):
        assert np.array_equal(a[k], b[k]), (what, k)


# n x M below the row ring's threshold (the instance without the ring); M sets the pairs
# per thread: 300 -> 1, 1000 -> 2, 1500 -> 3, 2000 -> 4
@pytest.mark.parametrize("M,n", [(300, 40), (1000, 50), (1500, 45), (2000, 48), (777, 30)])
def test_tmem_rows_are_bitwise_the_global_rows(M, n):
    w = inputs.random_case(600 + M, 20000, 2, 96, 6, n, M, d=0.05, g=1e-6)
    with tmem(False):
        ref = gpu_predict(w, "alc", "mixed")
    with tmem(True):
        got = gpu_predict(w, "alc", "mixed")
    assert (got["status"] == 0).all()
    _same(got, ref, (M, n))


def test_tmem_rows_paper_2d_against_the_oracle():
    w = inputs.paper_2d()
    w.XX = np.ascontiguousarray(w.XX[:600])
    with tmem(True):
        got = gpu_predict(w, "alc", "mixed")
    with tmem(False):
        ref = gpu_predict(w, "alc", "mixed")
    _same(got, ref, "paper-2d")
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in np.random.default_rng(8).choice(w.T, size=24, replace=False):
        info = check_location(w, t, cand[t], got["idx"][t], got["mean"][t], got["s2"][t], "alc",
                              gpu_var=got["var"][t])
        assert info["ok_vals"], info


def test_tmem_rows_edge_cases():
    # a design that ends inside the tensor-memory rows, no greedy step, an exhausted pool
    for w in (inputs.random_case(31, 3000, 2, 40, 4, 9, 300, d=0.05),
              inputs.random_case(32, 3000, 2, 40, 12, 12, 300, d=0.05),
              inputs.random_case(33, 3000, 3, 40, 3, 14, 14, d=0.1)):
        with tmem(False):
            ref = gpu_predict(w, "alc", "mixed")
        with tmem(True):
            got = gpu_predict(w, "alc", "mixed")
        _same(got, ref, w.name)


# n x M past the row ring's threshold: the ring instances (per-warp row copies, or the shared
# copy at large n), with 4 and 2 pairs per thread (4 and 8 rows in tensor memory)
@pytest.mark.parametrize("M,n", [(2000, 60), (1000, 120), (2000, 160)])
def test_tmem_rows_in_the_ring_instances_are_bitwise_the_global_rows(M, n):
    w = inputs.random_case(700 + M + n, 30000, 3, 40, 6, n, M, d=0.08, g=1e-6)
    with tmem(False):
        ref = gpu_predict(w, "alc", "mixed")
    with tmem(True):
        got = gpu_predict(w, "alc", "mixed")
    assert (got["status"] == 0).all()
    _same(got, ref, (M, n))
