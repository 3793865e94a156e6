"""The paper's own problems rebuilt from their formulas (Sec. 3.4 illustration surface on
the 201 x 201 grid; Sec. 5.2 borehole on a Latin hypercube): CUDA path vs CPU oracle on
seeded samples of locations, in the launch configuration of the benchmark (needs a GPU)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs
from tests.test_parity_gpu import gpu_knn, run_parity

pytestmark = pytest.mark.gpu


def test_knn_bit_exact_grid_2d():
    # predictive coordinates fall between design grid lines: distances tie or nearly tie
    w = inputs.grid_2d()
    got = gpu_knn(w.X, w.XX, w.ncand)
    locs = np.random.default_rng(5).choice(w.T, size=300, replace=False)
    assert np.array_equal(got[locs], oracle.knn(w.X, w.XX[locs], w.ncand))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alc_grid_2d_sampled(precision):
    w = inputs.grid_2d()
    locs = np.random.default_rng(6).choice(w.T, size=24, replace=False)
    g, infos, bad = run_parity(w, locs=locs, precision=precision)
    assert not bad, bad[:3]


def test_knn_bit_exact_borehole():
    w = inputs.borehole()
    assert np.array_equal(gpu_knn(w.X, w.XX, w.ncand), oracle.knn(w.X, w.XX, w.ncand))


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed"), ("nn", "fp64")])
def test_borehole_sampled(method, precision):
    w = inputs.borehole()
    locs = np.random.default_rng(7).choice(w.T, size=16, replace=False)
    g, infos, bad = run_parity(w, locs=locs, method=method, precision=precision)
    assert not bad, bad[:3]


def test_borehole_double_size_sampled():
    w = inputs.borehole(8000, 1000)
    locs = np.random.default_rng(8).choice(w.T, size=12, replace=False)
    g, infos, bad = run_parity(w, locs=locs, precision="mixed")
    assert not bad, bad[:3]
