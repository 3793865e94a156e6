"""The seeded input generators: shapes, determinism and the sampling designs they claim."""
from __future__ import annotations

import numpy as np

from paper_1303_0383_gb300 import inputs


def test_latin_hypercube_has_one_point_per_stratum():
    rng = np.random.default_rng(3)
    U = inputs.latin_hypercube(rng, 257, 5)
    assert U.shape == (257, 5) and (U >= 0).all() and (U < 1).all()
    for k in range(5):
        assert np.array_equal(np.sort(np.floor(U[:, k] * 257).astype(int)), np.arange(257))


def test_grid_2d_is_the_dense_201_grid():
    w = inputs.grid_2d()
    assert w.N == 201 * 201 and w.T == 10000 and w.p == 2
    xs = np.unique(w.X[:, 0])
    assert len(xs) == 201 and xs[0] == -2.0 and xs[-1] == 2.0
    assert np.allclose(np.diff(xs), 0.02)
    # f = -w(x1) w(x2) is symmetric under swapping the coordinates
    Zs = w.Z.reshape(201, 201)
    assert np.allclose(Zs, Zs.T, rtol=0, atol=1e-15)


def test_borehole_design_and_response():
    w = inputs.borehole()
    assert (w.N, w.T, w.p) == (4000, 500, 8)
    U = np.vstack([w.X, w.XX])  # one hypercube of 4500 points
    for k in range(8):
        assert np.array_equal(np.sort(np.floor(U[:, k] * 4500).astype(int)), np.arange(4500))
    # the flow rate grows with the head difference H_u - H_l (inputs 4 and 5)
    base = np.full((2, 8), 0.5)
    base[1, 4] = 0.9
    y = inputs.borehole_response(base)
    assert y[1] > y[0] > 0
    assert 0 < w.Z.min() and w.Z.max() < 400


def test_generators_are_deterministic():
    a, b = inputs.borehole(), inputs.borehole()
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Z, b.Z)
    c, d = inputs.paper_2d(), inputs.paper_2d()
    assert np.array_equal(c.XX, d.XX) and np.array_equal(c.Z, d.Z)


def test_borehole_domain_is_the_papers():
    # the eight input ranges printed below Eq. borehole (tests/golden/borehole_domain.txt)
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "borehole_domain.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert [r[0] for r in rows] == ["r_w", "r", "T_u", "T_l", "H_u", "H_l", "L", "K_w"]
    assert [(float(r[1]), float(r[2])) for r in rows] == [tuple(map(float, b)) for b in inputs.BOREHOLE_BOX]
