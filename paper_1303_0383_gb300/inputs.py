"""Seeded synthetic inputs for local approximate GP emulation.

This module only draws inputs; it holds none of the method's arithmetic (no
correlation function, no design criterion, no predictive equation), so both the
CUDA path and the CPU oracle can take their inputs from it.

The first five workloads stand in for the paper's own test problems (Sec. 3.4: a 2-d
surface on a dense 201x201 grid over [-2,2]^2; Sec. 5.2: the 8-d borehole function on
an LHS), which are not shipped as data; grid_2d and borehole rebuild those two problems
from their formulas.  Shapes follow the five workload
descriptions below; every draw comes from numpy's PCG64 (``default_rng``) with
seed 1303038300 + workload number, designs drawn first, then predictive sets,
then noise.

Arrays are float64, row-major (C order): X is N x p, Z is N, XX is T x p.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1303038300


@dataclasses.dataclass
class Workload:
    """One synthetic problem: a design (X, Z), a predictive set XX and the knobs."""
    name: str
    X: np.ndarray
    Z: np.ndarray
    XX: np.ndarray
    n0: int
    n: int
    ncand: int
    d: float      # lengthscale theta of exp(-||x-x'||^2 / theta)
    g: float      # nugget eta
    ZZ: np.ndarray | None = None  # the noise-free response at XX, where it is known

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def p(self) -> int:
        return int(self.X.shape[1])

    @property
    def T(self) -> int:
        return int(self.XX.shape[0])


def _surface_2d(X: np.ndarray) -> np.ndarray:
    # z = x1 * exp(-x1^2 - x2^2): the 2-d response of the tiny and paper-scale workloads
    return X[:, 0] * np.exp(-X[:, 0] ** 2 - X[:, 1] ** 2)


def _surface_8d(X: np.ndarray) -> np.ndarray:
    # z = sum_j sin(2 pi x_j)/j + x1 x2 x3 + exp(-||x - 0.5||^2)
    j = np.arange(1, X.shape[1] + 1, dtype=np.float64)
    s = np.sum(np.sin(2.0 * math.pi * X) / j, axis=1)
    return s + X[:, 0] * X[:, 1] * X[:, 2] + np.exp(-np.sum((X - 0.5) ** 2, axis=1))


def _surface_4d(X: np.ndarray) -> np.ndarray:
    # z = prod_j sin(3 x_j)
    return np.prod(np.sin(3.0 * X), axis=1)


def _grid(lo: float, hi: float, m: int) -> np.ndarray:
    g = np.linspace(lo, hi, m)
    a, b = np.meshgrid(g, g, indexing="ij")
    return np.ascontiguousarray(np.stack([a.ravel(), b.ravel()], axis=1))


def tiny_2d() -> Workload:
    """N=2000 uniform on [-2,2]^2, 10x10 grid over [-1.9,1.9]^2, d=0.5, g=1e-6, n0=6, n=50, 200 candidates."""
    rng = np.random.default_rng(SEED_BASE + 1)
    X = rng.uniform(-2.0, 2.0, size=(2000, 2))
    XX = _grid(-1.9, 1.9, 10)
    return Workload("tiny-2d N=2000 T=100 n=50 M=200", X, _surface_2d(X), XX,
                    n0=6, n=50, ncand=200, d=0.5, g=1e-6)


def paper_2d() -> Workload:
    """N=40000 uniform on [-2,2]^2, 100x100 grid over [-1.97,1.97]^2, d=0.5, g=1e-6, n0=6, n=50, 1000 candidates."""
    rng = np.random.default_rng(SEED_BASE + 2)
    X = rng.uniform(-2.0, 2.0, size=(40000, 2))
    XX = _grid(-1.97, 1.97, 100)
    return Workload("paper-2d N=40000 T=10000 n=50 M=1000", X, _surface_2d(X), XX,
                    n0=6, n=50, ncand=1000, d=0.5, g=1e-6)


def smooth_8d(T: int = 10000) -> Workload:
    """N=100000 uniform on [0,1]^8 with N(0, 1e-4) noise, T uniform points, d=1, g=1e-4, n0=8, n=100, 2000 candidates."""
    rng = np.random.default_rng(SEED_BASE + 3)
    X = rng.uniform(0.0, 1.0, size=(100000, 8))
    XX = rng.uniform(0.0, 1.0, size=(10000, 8))[:T]
    Z = _surface_8d(X) + rng.normal(0.0, math.sqrt(1e-4), size=X.shape[0])
    return Workload("smooth-8d N=100000 T=%d n=100 M=2000" % T, X, Z, np.ascontiguousarray(XX),
                    n0=8, n=100, ncand=2000, d=1.0, g=1e-4)


def _w_illustration(x: np.ndarray) -> np.ndarray:
    # w(x) of the paper's illustration surface (Sec. 3.4)
    return (np.exp(-(x - 1.0) ** 2) + np.exp(-0.8 * (x + 1.0) ** 2)
            - 0.05 * np.sin(8.0 * (x + 0.1)))


def grid_2d() -> Workload:
    """The paper's illustration problem (Sec. 3.4): f(x1, x2) = -w(x1) w(x2) on the dense
    201 x 201 regular grid over [-2, 2]^2 (40401 points), no noise.  Predictive set: 10000
    locations (Sec. 4.1), placed on a 100 x 100 grid over [-1.97, 1.97]^2 (the paper does
    not give their placement); every coordinate -1.97 + 3.94 k / 99 falls between design
    grid lines, so distances to the design tie or nearly tie.  d = 0.5, g = 1e-6 as for the
    other 2-d workloads; n0 = 6, n = 50, 1000 candidates (Sec. 3.4, Sec. 6)."""
    X = _grid(-2.0, 2.0, 201)
    Z = -_w_illustration(X[:, 0]) * _w_illustration(X[:, 1])
    XX = _grid(-1.97, 1.97, 100)
    ZZ = -_w_illustration(XX[:, 0]) * _w_illustration(XX[:, 1])
    return Workload("grid-2d N=40401 T=10000 n=50 M=1000", X, Z, XX,
                    n0=6, n=50, ncand=1000, d=0.5, g=1e-6, ZZ=ZZ)


# Ranges of the borehole function's eight inputs (Sec. 5.2), in the order
# r_w, r, T_u, T_l, H_u, H_l, L, K_w.
BOREHOLE_BOX = ((0.05, 0.15), (100.0, 5000.0), (63070.0, 115600.0), (63.1, 116.0),
                (990.0, 1110.0), (700.0, 820.0), (1120.0, 1680.0), (9855.0, 12045.0))


def borehole_response(U: np.ndarray) -> np.ndarray:
    """Eq. borehole at coded inputs U in [0, 1]^8 (mapped linearly onto BOREHOLE_BOX)."""
    lo = np.array([b[0] for b in BOREHOLE_BOX])
    hi = np.array([b[1] for b in BOREHOLE_BOX])
    V = lo + (hi - lo) * U
    rw, r, Tu, Tl, Hu, Hl, L, Kw = (V[:, k] for k in range(8))
    lg = np.log(r / rw)
    return 2.0 * math.pi * Tu * (Hu - Hl) / (lg * (1.0 + 2.0 * L * Tu / (lg * rw ** 2 * Kw) + Tu / Tl))


def latin_hypercube(rng: np.random.Generator, n: int, p: int) -> np.ndarray:
    """Random Latin hypercube on [0, 1]^p: in every dimension each of the n strata
    [i/n, (i+1)/n) holds exactly one point, at a uniform position inside it."""
    strata = np.stack([rng.permutation(n) for _ in range(p)], axis=1)
    return (strata + rng.random((n, p))) / n


def borehole(N: int = 4000, Npred: int = 500) -> Workload:
    """The borehole experiment (Sec. 5.2): one Latin hypercube of N + Npred points in the
    coded 8-d box, the first N for the design and the rest for prediction; response by
    Eq. borehole, no noise.  N = 4000 / Npred = 500 (Table 1) or 8000 / 1000 (Table SM.1).
    d = 0.64, about the 10% quantile of squared distances between points of the coded
    box (the paper's rule for the lengthscale's scale, Sec. 4.2; fixed here), g = 1e-6;
    n0 = 6, n = 50, 1000 candidates."""
    rng = np.random.default_rng(SEED_BASE + (6 if N <= 4000 else 7))
    U = latin_hypercube(rng, N + Npred, 8)
    X = np.ascontiguousarray(U[:N])
    XX = np.ascontiguousarray(U[N:])
    return Workload("borehole N=%d T=%d n=50 M=1000" % (N, Npred), X, borehole_response(X), XX,
                    n0=6, n=50, ncand=1000, d=0.64, g=1e-6, ZZ=borehole_response(XX))


def random_case(seed: int, N: int, p: int, T: int, n0: int, n: int, ncand: int,
                d: float = 0.3, g: float = 1e-6, lo: float = 0.0, hi: float = 1.0) -> Workload:
    """Small random problem for parity tests: X, XX uniform on [lo,hi]^p, Z a smooth random surface."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(lo, hi, size=(N, p))
    XX = rng.uniform(lo, hi, size=(T, p))
    a = rng.normal(size=p)
    Z = np.sin(X @ a) + 0.5 * np.cos(3.0 * X[:, 0])
    return Workload("random seed=%d N=%d p=%d T=%d" % (seed, N, p, T), X, Z, XX,
                    n0=n0, n=n, ncand=ncand, d=d, g=g)


@dataclasses.dataclass
class BatchWorkload:
    """Uneven local problems across several resident designs (one persistent launch)."""
    name: str
    designs: list          # list of Workload (X, Z, n0, d, g used; XX empty)
    design_of: np.ndarray  # T int32
    n: np.ndarray          # T int32
    ncand: np.ndarray      # T int32
    XX: np.ndarray         # T x 8, row t holds its design's p coordinates first

    @property
    def T(self) -> int:
        return int(self.n.shape[0])


def batched_uneven(T: int = 20000) -> BatchWorkload:
    """Three resident designs: the paper-scale 2-d design (N=40000, d=0.5, g=1e-6, n0=6), a
    4-d design N=200000 uniform on [0,1]^4 with z = prod_j sin(3 x_j) (d=0.2, g=1e-6, n0=6),
    and the 8-d design (N=100000, d=1, g=1e-4, n0=8).  T locations, a third per design at
    random, each uniform on its design's domain; n uniform on {30..200} and the candidate
    count uniform on {500..4000}, independently."""
    d2 = paper_2d()
    d8 = smooth_8d(T=1)
    rng = np.random.default_rng(SEED_BASE + 4)
    X4 = rng.uniform(0.0, 1.0, size=(200000, 4))
    d4 = Workload("4-d N=200000", X4, _surface_4d(X4), np.zeros((0, 4)), n0=6, n=30, ncand=500,
                  d=0.2, g=1e-6)
    designs = [Workload(d2.name, d2.X, d2.Z, np.zeros((0, 2)), d2.n0, 30, 500, d2.d, d2.g), d4,
               Workload(d8.name, d8.X, d8.Z, np.zeros((0, 8)), d8.n0, 30, 500, d8.d, d8.g)]
    design_of = rng.integers(0, 3, size=T).astype(np.int32)
    n = rng.integers(30, 201, size=T).astype(np.int32)
    ncand = rng.integers(500, 4001, size=T).astype(np.int32)
    XX = np.zeros((T, 8))
    lo = {0: -2.0, 1: 0.0, 2: 0.0}
    hi = {0: 2.0, 1: 1.0, 2: 1.0}
    for t in range(T):
        d = int(design_of[t])
        p = designs[d].p
        XX[t, :p] = rng.uniform(lo[d], hi[d], size=p)
    return BatchWorkload("batched-uneven T=%d over 2-d/4-d/8-d designs, n~U{30..200}, "
                         "ncand~U{500..4000}" % T, designs, design_of, n, ncand, XX)
