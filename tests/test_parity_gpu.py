"""CUDA path vs CPU oracle, through the C ABI (needs a GPU)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import check_location, VAL_RTOL

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def dev(a, dtype=None):
    torch = _torch()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def gpu_knn(X, XX, M):
    torch = _torch()
    Xd, XXd = dev(X, torch.float64), dev(XX, torch.float64)
    cand = torch.empty((XX.shape[0], M), dtype=torch.int32, device="cuda")
    ws = lagp.workspace(lagp.lagp_knn_workspace_bytes(X.shape[0], XX.shape[0], M))
    lagp.lagp_knn_dev(Xd, XXd, M, cand, ws)
    torch.cuda.synchronize()
    return cand.cpu().numpy()


def gpu_predict(w, method="alc", precision="fp64"):
    torch = _torch()
    out = lagp.predict_torch(dev(w.X, torch.float64), dev(w.Z, torch.float64),
                             dev(w.XX, torch.float64), w.n0, w.n, w.ncand, w.d, w.g, method,
                             precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def run_parity(w, locs=None, method="alc", precision="fp64", val_rtol=VAL_RTOL):
    g = gpu_predict(w, method, precision)
    assert (g["status"] == 0).all()
    locs = range(w.T) if locs is None else locs
    XXs = w.XX[list(locs)]
    cand = oracle.knn(w.X, XXs, w.ncand)
    infos, bad = [], []
    for k, t in enumerate(locs):
        info = check_location(w, t, cand[k], g["idx"][t], g["mean"][t], g["s2"][t], method,
                              val_rtol=val_rtol, gpu_var=g["var"][t])
        infos.append(info)
        if not info["ok_vals"]:
            bad.append(info)
    return g, infos, bad


def test_knn_bit_exact_tiny_2d():
    w = inputs.tiny_2d()
    got = gpu_knn(w.X, w.XX, w.ncand)
    ref = oracle.knn(w.X, w.XX, w.ncand)
    assert np.array_equal(got, ref)


# the last two: survivor capacities 8192 (the bucket sort's own permutation array) and
# 16384 (the largest candidate count, 8192; permutation in the histogram or bitonic sort)
@pytest.mark.parametrize("p,N,T,M", [(1, 777, 13, 64), (3, 1234, 37, 97), (8, 3001, 19, 500),
                                     (2, 12000, 5, 4000), (2, 20000, 5, 8192)])
def test_knn_bit_exact_random_ragged(p, N, T, M):
    w = inputs.random_case(11 + p, N, p, T, 3, 10, M)
    assert np.array_equal(gpu_knn(w.X, w.XX, M), oracle.knn(w.X, w.XX, M))


def test_knn_ties_and_boundary_refinement():
    # many exactly equal distances: duplicated rows force the index tie-break and a
    # boundary bin larger than shared memory (radix refinement path)
    rng = np.random.default_rng(5)
    base = rng.uniform(0, 1, size=(40, 2))
    X = np.concatenate([np.repeat(base, 250, axis=0), rng.uniform(0, 1, size=(3000, 2))])
    XX = np.concatenate([base[:5], rng.uniform(0, 1, size=(6, 2))])
    for M in (100, 1500, 4000):
        assert np.array_equal(gpu_knn(X, XX, M), oracle.knn(X, XX, M)), M


@pytest.mark.parametrize("near", [True, False])
def test_knn_when_the_strided_sample_misleads(near):
    # kernel (a) bounds the ncand-th distance from a sample of the design -- the blocks of
    # 32 consecutive points that start every 512 points -- and falls back to two full
    # passes when that bound misses; here the sampled points are either all close to the
    # locations (too few points under the bound) or all far from them (too many), and the
    # candidate lists must still equal a full sort's
    rng = np.random.default_rng(17 + near)
    N, M = 512 * 10 + 40, 500
    X = rng.uniform(-1.0, 1.0, size=(N, 2))
    sampled = np.nonzero((np.arange(N) // 32) % 16 == 0)[0]
    if near:
        X[sampled] = rng.uniform(-0.02, 0.02, size=(len(sampled), 2))
    else:
        X[sampled] = rng.uniform(5.0, 6.0, size=(len(sampled), 2))
    XX = rng.uniform(-0.01, 0.01, size=(9, 2))
    assert np.array_equal(gpu_knn(X, XX, M), oracle.knn(X, XX, M))


def test_knn_grid_ties():
    # regular grid design (as in the paper's 201 x 201 illustration): exact ties in d2
    g = np.linspace(-2, 2, 41)
    a, b = np.meshgrid(g, g, indexing="ij")
    X = np.stack([a.ravel(), b.ravel()], 1)
    XX = np.array([[0.0, 0.0], [0.1, 0.1], [-2.0, 2.0], [0.05, -0.3]])
    assert np.array_equal(gpu_knn(X, XX, 200), oracle.knn(X, XX, 200))


def test_alc_parity_tiny_2d_all_locations():
    w = inputs.tiny_2d()
    g, infos, bad = run_parity(w)
    assert not bad, "value mismatches beyond %.0e: %s" % (VAL_RTOL, bad[:3])


def test_nn_parity_tiny_2d():
    w = inputs.tiny_2d()
    g, infos, bad = run_parity(w, method="nn")
    assert not any(i["forced"] for i in infos)
    assert not bad, bad[:3]


@pytest.mark.parametrize("p,seed", [(1, 1), (2, 2), (3, 3), (8, 4)])
def test_alc_parity_random_small(p, seed):
    w = inputs.random_case(100 + seed, 300, p, 23, 4, 20, 60, d=0.2 * p, g=1e-6)
    g, infos, bad = run_parity(w)
    assert not bad, bad[:3]


def test_edge_n0_equals_n_and_m_equals_n():
    w = inputs.random_case(7, 200, 2, 9, 12, 12, 12)   # no greedy step, M == n
    g, infos, bad = run_parity(w)
    assert not bad
    w = inputs.random_case(8, 200, 2, 9, 3, 12, 12)    # pool exhausted exactly
    g, infos, bad = run_parity(w)
    assert not bad


def test_single_and_empty_batch():
    torch = _torch()
    w = inputs.random_case(9, 300, 2, 1, 4, 15, 40)
    g, infos, bad = run_parity(w)
    assert not bad
    # T = 0 is a no-op that succeeds
    X = dev(w.X, torch.float64)
    Z = dev(w.Z, torch.float64)
    XX = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    lagp.lagp_predict_dev(X, Z, XX, 4, 15, 40, 0.3, 1e-6, "alc", "fp64", e, e, ws=lagp.workspace(256))


def test_host_api_matches_device_api():
    w = inputs.tiny_2d()
    gd = gpu_predict(w)
    d = lagp.Design(w.X, w.Z)
    h = d.predict(w.XX, w.n0, w.n, w.ncand, w.d, w.g)
    d.close()
    assert np.array_equal(h["idx"], gd["idx"])
    assert np.array_equal(h["mean"], gd["mean"]) and np.array_equal(h["s2"], gd["s2"])


def test_paper_2d_full_size_sampled():
    # the full paper-scale workload in the benchmark's launch configuration; the oracle
    # checks a seeded sample of locations
    w = inputs.paper_2d()
    locs = np.random.default_rng(0).choice(w.T, size=40, replace=False)
    g, infos, bad = run_parity(w, locs=locs)
    assert not bad, bad[:3]


def test_library_exp_against_cuda_and_long_double():
    """The table-driven FP64 exp used for correlations: within 1 ulp of a long-double
    reference over the argument range the kernels use, and within 2 ulp of CUDA's exp."""
    torch = _torch()
    rng = np.random.default_rng(3)
    x = np.concatenate([-rng.exponential(1.0, 200000), -rng.uniform(0, 707, 200000),
                        -np.logspace(-18, 2.8, 20000), [0.0, -0.0, -1e-300, -706.9]])
    xd = torch.as_tensor(x).cuda()
    y = torch.empty_like(xd)
    lagp.lagp_exp_dev(xd, y)
    ours = y.cpu().numpy()
    cuda = torch.exp(xd).cpu().numpy()
    ref = np.exp(x.astype(np.longdouble))
    ulp = np.spacing(np.abs(ref.astype(np.float64)))
    err_ref = np.abs(ours.astype(np.longdouble) - ref) / ulp
    assert float(err_ref.max()) <= 1.0, float(err_ref.max())
    err_cuda = np.abs(ours - cuda) / ulp
    assert float(err_cuda.max()) <= 2.0, float(err_cuda.max())
    assert np.all(lagp_exp_zero_below(x, ours))


def lagp_exp_zero_below(x, y):
    return np.where(x < -707.0, y == 0.0, True)


# ----------------------------------------------------------------- mixed precision

def test_mixed_parity_tiny_2d_all_locations():
    w = inputs.tiny_2d()
    g, infos, bad = run_parity(w, precision="mixed")
    assert not bad, bad[:3]


@pytest.mark.parametrize("p,seed", [(1, 1), (2, 2), (3, 3), (8, 4)])
def test_mixed_parity_random_small(p, seed):
    w = inputs.random_case(100 + seed, 300, p, 23, 4, 20, 60, d=0.2 * p, g=1e-6)
    g, infos, bad = run_parity(w, precision="mixed")
    assert not bad, bad[:3]


def test_mixed_edge_cases():
    for w in (inputs.random_case(7, 200, 2, 9, 12, 12, 12), inputs.random_case(8, 200, 2, 9, 3, 12, 12),
              inputs.random_case(9, 300, 2, 1, 4, 15, 40)):
        g, infos, bad = run_parity(w, precision="mixed")
        assert not bad, bad[:3]


def test_mixed_paper_2d_full_size_sampled_and_agrees_with_fp64():
    w = inputs.paper_2d()
    locs = np.random.default_rng(1).choice(w.T, size=40, replace=False)
    g, infos, bad = run_parity(w, locs=locs, precision="mixed")
    assert not bad, bad[:3]
    f = gpu_predict(w, precision="fp64")
    same = (f["idx"] == g["idx"]).all(axis=1)
    # designs differ only where some step was a near-tie within FP64 rounding
    assert same.mean() >= 0.999, same.mean()
    rel = np.abs(f["s2"][same] - g["s2"][same]) / f["s2"][same]
    assert rel.max() <= 1e-9, rel.max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_repeated_runs_are_bitwise_identical(precision):
    """Every location's arithmetic depends only on its own inputs: two runs (and the host
    entry point) give bitwise-identical designs and values."""
    w = inputs.paper_2d()
    w.XX = np.ascontiguousarray(w.XX[:3000])
    a = gpu_predict(w, precision=precision)
    b = gpu_predict(w, precision=precision)
    for k in ("idx", "mean", "s2", "var", "status"):
        assert np.array_equal(a[k], b[k]), k
    d = lagp.Design(w.X, w.Z)
    h = d.predict(w.XX, w.n0, w.n, w.ncand, w.d, w.g, "alc", precision)
    d.close()
    for k in ("idx", "mean", "s2", "var", "status"):
        assert np.array_equal(h[k], a[k]), k


# ----------------------------------------------------------------- MSPE (FP64)

def test_mspe_parity_tiny_2d():
    w = inputs.tiny_2d()
    g, infos, bad = run_parity(w, method="mspe")
    assert not bad, bad[:3]


@pytest.mark.parametrize("p,seed,g", [(1, 11, 1e-4), (2, 12, 1e-6), (3, 13, 1e-4), (8, 14, 1e-4)])
def test_mspe_parity_random_small(p, seed, g):
    w = inputs.random_case(200 + seed, 300, p, 19, 4, 18, 60, d=0.25 * p, g=g)
    g_, infos, bad = run_parity(w, method="mspe")
    assert not bad, bad[:3]


def test_mspe_parity_smooth_8d_sample():
    # the 8-d workload's shape (n0=8, n=100, 2000 candidates, g=1e-4) on a small sample
    w = inputs.smooth_8d(T=24)
    g, infos, bad = run_parity(w, locs=range(0, 24, 3), method="mspe")
    assert not bad, bad[:3]


# ----------------------------------------------------------------- MSPE (mixed)

def test_mspe_mixed_parity_tiny_2d():
    w = inputs.tiny_2d()
    g, infos, bad = run_parity(w, method="mspe", precision="mixed")
    assert not bad, bad[:3]


@pytest.mark.parametrize("p,seed,g", [(1, 11, 1e-4), (2, 12, 1e-6), (3, 13, 1e-4), (8, 14, 1e-4)])
def test_mspe_mixed_parity_random_small(p, seed, g):
    w = inputs.random_case(200 + seed, 300, p, 19, 4, 18, 60, d=0.25 * p, g=g)
    g_, infos, bad = run_parity(w, method="mspe", precision="mixed")
    assert not bad, bad[:3]


def test_mspe_mixed_edge_cases():
    # n0 = n (no greedy step), ncand = n, and the smallest admissible n0
    for w in (inputs.random_case(7, 200, 2, 9, 12, 12, 12), inputs.random_case(8, 200, 2, 9, 3, 12, 12),
              inputs.random_case(9, 300, 2, 1, 3, 15, 40)):
        g, infos, bad = run_parity(w, method="mspe", precision="mixed")
        assert not bad, bad[:3]


def test_mspe_mixed_agrees_with_fp64():
    # the 8-d workload's shape on a sample: the two precisions choose the same designs except
    # where a step is a near-tie within FP64 rounding, and kernel (c) gives the same values
    w = inputs.smooth_8d(T=64)
    f = gpu_predict(w, "mspe", "fp64")
    m = gpu_predict(w, "mspe", "mixed")
    assert (m["status"] == 0).all()
    same = (f["idx"] == m["idx"]).all(axis=1)
    assert same.mean() >= 0.95, same.mean()
    rel = np.abs(f["s2"][same] - m["s2"][same]) / f["s2"][same]
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed")])
def test_smooth_8d_full_size_sampled(method, precision):
    # the 8-d workload in the benchmark's launch configuration (10000 locations, n = 100,
    # 2000 candidates); the oracle checks a seeded sample
    w = inputs.smooth_8d()
    locs = np.random.default_rng(9).choice(w.T, size=10, replace=False)
    g, infos, bad = run_parity(w, locs=locs, method=method, precision=precision)
    assert not bad, bad[:3]


# ----------------------------------------------------------------- largest sizes

@pytest.mark.parametrize("method,precision", [("alc", "fp64"), ("alc", "mixed"), ("mspe", "fp64"),
                                              ("mspe", "mixed")])
def test_largest_candidate_count_parity(method, precision):
    # 8192 candidates, the largest accepted: the mixed MSPE kernel runs without its row ring
    # here (its shared memory would not fit)
    w = inputs.random_case(31, 9000, 2, 2, 6, 40, 8192, d=0.2)
    g, infos, bad = run_parity(w, method=method, precision=precision)
    assert not bad, bad[:3]


@pytest.mark.parametrize("method", ["alc", "mspe"])
def test_largest_design_and_candidate_count_run(method):
    # n = 256 and 8192 candidates (both limits): both precisions run, and the mixed designs
    # and values agree with the FP64 ones (the oracle would take minutes here)
    w = inputs.random_case(32, 9000, 2, 2, 6, 256, 8192, d=0.2, g=1e-4)
    f = gpu_predict(w, method, "fp64")
    m = gpu_predict(w, method, "mixed")
    assert (f["status"] == 0).all() and (m["status"] == 0).all()
    assert np.array_equal(f["idx"][:, :w.n0], m["idx"][:, :w.n0])
    same = (f["idx"] == m["idx"]).all(axis=1)
    rel = np.abs(f["s2"][same] - m["s2"][same]) / f["s2"][same]
    assert same.any() and rel.max() <= 1e-9, (same, rel)


def test_mixed_shared_factor_row_instance_parity():
    # n = 180 with 4000 candidates: the per-warp copies of the factor row would leave no
    # room for the row ring, so the mixed kernel runs its instance with one shared copy
    w = inputs.random_case(33, 9000, 2, 2, 6, 180, 4000, d=0.2)
    g, infos, bad = run_parity(w, precision="mixed")
    assert not bad, bad[:3]


@pytest.mark.parametrize("method", ["alc", "mspe"])
def test_rescore_count_on_exact_ties(method):
    # a location at the centre of a symmetric grid: mirror-image candidates have equal
    # scores, so the mixed screen must hand steps to the FP64 re-score; the count is that
    # of the last call on the workspace, at most one per location and greedy step, and the
    # designs still pass the protocol
    torch = _torch()
    g1 = np.linspace(-1.0, 1.0, 31)
    a, b = np.meshgrid(g1, g1, indexing="ij")
    X = np.stack([a.ravel(), b.ravel()], 1)
    Z = np.sin(2.0 * X[:, 0]) * np.cos(X[:, 1])
    XX = np.array([[0.0, 0.0], [1.0 / 30.0, 1.0 / 30.0], [0.5, 0.0], [-1.0 / 3.0, 1.0 / 3.0]])
    import types
    w = types.SimpleNamespace(X=X, Z=Z, XX=XX, n0=6, n=30, ncand=200, d=0.02, g=1e-6, T=4, p=2)
    cand = gpu_knn(X, XX, w.ncand)
    out = {k: torch.empty(w.T, dtype=torch.float64, device="cuda") for k in ("mean", "s2", "var")}
    idx = torch.empty((w.T, w.n), dtype=torch.int32, device="cuda")
    st = torch.empty(w.T, dtype=torch.int8, device="cuda")
    ws = lagp.workspace(lagp.lagp_select_workspace_bytes(w.T, 2, w.n, w.ncand, method, "mixed"))
    lagp.lagp_select_dev(dev(X, torch.float64), dev(Z, torch.float64), dev(XX, torch.float64),
                         dev(cand, torch.int32), w.n0, w.n, w.d, w.g, method, "mixed", out["mean"],
                         out["s2"], out["var"], idx, st, ws)
    torch.cuda.synchronize()
    count = lagp.lagp_select_rescore_count(ws, method, "mixed")
    assert 1 <= count <= w.T * (w.n - w.n0), count
    assert lagp.lagp_select_rescore_count(ws, method, "fp64") == 0
    assert (st.cpu().numpy() == 0).all()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    gi = idx.cpu().numpy()
    ocand = oracle.knn(X, XX, w.ncand)
    assert np.array_equal(cand, ocand)
    for t in range(w.T):
        info = check_location(w, t, ocand[t], gi[t], g["mean"][t], g["s2"][t], method,
                              gpu_var=g["var"][t])
        assert info["ok_vals"], info
