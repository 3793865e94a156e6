"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks an oracle function against something other than itself: an
independent numpy computation of the paper's definitions (np.linalg), a closed form, a
finite difference, a brute-force search or a Monte Carlo expectation.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs


def corrmat(A, B, d):
    D2 = ((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)
    return np.exp(-D2 / d)


def Kdesign(Xd, d, g):
    K = corrmat(Xd, Xd, d)
    np.fill_diagonal(K, 1.0 + g)
    return K


def np_pred(Xd, Y, x, d, g):
    """Eqs. predgp, preds2 by np.linalg.solve: mean, s2 (df = j), v, psi."""
    K = Kdesign(Xd, d, g)
    k = corrmat(x[None, :], Xd, d)[0]
    Ki_Y = np.linalg.solve(K, Y)
    Ki_k = np.linalg.solve(K, k)
    psi = Y @ Ki_Y
    v = 1.0 + g - k @ Ki_k
    return k @ Ki_Y, psi * v / len(Y), v, psi


def small_design(seed=0, j=12, p=2, d=0.3, g=1e-4):
    rng = np.random.default_rng(seed)
    Xd = rng.uniform(0, 1, size=(j, p))
    Y = np.sin(3 * Xd[:, 0]) + Xd[:, 1] ** 2
    x = rng.uniform(0.2, 0.8, size=p)
    xc = rng.uniform(0, 1, size=p)
    return Xd, Y, x, xc, d, g


# ---------------------------------------------------------------- kNN (Sec. 3, Sec. 6)

@pytest.mark.parametrize("p", [1, 2, 5])
def test_knn_equals_full_lexsort(p):
    rng = np.random.default_rng(p)
    X = np.round(rng.uniform(0, 1, size=(700, p)), 2)   # rounding creates exact ties
    XX = np.round(rng.uniform(0, 1, size=(9, p)), 2)
    cand, d2 = oracle.knn(X, XX, 80, with_d2=True)
    for t in range(XX.shape[0]):
        diff = XX[t][None, :] - X
        dd = np.zeros(X.shape[0])
        for k in range(p):           # same summation order as the definition
            dd = dd + diff[:, k] * diff[:, k]
        order = np.lexsort((np.arange(X.shape[0]), dd))[:80]
        assert np.array_equal(cand[t], order)
        assert np.array_equal(d2[t], dd[order])


def test_nn_rule_is_the_nearest_n():
    w = inputs.random_case(3, 400, 2, 5, 6, 30, 100)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        r = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "nn")
        assert np.array_equal(r["idx"], cand[t][: w.n])


# ---------------------------------------------------------------- linear algebra

def test_cholesky_and_inverse_against_numpy():
    Xd, Y, x, xc, d, g = small_design(j=20, g=1e-6)
    K = Kdesign(Xd, d, g)
    st, L = oracle.chol(K)
    assert st == 0
    assert np.allclose(L, np.linalg.cholesky(K), rtol=1e-9, atol=1e-12)
    Ki = oracle.inverse(K)
    kappa = np.linalg.cond(K)
    assert np.max(np.abs(K @ Ki - np.eye(20))) <= 50 * kappa * 2.2e-16
    assert np.allclose(Ki, np.linalg.inv(K), rtol=kappa * 1e-14, atol=0)


def test_cholesky_reports_not_pd():
    K = np.array([[1.0, 2.0], [2.0, 1.0]])
    st, _ = oracle.chol(K)
    assert st == oracle.NOT_PD


@pytest.mark.parametrize("g", [1e-2, 1e-4, 1e-6])
def test_partitioned_inverse_equals_direct_inverse(g):
    """SM Sec. 1 (Barnett): sequentially updated K_j^{-1} equals the direct inverse."""
    rng = np.random.default_rng(1)
    Xd = rng.uniform(0, 1, size=(15, 2))
    d = 0.4
    Ki = np.linalg.inv(Kdesign(Xd[:3], d, g))
    for j in range(3, 15):
        k = corrmat(Xd[j:j + 1], Xd[:j], d)[0]
        Ki = oracle.pinv_update(Ki, k, 1.0 + g)
        direct = np.linalg.inv(Kdesign(Xd[:j + 1], d, g))
        kappa = np.linalg.cond(Kdesign(Xd[:j + 1], d, g))
        assert np.max(np.abs(Ki - direct)) <= kappa * 1e-13 * np.max(np.abs(direct))


def test_partitioned_inverse_sign_reading():
    """With g = +K^{-1}k/v (the main text's sign) the bordered inverse is wrong; the SM's
    g = -K^{-1}k/v is right.  The oracle follows the SM."""
    Xd, Y, x, xc, d, g = small_design(j=6)
    K = Kdesign(Xd, d, g)
    Ki = np.linalg.inv(K)
    k = corrmat(xc[None, :], Xd, d)[0]
    v = 1 + g - k @ Ki @ k
    gp = +Ki @ k / v
    wrong = np.block([[Ki + np.outer(gp, gp) * v, gp[:, None]], [gp[None, :], np.array([[1 / v]])]])
    K1 = np.block([[K, k[:, None]], [k[None, :], np.array([[1 + g]])]])
    right = oracle.pinv_update(Ki, k, 1 + g)
    assert np.allclose(right @ K1, np.eye(7), atol=1e-8)
    assert not np.allclose(wrong @ K1, np.eye(7), atol=1e-2)


# ---------------------------------------------------------------- ALC (Eq. dxy, SM dxy2)

@pytest.mark.parametrize("seed", range(6))
def test_alc_three_forms_agree_and_are_nonnegative(seed):
    Xd, Y, x, xc, d, g = small_design(seed=seed, j=10, g=1e-5)
    closed, dxy, brute = oracle.alc_forms(Xd, x, xc, d, g)
    # independent numpy brute force: v_j(x) - v_{j+1}(x) by solves
    _, _, vj, _ = np_pred(Xd, np.ones(len(Xd)), x, d, g)
    _, _, vj1, _ = np_pred(np.vstack([Xd, xc]), np.ones(len(Xd) + 1), x, d, g)
    ref = vj - vj1
    # the subtraction v_j - v_{j+1} loses about kappa(K_{j+1}) eps absolutely
    kappa = np.linalg.cond(Kdesign(np.vstack([Xd, xc]), d, g))
    atol = 10 * kappa * 2.2e-16
    assert closed >= 0 and dxy >= -atol and ref >= -atol
    for val in (closed, dxy, brute):
        assert abs(val - ref) <= 1e-8 * abs(ref) + atol


def test_alc_expanded_form_needs_the_sm_sign():
    """Eq. dxy with the main text's g = +K^{-1}k/v disagrees with the direct reduction."""
    Xd, Y, x, xc, d, g = small_design(seed=3, j=8, g=1e-4)
    K = Kdesign(Xd, d, g)
    Ki = np.linalg.inv(K)
    kx = corrmat(x[None, :], Xd, d)[0]
    kc = corrmat(xc[None, :], Xd, d)[0]
    kxc = corrmat(x[None, :], xc[None, :], d)[0, 0]
    v = 1 + g - kc @ Ki @ kc
    gplus = Ki @ kc / v
    plus = (kx @ gplus) ** 2 * v + 2 * (kx @ gplus) * kxc + kxc ** 2 / v
    closed = oracle.alc_forms(Xd, x, xc, d, g)[0]
    assert abs(plus - closed) > 1e-3 * abs(closed)


def brute_force_alc_path(w, t, cand):
    """Greedy ALC by brute force: at each step invert every K_{j+1} (np.linalg)."""
    x = w.XX[t]
    design = list(cand[: w.n0])
    pool = list(cand[w.n0:])
    for j in range(w.n0, w.n):
        best, bestv = None, np.inf
        for c in pool:
            Xd = w.X[design + [c]]
            _, _, v, _ = np_pred(Xd, np.ones(len(Xd)), x, w.d, w.g)
            if v < bestv:
                best, bestv = c, v
        design.append(best)
        pool.remove(best)
    return np.array(design)


def test_alc_selection_matches_brute_force_tiny():
    w = inputs.random_case(21, 150, 2, 6, 3, 12, 40, d=0.2, g=1e-4)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        r = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        assert np.array_equal(r["idx"], brute_force_alc_path(w, t, cand[t])), t


def test_variance_at_x_is_nonincreasing_along_the_design():
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX[:10], w.ncand)
    for t in range(10):
        r = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        vx = r["trace"][:, 5]
        assert np.all(np.diff(vx) <= 1e-15)
        assert np.all(r["trace"][:, 1] >= 0)   # ALC reductions are non-negative


# ---------------------------------------------------------------- predictive equations

def test_predictive_equations_match_direct_solve():
    w = inputs.random_case(5, 500, 3, 8, 5, 25, 120, d=0.5, g=1e-6)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        r = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        Xd, Y = w.X[r["idx"]], w.Z[r["idx"]]
        mu, s2, v, psi = np_pred(Xd, Y, w.XX[t], w.d, w.g)
        kappa = np.linalg.cond(Kdesign(Xd, w.d, w.g))
        tol = max(1e-10, kappa * 1e-15)
        assert abs(r["mean"] - mu) <= tol * max(abs(mu), 1e-3)
        assert abs(r["s2"] - s2) <= tol * s2 * 10
        assert abs(r["var"] - s2 * w.n / (w.n - 2)) <= tol * s2 * 10


def test_n_equals_N_reproduces_the_full_gp():
    """Sec. 3: as n -> N the local predictor is the full-data GP (Eqs. predgp, preds2)."""
    rng = np.random.default_rng(2)
    N = 60
    X = rng.uniform(-1, 1, size=(N, 2))
    Z = np.cos(2 * X[:, 0]) * X[:, 1]
    x = np.array([0.1, -0.2])
    d, g = 0.7, 1e-5
    cand = oracle.knn(X, x[None, :], N)[0]
    for method in ("alc", "nn", "mspe"):
        r = oracle.local_design(X, Z, x, cand, 4, N, d, g, method)
        mu, s2, _, _ = np_pred(X, Z, x, d, g)
        assert abs(r["mean"] - mu) <= 1e-8 * abs(mu), method
        assert abs(r["s2"] - s2) <= 1e-7 * s2, method
        m2, s22 = oracle.full_gp(X, Z, x, d, g)
        assert abs(m2 - mu) <= 1e-8 * abs(mu) and abs(s22 - s2) <= 1e-7 * s2


# ---------------------------------------------------------------- likelihood and MSPE pieces

def np_loglik(Xd, Y, d, g):
    K = Kdesign(Xd, d, g)
    _, logdet = np.linalg.slogdet(K)
    psi = Y @ np.linalg.solve(K, Y)
    return -0.5 * logdet - len(Y) / 2 * np.log(psi / 2)


@pytest.mark.parametrize("seed", range(3))
def test_loglik_derivatives_match_finite_differences(seed):
    """Eqs. dl and d2l against central differences of Eq. gpk."""
    Xd, Y, x, xc, d, g = small_design(seed=seed, j=15, g=1e-3)
    l, dl, d2l = oracle.loglik(Xd, Y, d, g)
    assert abs(l - np_loglik(Xd, Y, d, g)) <= 1e-9 * abs(l)
    h = 1e-4 * d
    lp, lm = np_loglik(Xd, Y, d + h, g), np_loglik(Xd, Y, d - h, g)
    fd1 = (lp - lm) / (2 * h)
    fd2 = (lp - 2 * np_loglik(Xd, Y, d, g) + lm) / h ** 2
    assert abs(dl - fd1) <= 1e-6 * max(abs(dl), 1.0)
    assert abs(d2l - fd2) <= 1e-4 * max(abs(d2l), 1.0)


@pytest.mark.parametrize("seed", range(3))
def test_predictive_derivatives_match_finite_differences(seed):
    """SM Eqs. dmu, dV, d2V (and dz, d2z, d2w behind them) vs central differences."""
    Xd, Y, x, xc, d, g = small_design(seed=seed, j=12, g=1e-4)
    j = len(Y)
    mu, dmu, d2mu, V, dV, d2V, v, psi = oracle.pred_derivs(Xd, Y, xc, d, g)

    def mv(th):
        m, _, vv, ps = np_pred(Xd, Y, xc, th, g)
        return m, ps * vv / (j - 2)

    m0, V0 = mv(d)
    assert abs(mu - m0) <= 1e-9 * abs(m0) and abs(V - V0) <= 1e-8 * V0
    h = 1e-4 * d
    (mp, Vp), (mm, Vm) = mv(d + h), mv(d - h)
    assert abs(dmu - (mp - mm) / (2 * h)) <= 1e-5 * max(abs(dmu), 1e-3)
    assert abs(dV - (Vp - Vm) / (2 * h)) <= 1e-5 * max(abs(dV), V0)
    assert abs(d2mu - (mp - 2 * m0 + mm) / h ** 2) <= 1e-3 * max(abs(d2mu), 1.0)
    assert abs(d2V - (Vp - 2 * V0 + Vm) / h ** 2) <= 1e-3 * max(abs(d2V), V0)


def test_dV_sign_reading():
    """The main text's first term of dV/dtheta carries +Y^T K^-1 Kdot-cal Y; the SM's
    Eq. dV gives Y^T dw v = -w^T Kdot w v.  Only the minus sign matches a finite
    difference."""
    Xd, Y, x, xc, d, g = small_design(seed=1, j=12, g=1e-4)
    j = len(Y)
    _, _, _, V, dV, _, v, psi = oracle.pred_derivs(Xd, Y, xc, d, g)
    K = Kdesign(Xd, d, g)
    r2 = ((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)
    Kd = corrmat(Xd, Xd, d) * r2 / d ** 2
    np.fill_diagonal(Kd, 0.0)
    w = np.linalg.solve(K, Y)
    flip = dV + 2 * (w @ Kd @ w) * v / (j - 2)   # dV with the first term's sign flipped
    h = 1e-4 * d
    fd = []
    for th in (d + h, d - h):
        m, _, vv, ps = np_pred(Xd, Y, xc, th, g)
        fd.append(ps * vv / (j - 2))
    fd = (fd[0] - fd[1]) / (2 * h)
    assert abs(dV - fd) <= 1e-5 * abs(fd)
    assert abs(flip - fd) > 1e-2 * abs(fd)


@pytest.mark.parametrize("seed", range(3))
def test_information_recursion_matches_direct(seed):
    """SM Eq. d2lx: F_{j+1} = F_j - l''_j(y_{j+1}) equals -l'' on D_{j+1} (Eq. d2l)."""
    Xd, Y, x, xc, d, g = small_design(seed=seed, j=14, g=1e-4)
    j = 13
    F_j = -oracle.loglik(Xd[:j], Y[:j], d, g)[2]
    F_j1 = -oracle.loglik(Xd, Y, d, g)[2]
    pd = oracle.pred_derivs(Xd[:j], Y[:j], Xd[j], d, g)
    rec = F_j - oracle.d2l_conditional(pd, Y[j], j)
    assert abs(rec - F_j1) <= 1e-6 * max(abs(F_j1), 1.0)


def test_expected_psi_update_by_monte_carlo():
    """SM: E{psi_{j+1} | Y_j} = (j-1) psi_j / (j-2) when y_{j+1} follows the Student-t
    predictive (Eqs. predgp, preds2) at x_{j+1}."""
    Xd, Y, x, xc, d, g = small_design(seed=4, j=10, g=1e-3)
    j = len(Y)
    mu, _, _, V, _, _, v, psi = oracle.pred_derivs(Xd, Y, xc, d, g)
    rng = np.random.default_rng(0)
    n_mc = 20000
    scale = np.sqrt(psi * v / j)                    # Student-t scale, df = j
    ys = mu + scale * rng.standard_t(j, size=n_mc)
    X1 = np.vstack([Xd, xc])
    psis = np.empty(n_mc)
    probe = np.array([0.5] * Xd.shape[1])
    for i in range(0, n_mc):
        psis[i] = oracle.pred_derivs(X1, np.append(Y, ys[i]), probe, d, g)[7]
    target = (j - 1) * psi / (j - 2)
    se = psis.std() / np.sqrt(n_mc)
    assert abs(psis.mean() - target) <= 4 * se


def test_mspe_without_derivative_term_ranks_as_alc():
    """Sec. 3.3: dropping the derivative term, argmin of the MSPE is argmax of ALC."""
    w = inputs.random_case(31, 400, 2, 6, 4, 20, 80, d=0.3, g=1e-5)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        a = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        m = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g,
                                oracle.MSPE_NODERIV)
        assert np.array_equal(a["idx"], m["idx"])


def test_mspe_criterion_matches_finite_difference_assembly():
    """MSPE step on a tiny case: J(c) assembled from finite differences of the
    predictive mean/variance and of the log-likelihood (Eqs. mspe, newv, G; SM Ed2la)
    picks the same candidate as the oracle's first MSPE step, and its best and
    second-best values agree with the oracle's (the finite differences are accurate to
    about 1e-7 here)."""
    w = inputs.random_case(41, 120, 2, 3, 5, 6, 30, d=0.3, g=1e-4)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        x = w.XX[t]
        r = oracle.local_design(w.X, w.Z, x, cand[t], w.n0, w.n, w.d, w.g, "mspe")
        design = list(cand[t][: w.n0])
        Xd, Y = w.X[design], w.Z[design]
        j, d, g = len(design), w.d, w.g
        h = 1e-4 * d

        def mv(Xa, Ya, xs, th):
            m, _, vv, ps = np_pred(Xa, Ya, xs, th, g)
            return m, ps * vv / (len(Ya) - 2), vv, ps

        dmu_x = (mv(Xd, Y, x, d + h)[0] - mv(Xd, Y, x, d - h)[0]) / (2 * h)
        F = -(np_loglik(Xd, Y, d + h, g) - 2 * np_loglik(Xd, Y, d, g) + np_loglik(Xd, Y, d - h, g)) / h ** 2
        _, _, _, psi = mv(Xd, Y, x, d)
        best, bestJ, Js = None, np.inf, []
        for c in cand[t][w.n0:]:
            xc = w.X[c]
            mp, Vp, _, _ = mv(Xd, Y, xc, d + h)
            mm, Vm, _, _ = mv(Xd, Y, xc, d - h)
            _, Vc, _, _ = mv(Xd, Y, xc, d)
            dmu_c, dV_c = (mp - mm) / (2 * h), (Vp - Vm) / (2 * h)
            G = F + dV_c ** 2 / (2 * Vc ** 2) + dmu_c ** 2 / Vc
            _, _, v1, _ = np_pred(np.vstack([Xd, xc]), np.ones(j + 1), x, d, g)
            J = psi / (j - 2) * v1 + dmu_x ** 2 / G
            Js.append(J)
            if J < bestJ:
                best, bestJ = c, J
        assert r["idx"][w.n0] == best, t
        first, second = np.sort(Js)[:2]
        tr = r["trace"][0]                  # best, best score, chosen, its score, second
        assert abs(tr[1] - first) <= 1e-5 * abs(first), (t, tr[1], first)
        assert abs(tr[4] - second) <= 1e-5 * abs(second), (t, tr[4], second)


def test_long_double_oracle_agrees():
    """The long-double build of the same source agrees with the FP64 oracle to the
    conditioning of the problem (it is the adjudicating reference)."""
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX[:5], w.ncand)
    for t in range(5):
        a = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        b = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc",
                                forced=a["idx"], long_double=True)
        assert abs(a["mean"] - b["mean"]) <= 1e-8 * abs(b["mean"])
        assert abs(a["s2"] - b["s2"]) <= 1e-6 * b["s2"]


# ---- local maximum-likelihood lengthscale (Sec. 4.2 step 3): pinned by the likelihood
# itself (numpy slogdet/solve), not by the derivatives the Newton iteration uses

def _mle_case(seed, n=30, p=2):
    rng = np.random.default_rng(400 + seed)
    X = rng.uniform(-1, 1, size=(n, p))
    Z = np.sin(2.0 * X[:, 0]) + 0.3 * np.cos(3.0 * X[:, -1]) + 0.01 * rng.normal(size=n)
    return X, Z, np.arange(n, dtype=np.int32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mle_maximises_the_likelihood_on_a_grid(seed):
    X, Z, idx = _mle_case(seed)
    g = 1e-4
    th, it, st = oracle.mle(X, Z, idx, 0.5, g, 1e-3, 20.0)
    assert st == oracle.OK and 1 <= it < 100
    grid = np.exp(np.linspace(np.log(1e-3), np.log(20.0), 2001))
    ll = np.array([np_loglik(X, Z, t, g) for t in grid])
    k = int(np.argmax(ll))
    # the grid's best point brackets the estimate, and nothing on the grid beats it
    assert grid[max(k - 1, 0)] <= th <= grid[min(k + 1, len(grid) - 1)]
    assert np_loglik(X, Z, th, g) >= ll.max() - 1e-9 * abs(ll.max())
    # an interior maximum: l' = 0 and l'' < 0 there
    l, dl, d2l = oracle.loglik(X, Z, th, g)
    assert abs(dl) <= 1e-6 * max(1.0, abs(d2l) * th) and d2l < 0


def test_mle_from_different_starts_agrees():
    X, Z, idx = _mle_case(5)
    ths = [oracle.mle(X, Z, idx, t0, 1e-4, 1e-3, 20.0)[0] for t0 in (0.01, 0.3, 1.0, 15.0)]
    assert max(ths) - min(ths) <= 1e-7 * max(ths), ths


def test_mle_boundary_maximum():
    X, Z, idx = _mle_case(1)
    g = 1e-4
    th_int = oracle.mle(X, Z, idx, 0.5, g, 1e-3, 20.0)[0]
    # with the interval ending below the interior maximum the likelihood still rises at
    # its upper end: the estimate is that end
    th, it, st = oracle.mle(X, Z, idx, 0.5 * th_int, g, 1e-3, 0.6 * th_int)
    assert st == oracle.OK and th == 0.6 * th_int
    assert oracle.loglik(X, Z, th, g)[1] > 0
    # and symmetrically at the lower end
    th, it, st = oracle.mle(X, Z, idx, 3.0 * th_int, g, 2.0 * th_int, 20.0)
    assert st == oracle.OK and th == 2.0 * th_int
    assert oracle.loglik(X, Z, th, g)[1] < 0


def test_mle_batch_matches_single():
    X, Z, _ = _mle_case(2, n=60)
    idx = np.stack([np.arange(i, i + 30) for i in (0, 10, 30)]).astype(np.int32)
    b = oracle.mle_batch(X, Z, idx, [0.2, 0.5, 2.0], 1e-4, 1e-3, 20.0)
    for t in range(3):
        th, it, st = oracle.mle(X, Z, idx[t], [0.2, 0.5, 2.0][t], 1e-4, 1e-3, 20.0)
        assert b["theta"][t] == th and b["iters"][t] == it and b["status"][t] == st


# ---- design augmentation from a saved start design (Sec. 6)

@pytest.mark.parametrize("method", ["alc", "mspe"])
def test_augmenting_a_prefix_reproduces_the_design(method):
    # the greedy choice depends only on the current design: growing the first n1 points of
    # a design of size n back to n reproduces it, bit for bit
    w = inputs.random_case(71, 400, 2, 3, 5, 16, 60, d=0.3, g=1e-4)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in range(w.T):
        full = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, method)
        assert full["status"] == 0
        for n1 in (w.n0, 9, w.n - 1):
            a = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], 0, w.n, w.d, w.g, method,
                                    start=full["idx"][:n1])
            assert a["status"] == 0
            assert np.array_equal(a["idx"], full["idx"])
            assert a["mean"] == full["mean"] and a["s2"] == full["s2"]


def test_augmenting_rejects_a_start_point_outside_the_candidates():
    w = inputs.random_case(72, 400, 2, 1, 5, 16, 60, d=0.3, g=1e-4)
    cand = oracle.knn(w.X, w.XX, w.ncand)[0]
    outside = np.setdiff1d(np.arange(w.N), cand)[:1]
    start = np.concatenate([cand[:4], outside]).astype(np.int32)
    r = oracle.local_design(w.X, w.Z, w.XX[0], cand, 0, w.n, w.d, w.g, "alc", start=start)
    assert r["status"] == oracle.INVALID
    dup = np.array([cand[0], cand[1], cand[0]], np.int32)
    r = oracle.local_design(w.X, w.Z, w.XX[0], cand, 0, w.n, w.d, w.g, "alc", start=dup)
    assert r["status"] == oracle.INVALID


def test_fp64_oracle_s2_error_within_the_cancellation_rounding_scale():
    # the tolerance the parity protocol grants s2 in strongly cancelling cases
    # (tests/parity.cancellation_bound) is met by the FP64 oracle itself against its
    # long-double build, at every tiny-2d location
    from tests.parity import cancellation_bound
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    worst = 0.0
    for t in range(w.T):
        o = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        ld = oracle.design_predict(w.X, w.Z, w.XX[t], o["idx"], w.d, w.g, long_double=True)
        e = abs(o["s2"] - ld[1]) / ld[1]
        worst = max(worst, e / cancellation_bound(w, w.XX[t], o["idx"]))
    assert worst <= 1.0, worst


# ---- adaptive design size: the stopping rule of Sec. 6 (ALC)

def test_stopping_rule_definition_and_monotonicity():
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in (0, 17, 55, 99):
        full = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc")
        # the ratio v_j(x)/v_{j+1}(x) of each chosen point, from the trace
        vx, sc = full["trace"][:, 5], full["trace"][:, 3]
        ratio = vx / (vx - sc)
        assert np.allclose(ratio, full["trace"][:, 6], rtol=1e-12)
        assert (ratio >= 1).all()
        prev = w.n
        for r_min in (1.0001, 1.001, 1.01, 1.1, 2.0):
            a = oracle.local_design(w.X, w.Z, w.XX[t], cand[t], w.n0, w.n, w.d, w.g, "alc",
                                    r_min=r_min)
            k = a["n_out"]
            assert a["status"] == 0 and w.n0 <= k <= prev
            prev = k
            # the first k points are the fixed-size design's; its first step below r_min is k
            assert np.array_equal(a["idx"][:k], full["idx"][:k]) and (a["idx"][k:] == -1).all()
            below = np.nonzero(ratio < r_min)[0]
            assert k == (w.n0 + below[0] if len(below) else w.n)
            # predictions are those of the k-point design
            m, s2, v = oracle.design_predict(w.X, w.Z, w.XX[t], a["idx"][:k], w.d, w.g)
            assert abs(a["mean"] - m) <= 1e-12 * abs(m) and abs(a["s2"] - s2) <= 1e-9 * s2
