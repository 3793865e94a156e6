"""The oracle's pins catch plausible mistakes (no GPU).

Each case plants one mistake in a copy of the oracle's C source -- a flipped sign, a
dropped term or factor, a transposed index, a wrong divisor, a reversed tie rule -- builds
it (FP64 and long double alike, so comparisons of the two builds share the mistake), loads
it in place of the oracle and runs every pin of test_oracle_pins.py against it.  At least
one pin must fail for every mistake.
"""
from __future__ import annotations

import inspect

import pytest

import oracle
from tests import test_oracle_pins as pins

# (what the mistake is, text in the oracle source, the mistaken text)
MUTANTS = [
    ("kNN: equal distances ordered by the larger index first",
     "return (a->idx > b->idx) - (a->idx < b->idx);",
     "return (a->idx < b->idx) - (a->idx > b->idx);"),
    ("kNN: the last coordinate left out of the distance",
     "for (int k = 0; k < p; k++) {\n    double t = a[k] - b[k];",
     "for (int k = 0; k < p - 1; k++) {\n    double t = a[k] - b[k];"),
    ("correlation exp(-r^2 / (2 theta)) instead of exp(-r^2 / theta)",
     "return R_EXP(-sqdist_r(a, b, p) / theta);",
     "return R_EXP(-sqdist_r(a, b, p) / (2 * theta));"),
    ("Cholesky: the last term of an off-diagonal sum dropped",
     "for (int m = 0; m < k; m++) t = t - L[i * j + m] * L[k * j + m];",
     "for (int m = 0; m < k - 1; m++) t = t - L[i * j + m] * L[k * j + m];"),
    ("forward substitution with the transposed factor",
     "for (int m = 0; m < i; m++) t = t - L[i * j + m] * u[m];",
     "for (int m = 0; m < i; m++) t = t - L[m * j + i] * u[m];"),
    ("nugget left off the design's diagonal",
     "W->K[a * j + b] = (a == b) ? 1 + P->g :",
     "W->K[a * j + b] = (a == b) ? 1 :"),
    ("partitioned inverse with g = +K^-1 k / v (the main text's sign)",
     "real ga = -Kk[a] / v;",
     "real ga = Kk[a] / v;"),
    ("ALC score without the division by v_j(c)",
     "real alc = cov * cov / vc;",
     "real alc = cov * cov;"),
    ("cov_j(x, c) with the wrong sign of the correction",
     "for (int a = 0; a < j; a++) cov = cov - W->ux[a] * W->u[a];",
     "for (int a = 0; a < j; a++) cov = cov + W->ux[a] * W->u[a];"),
    ("predictive scale s2 divided by n - 2 instead of n",
     "*s2 = (double)(psi * vx / n);",
     "*s2 = (double)(psi * vx / (n - 2));"),
    ("predictive variance divided by n instead of n - 2",
     "*var = (double)(psi * vx / (n - 2));",
     "*var = (double)(psi * vx / n);"),
    ("predictive mean from Y instead of L^-1 Y",
     "mu += W->ux[a] * W->yt[a];",
     "mu += W->ux[a] * W->y[a];"),
    ("MSPE: dV with the main text's + sign on its first term",
     "real dVc = (-S.wKdw * vc - S.psi * (2 * kdz - zKdz)) / dj2;",
     "real dVc = (S.wKdw * vc - S.psi * (2 * kdz - zKdz)) / dj2;"),
    ("MSPE: F_j = +l'' instead of -l''",
     "S->F = -l2;",
     "S->F = l2;"),
    ("MSPE: the factor 2 of K^-1 Kd K^-1 Kd dropped in l''",
     "(wKddw - 2 * q2)",
     "(wKddw - q2)"),
    ("MSPE: dmu_x with the wrong sign of its second term",
     "dmu += W->kdx[a] * W->w[a] - kt * W->kdw[a];",
     "dmu += W->kdx[a] * W->w[a] + kt * W->kdw[a];"),
    ("MSPE: dK/dtheta of the design divided by theta instead of theta^2",
     "W->Kd[a * j + b] = kab * r2 / (th * th);",
     "W->Kd[a * j + b] = kab * r2 / th;"),
    ("MSPE: dk_c/dtheta divided by theta instead of theta^2",
     "W->ud[a] = W->kcol[a] * r2 / (P->theta * P->theta);",
     "W->ud[a] = W->kcol[a] * r2 / P->theta;"),
    ("MSPE: G without the 1/2 of its dV^2 / V^2 term",
     "real G = S.F + dVc * dVc / (2 * Vc * Vc) + dmu_c * dmu_c / Vc;",
     "real G = S.F + dVc * dVc / (Vc * Vc) + dmu_c * dmu_c / Vc;"),
    ("l' with the wrong sign of its trace term",
     "out[1] = (double)(-0.5 * tr0 + dj / 2 * q3 / psi);",
     "out[1] = (double)(0.5 * tr0 + dj / 2 * q3 / psi);"),
    ("l'' without the factor 2 of its K^-1 Kd K^-1 Kd term",
     "dj / (2 * psi) * (q1 - 2 * q2)",
     "dj / (2 * psi) * (q1 - q2)"),
    ("MLE: l' > 0 narrows the bracket from above",
     "lo = th; lo_open = 0;",
     "hi = th; hi_open = 0;"),
    ("dz = K^-1 (kd + Kd z) instead of K^-1 (kd - Kd z)",
     "for (int a = 0; a < j; a++) t1[a] = kd[a] - t1[a];",
     "for (int a = 0; a < j; a++) t1[a] = kd[a] + t1[a];"),
    ("conditional log-likelihood with j/2 instead of (j+1)/2",
     "real h = (real)(j + 1) / 2;",
     "real h = (real)j / 2;"),
    ("Eq. dxy expanded with the wrong sign of its cross term",
     "out[1] = (double)(kg * kg * vc + 2 * kg * kxc + kxc * kxc / vc);",
     "out[1] = (double)(kg * kg * vc - 2 * kg * kxc + kxc * kxc / vc);"),
    ("stopping rule ratio v_j(x) / score instead of v_j(x) / v_{j+1}(x)",
     "vx / (vx - chosen_s)",
     "vx / chosen_s"),
    ("stopping rule stops where the ratio is above r_min",
     "if (r_min > 0 && !forced && ratio < r_min) {",
     "if (r_min > 0 && !forced && ratio > r_min) {"),
    ("saved start design accepted with a repeated point",
     "if (r < 0 || W->used[r]) return LAGP_ORC_INVALID;",
     "if (r < 0) return LAGP_ORC_INVALID;"),
    ("predictions on a given design: s2 divided by n - 2",
     "out[1] = (double)(psi * v / n);",
     "out[1] = (double)(psi * v / (n - 2));"),
]


def _pin_calls():
    """Every pin with every parameter set of its parametrize marks."""
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        sets = [{}]
        for m in getattr(fn, "pytestmark", []):
            if m.name != "parametrize":
                continue
            names = [a.strip() for a in m.args[0].split(",")]
            new = []
            for kw in sets:
                for v in m.args[1]:
                    vals = v if len(names) > 1 else (v,)
                    new.append(dict(kw, **dict(zip(names, vals))))
            sets = new
        calls += [(name, fn, kw) for kw in sets]
    return calls


def test_every_pin_passes_on_the_oracle_itself():
    for name, fn, kw in _pin_calls():
        fn(**kw)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a mistaken oracle may return NaN
@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_a_planted_mistake_fails_a_pin(what, old, new, tmp_path, monkeypatch):
    src = open(oracle._SRC).read()
    assert src.count(old) == 1, "the mistake's anchor must occur once: %r" % old
    p64, pld = oracle.build_variant(src.replace(old, new), str(tmp_path))
    monkeypatch.setitem(oracle._libs, False, oracle.load_variant(p64))
    monkeypatch.setitem(oracle._libs, True, oracle.load_variant(pld))
    caught = []
    for name, fn, kw in _pin_calls():
        try:
            fn(**kw)
        except Exception:  # an assertion, or an oracle call that now reports a failure
            caught.append(name)
    assert caught, "no pin fails with the mistake: " + what
