"""The cluster form of the mixed ALC kernel (a thread-block cluster of several CTAs per
location, each CTA holding a share of the candidates) against the one-CTA form and the
oracle (needs a GPU).

Every candidate's arithmetic is the same in both forms and the argmax is merged with the
same tie rule, so designs and outputs must be bitwise identical.  The cluster size and
the row ring are forced through the library's launch-shape overrides."""
from __future__ import annotations

import contextlib
import os

import numpy as np
import pytest

import oracle
from paper_1303_0383_gb300 import inputs, lagp
from tests.parity import check_location
from tests.test_adaptive_gpu import gpu_adaptive
from tests.test_augment_gpu import gpu_augment
from tests.test_parity_gpu import gpu_predict

pytestmark = pytest.mark.gpu


@contextlib.contextmanager
def shape(cluster=None, ring=None):
    old = {k: os.environ.get(k) for k in ("LAGP_MIX_CLUSTER", "LAGP_MIX_RING")}
    try:
        for k, v in (("LAGP_MIX_CLUSTER", cluster), ("LAGP_MIX_RING", ring)):
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = str(v)
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _same(a, b, what):
    for k in ("idx", "mean", "s2", "var", "status"):
        assert np.array_equal(a[k], b[k]), (what, k)


def _cut(w, T):
    w.XX = np.ascontiguousarray(w.XX[:T])
    return w


@pytest.mark.parametrize("cl", [2, 4, 8])
def test_cluster_form_is_bitwise_the_one_cta_form_tiny_2d(cl):
    w = inputs.tiny_2d()
    with shape(1):
        ref = gpu_predict(w, "alc", "mixed")
    with shape(cl):
        got = gpu_predict(w, "alc", "mixed")
    _same(got, ref, cl)


@pytest.mark.parametrize("p,M,n0,n,cl", [(3, 333, 4, 30, 2), (3, 333, 4, 30, 8), (1, 97, 3, 20, 4),
                                         (8, 501, 5, 40, 4)])
def test_cluster_form_ragged_candidate_counts(p, M, n0, n, cl):
    # candidate counts that leave the last CTA of a cluster part-filled or empty
    w = inputs.random_case(200 + p, 2500, p, 37, n0, n, M, d=0.25 * p, g=1e-6)
    with shape(1):
        ref = gpu_predict(w, "alc", "mixed")
    with shape(cl):
        got = gpu_predict(w, "alc", "mixed")
    _same(got, ref, (p, M, cl))


def test_cluster_form_paper_2d_against_one_cta_and_oracle():
    w = _cut(inputs.paper_2d(), 480)
    with shape(1):
        ref = gpu_predict(w, "alc", "mixed")
    for cl in (2, 4):
        with shape(cl):
            got = gpu_predict(w, "alc", "mixed")
        _same(got, ref, cl)
    cand = oracle.knn(w.X, w.XX, w.ncand)
    for t in np.random.default_rng(3).choice(w.T, size=16, replace=False):
        info = check_location(w, t, cand[t], got["idx"][t], got["mean"][t], got["s2"][t], "alc",
                              gpu_var=got["var"][t])
        assert info["ok_vals"], info


@pytest.mark.parametrize("ring", [0, 1])
def test_cluster_form_8d_with_and_without_row_ring(ring):
    w = _cut(inputs.smooth_8d(), 120)
    with shape(1):
        ref = gpu_predict(w, "alc", "mixed")
    with shape(4, ring):
        got = gpu_predict(w, "alc", "mixed")
    _same(got, ref, ring)


def test_cluster_form_edge_cases():
    # no greedy step (n0 == n), and a pool that runs out exactly (ncand == n)
    for w in (inputs.random_case(7, 300, 2, 9, 12, 12, 40), inputs.random_case(8, 300, 2, 9, 3, 12, 12)):
        with shape(1):
            ref = gpu_predict(w, "alc", "mixed")
        for cl in (2, 8):
            with shape(cl):
                got = gpu_predict(w, "alc", "mixed")
            _same(got, ref, cl)


def test_cluster_form_adaptive_and_augmented_designs():
    w = inputs.tiny_2d()
    cand = oracle.knn(w.X, w.XX, w.ncand)
    with shape(1):
        ref = gpu_adaptive(w, cand, "mixed", 1.01)
        full = gpu_predict(w, "alc", "mixed")
        aref = gpu_augment(w, cand, np.ascontiguousarray(full["idx"][:, :20]), "alc", "mixed")
    with shape(2):
        got = gpu_adaptive(w, cand, "mixed", 1.01)
        aug = gpu_augment(w, cand, np.ascontiguousarray(full["idx"][:, :20]), "alc", "mixed")
    for k in ("idx", "n_out", "mean", "s2", "var", "status"):
        assert np.array_equal(got[k], ref[k]), k
    _same(aug, aref, "augment")
    _same(aug, full, "augment vs full")
