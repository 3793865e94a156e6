"""Concurrent host calls on one resident design (needs a GPU): lagp_predict takes its device
block from the library's pool on the calling thread's stream and only reads the design, so
calls from several threads at once -- mixing ALC in both precisions and MSPE, whose kernels
then share the SMs (the mixed screens' tensor-memory instances among them) -- must each return
exactly what the same call returns alone."""
from __future__ import annotations

import threading

import numpy as np
import pytest

from paper_1303_0383_gb300 import inputs, lagp

pytestmark = pytest.mark.gpu


def test_concurrent_predict_calls_on_one_design_match_the_calls_alone():
    w = inputs.paper_2d()
    d = lagp.Design(w.X, w.Z)
    try:
        jobs = [(w.XX[0:400], "alc", "mixed"), (w.XX[400:800], "alc", "mixed"),
                (w.XX[800:1000], "alc", "fp64"), (w.XX[1000:1200], "mspe", "mixed")]
        alone = [d.predict(np.ascontiguousarray(x), w.n0, w.n, w.ncand, w.d, w.g, m, p)
                 for x, m, p in jobs]
        got = [[None] * 3 for _ in jobs]
        errors = []

        def run(k):
            x, m, p = jobs[k]
            try:
                for r in range(3):
                    got[k][r] = d.predict(np.ascontiguousarray(x), w.n0, w.n, w.ncand, w.d, w.g, m, p)
            except Exception as e:  # reported below, after every thread has finished
                errors.append(repr(e))

        threads = [threading.Thread(target=run, args=(k,)) for k in range(len(jobs))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for k in range(len(jobs)):
            assert (alone[k]["status"] == 0).all()
            for r in range(3):
                for key in ("idx", "mean", "s2", "var", "status"):
                    assert np.array_equal(got[k][r][key], alone[k][key]), (k, r, key)
    finally:
        d.close()
