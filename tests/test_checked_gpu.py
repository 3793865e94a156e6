"""The checked build (-DLAGP_CHECKED, liblagp_checked.so): device-side bounds checks in the
kNN, FP64 ALC, mixed ALC and paper-form kernels that record a violation and skip the access
(needs a GPU).

A child process runs the headline paths on small cases in the checked build -- kNN up to
8192 candidates, both precisions (the tensor-memory and the row-ring instances of the mixed
screen), the paper's form, uneven batches -- and must record no violation and choose the
same designs as the normal build.  Then an out-of-range design index planted in a candidate
list must be reported with its site, index and extent: past the start design the location is
served from its other candidates, inside it the location fails (every access the planted
index could reach is one the checks guard)."""
from __future__ import annotations

import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1303_0383_gb300 import inputs, lagp

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_worker(tmp_path, checked):
    out = os.path.join(str(tmp_path), "checked_%d.npz" % checked)
    env = dict(os.environ, LAGP_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_worker.py"), out],
                       env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_records_nothing_and_matches_the_normal_build(tmp_path):
    got = _run_worker(tmp_path, True)
    ref = _run_worker(tmp_path, False)
    assert got["check/checked"] == 1 and ref["check/checked"] == 0
    assert got["check/count"] == 0, {k: got[k] for k in got if k.startswith("check/")}
    for k in ref:
        if k.startswith("check/"):
            continue
        if k.endswith("/idx") or k.endswith("/cand") or k.endswith("/status"):
            assert np.array_equal(got[k], ref[k]), k
        else:
            assert np.allclose(got[k], ref[k], rtol=1e-12, atol=0.0, equal_nan=True), k


PLANT = r'''
import sys, numpy as np, torch
sys.path.insert(0, %(root)r)
from paper_1303_0383_gb300 import inputs, lagp
from tests.checked_worker import knn, select
w = inputs.random_case(93, 3000, 2, 8, 4, 20, 200, d=0.3, g=1e-6)
cand = knn(w, w.ncand)
bad = w.N + 5
cand[2, w.ncand - 1] = bad               # past the start design: never forced into it
cand[5, 1] = bad                         # inside the start design (n0 = 4): that location fails
out = []
for method, prec, dense in (("alc", "mixed", False), ("alc", "fp64", False), ("alc", "fp64", True)):
    r = select(w, cand, method, prec, dense=dense)
    c = lagp.lagp_check_take()
    out.append((c["checked"], c["count"], c["site"], c["index"], c["bound"], int(r["status"][2]),
                int((r["idx"][2] == bad).sum()), int(r["status"][5]), int((r["idx"][5] == bad).sum()),
                int((r["status"] == 0).sum())))
print(out)
'''


def test_checked_build_reports_a_planted_design_index():
    env = dict(os.environ, LAGP_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", PLANT % {"root": ROOT}], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    rows = eval(r.stdout.strip().splitlines()[-1])
    N = 3000
    for row, want in zip(rows, (11, 24, 31)):
        checked, count, site, index, bound, status, chosen, status5, chosen5, served = row
        assert checked == 1 and count >= 2, rows
        assert (site, index, bound) == (want, N + 5, N), rows
        assert status == 0 and chosen == 0, rows                       # served without it
        assert status5 == lagp.LAGP_ERR_NOT_PD and chosen5 == 0, rows  # failed, no index out
        assert served == 7, rows                                       # the other locations
