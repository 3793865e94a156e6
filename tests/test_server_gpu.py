"""The continuous-batching server (lagp_server_*) through the C ABI (needs a GPU).

A request's results must be the same alone and in a mix of concurrent requests (every
location's arithmetic depends only on its own inputs), and equal to the uniform entry
point's for the same locations."""
from __future__ import annotations

import threading

import numpy as np
import pytest

from paper_1303_0383_gb300 import inputs, lagp

pytestmark = pytest.mark.gpu


def _designs():
    import torch
    ws = [inputs.random_case(41, 3000, 2, 1, 4, 10, 10, d=0.3, g=1e-6),
          inputs.random_case(42, 5000, 4, 1, 4, 10, 10, d=0.6, g=1e-6),
          inputs.random_case(43, 4000, 8, 1, 5, 10, 10, d=1.2, g=1e-4)]
    descs = [dict(X=torch.as_tensor(w.X, device="cuda"), Z=torch.as_tensor(w.Z, device="cuda"),
                  n0=w.n0, theta=w.d, g=w.g) for w in ws]
    return ws, descs


def _uniform(desc, w, XX, n, ncand, precision, method="alc"):
    import torch
    out = lagp.predict_torch(desc["X"], desc["Z"], torch.as_tensor(XX, device="cuda"), w.n0, n,
                             ncand, w.d, w.g, method, precision)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("method,precision", [("alc", "mixed"), ("alc", "fp64"), ("mspe", "mixed")])
def test_server_results_same_alone_and_in_the_mix(method, precision):
    ws, descs = _designs()
    srv = lagp.Server(descs, method, precision, nmax=64, ncand_max=400, max_batch=2048,
                      memory_budget=2 << 30, max_slots=3)
    try:
        rng = np.random.default_rng(7)
        XR = rng.uniform(0, 1, size=(37, 4))
        rid = srv.submit(1, XR, 30, 200)
        assert srv.wait(rid, 60000)
        alone = srv.results(rid)
        assert (alone["status"] == 0).all() and alone["latency_ms"] > 0
        uni = _uniform(descs[1], ws[1], XR, 30, 200, precision, method)
        assert np.array_equal(uni["idx"], alone["idx"])
        for k in ("mean", "s2", "var"):
            assert np.array_equal(uni[k], alone[k]), k
        # a mix of concurrent requests from two submitting threads, R among them
        reqs, lock = [], threading.Lock()

        def client(seed):
            r = np.random.default_rng(seed)
            for _ in range(15):
                d = int(r.integers(0, 3))
                p = ws[d].p
                L = int(r.integers(1, 300))
                n = int(r.choice([20, 40]))
                if n < ws[d].n0:
                    n = ws[d].n0
                ncand = int(r.integers(n, 401))
                x = r.uniform(0, 1, size=(L, p))
                i = srv.submit(d, x, n, ncand)
                with lock:
                    reqs.append((i, d, x, n, ncand))

        th = [threading.Thread(target=client, args=(s,)) for s in (1, 2)]
        for t in th:
            t.start()
        rid2 = srv.submit(1, XR, 30, 200)
        for t in th:
            t.join()
        for i, *_ in reqs:
            assert srv.wait(i, 60000)
        assert srv.wait(rid2, 60000)
        mixed = srv.results(rid2)
        for k in ("idx", "mean", "s2", "var", "status"):
            assert np.array_equal(mixed[k], alone[k]), k
        # spot-check some of the others against the uniform entry point
        for i, d, x, n, ncand in reqs[::6]:
            got = srv.results(i)
            ref = _uniform(descs[d], ws[d], x, n, ncand, precision, method)
            assert np.array_equal(got["idx"], ref["idx"])
            assert np.array_equal(got["mean"], ref["mean"]) and np.array_equal(got["s2"], ref["s2"])
        st = srv.stats()
        assert st["last_error"] == 0 and st["batches"] >= 2 and st["slots"] >= 1
    finally:
        srv.close()
