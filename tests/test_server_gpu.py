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


def _w_at(w, x, n, ncand):
    """The workload view of one served location for the parity protocol."""
    import types
    return types.SimpleNamespace(X=w.X, Z=w.Z, XX=np.asarray(x, np.float64)[None, :], n0=w.n0, n=n,
                                 ncand=ncand, d=w.d, g=w.g)


@pytest.mark.parametrize("method,precision", [("alc", "mixed"), ("mspe", "mixed"), ("alc", "fp64")])
def test_served_results_match_the_oracle(method, precision):
    # a mix of concurrent requests; a seeded sample of the served locations goes through the
    # parity protocol against the CPU oracle
    import oracle
    from tests.parity import check_location
    ws, descs = _designs()
    srv = lagp.Server(descs, method, precision, nmax=64, ncand_max=400, max_batch=2048,
                      memory_budget=2 << 30, max_slots=3)
    try:
        rng = np.random.default_rng(31)
        reqs = []
        for _ in range(12):
            d = int(rng.integers(0, 3))
            L = int(rng.integers(1, 200))
            n = max(int(rng.choice([20, 40])), ws[d].n0)
            ncand = int(rng.integers(n, 401))
            x = rng.uniform(0, 1, size=(L, ws[d].p))
            reqs.append((srv.submit(d, x, n, ncand), d, x, n, ncand))
        checked = 0
        for rid, d, x, n, ncand in reqs:
            assert srv.wait(rid, 60000)
            got = srv.results(rid)
            assert (got["status"] == 0).all()
            for l in rng.choice(len(x), size=min(3, len(x)), replace=False):
                wl = _w_at(ws[d], x[l], n, ncand)
                cand = oracle.knn(ws[d].X, wl.XX, ncand)[0]
                info = check_location(wl, 0, cand, got["idx"][l], got["mean"][l], got["s2"][l], method,
                                      gpu_var=got["var"][l])
                assert info["ok_vals"], info
                checked += 1
        assert checked >= 30
    finally:
        srv.close()


def test_server_cancel_queued_and_in_flight_requests():
    # one slot, batches capped at the first request's size: later requests queue behind it
    ws, descs = _designs()
    srv = lagp.Server(descs, "alc", "mixed", nmax=64, ncand_max=800, max_batch=4096,
                      memory_budget=4 << 30, max_slots=1)
    try:
        rng = np.random.default_rng(5)
        xa = rng.uniform(0, 1, size=(4096, 8))
        xb = rng.uniform(0, 1, size=(100, 8))
        xc = rng.uniform(0, 1, size=(57, 8))
        a = srv.submit(2, xa, 64, 800)
        b = srv.submit(2, xb, 30, 300)
        c = srv.submit(2, xc, 30, 300)
        assert srv.cancel(b) == lagp.LAGP_OK
        for r in (a, b, c):
            assert srv.wait(r, 120000)
        assert srv.try_results(b)[0] == lagp.LAGP_ERR_CANCELLED
        code_a, ra = srv.try_results(a)
        code_c, rc = srv.try_results(c)
        assert code_a == 0 and code_c == 0
        # the cancelled request's place went to the next one, whose results are unaffected
        for got, (x, n, m) in ((ra, (xa, 64, 800)), (rc, (xc, 30, 300))):
            ref = _uniform(descs[2], ws[2], x, n, m, "mixed")
            assert np.array_equal(got["idx"], ref["idx"])
            assert np.array_equal(got["mean"], ref["mean"]) and np.array_equal(got["s2"], ref["s2"])
        st = srv.stats()
        assert st["slots"] == 1 and st["last_error"] == 0
        assert st["locations"] == 4096 + 57          # the cancelled request was not served
        # a request cancelled right after submission (queued, or already in a batch on the
        # GPU) completes as cancelled either way; the next request is served
        d = srv.submit(2, xa, 64, 800)
        assert srv.cancel(d) == lagp.LAGP_OK
        e = srv.submit(2, xc, 30, 300)
        assert srv.wait(d, 120000) and srv.wait(e, 120000)
        assert srv.try_results(d)[0] == lagp.LAGP_ERR_CANCELLED
        code_e, re_ = srv.try_results(e)
        assert code_e == 0 and np.array_equal(re_["idx"], rc["idx"])
        # nothing left to cancel: unknown and completed requests are refused
        assert srv.cancel(10 ** 9) == lagp.LAGP_ERR_INVALID_ARG
        f = srv.submit(2, xc, 30, 300)
        assert srv.wait(f, 120000)
        assert srv.cancel(f) == lagp.LAGP_ERR_INVALID_ARG
        assert srv.try_results(f)[0] == 0
    finally:
        srv.close()


def test_server_injected_batch_error_reaches_only_its_request():
    # a failure of the batched call, injected on the host (no GPU fault): the request whose
    # batch failed gets the code from results and stats reports it; the requests before and
    # after it are served
    ws, descs = _designs()
    srv = lagp.Server(descs, "alc", "mixed", nmax=64, ncand_max=800, max_batch=4096,
                      memory_budget=4 << 30, max_slots=1)
    try:
        rng = np.random.default_rng(6)
        xa = rng.uniform(0, 1, size=(4096, 8))
        xe = rng.uniform(0, 1, size=(64, 8))
        xf = rng.uniform(0, 1, size=(33, 8))
        a = srv.submit(2, xa, 64, 800)
        e = srv.submit(2, xe, 30, 300)
        assert srv.inject_error(e, lagp.LAGP_ERR_CUDA) == lagp.LAGP_OK
        f = srv.submit(2, xf, 30, 300)
        for r in (a, e, f):
            assert srv.wait(r, 120000)
        assert srv.try_results(e)[0] == lagp.LAGP_ERR_CUDA
        assert srv.stats()["last_error"] == lagp.LAGP_ERR_CUDA
        for r, (x, n, m) in ((a, (xa, 64, 800)), (f, (xf, 30, 300))):
            code, got = srv.try_results(r)
            assert code == 0 and (got["status"] == 0).all()
            ref = _uniform(descs[2], ws[2], x, n, m, "mixed")
            assert np.array_equal(got["idx"], ref["idx"]) and np.array_equal(got["mean"], ref["mean"])
        # the hook refuses what it cannot mark: a finished request, a non-negative code
        assert srv.inject_error(f, lagp.LAGP_ERR_CUDA) == lagp.LAGP_ERR_INVALID_ARG
        g = srv.submit(2, xf, 30, 300)
        assert srv.inject_error(g, 0) == lagp.LAGP_ERR_INVALID_ARG
        assert srv.wait(g, 120000) and srv.try_results(g)[0] == 0
    finally:
        srv.close()


def test_server_admission_by_memory_budget():
    # slots = memory budget / bytes of one slot: a budget of exactly one slot serves
    # overlapping submissions one batch at a time (they queue, none fails); below one slot
    # the server is refused
    ws, descs = _designs()
    kw = dict(nmax=40, ncand_max=300, max_batch=512)
    slot = lagp.lagp_server_slot_bytes(descs, "alc", "mixed", **kw)
    assert slot > 0
    with pytest.raises(lagp.LagpError) as ei:
        lagp.Server(descs, "alc", "mixed", memory_budget=slot - 1, max_slots=4, **kw)
    assert ei.value.code == lagp.LAGP_ERR_OOM
    two = lagp.Server(descs, "alc", "mixed", memory_budget=2 * slot, max_slots=4, **kw)
    assert two.stats()["slots"] == 2
    two.close()
    srv = lagp.Server(descs, "alc", "mixed", memory_budget=slot, max_slots=4, **kw)
    try:
        assert srv.stats()["slots"] == 1
        reqs, lock = [], threading.Lock()

        def client(seed):
            r = np.random.default_rng(seed)
            for _ in range(12):
                d = int(r.integers(0, 3))
                L = int(r.integers(1, 512))
                n = max(int(r.choice([20, 40])), ws[d].n0)
                ncand = int(r.integers(n, 301))
                x = r.uniform(0, 1, size=(L, ws[d].p))
                i = srv.submit(d, x, n, ncand)
                with lock:
                    reqs.append((i, d, x, n, ncand))

        th = [threading.Thread(target=client, args=(s,)) for s in (11, 12, 13)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for k, (i, d, x, n, ncand) in enumerate(reqs):
            assert srv.wait(i, 120000)
            code, got = srv.try_results(i)
            assert code == 0 and (got["status"] == 0).all()
            if k % 5 == 0:
                ref = _uniform(descs[d], ws[d], x, n, ncand, "mixed")
                assert np.array_equal(got["idx"], ref["idx"]) and np.array_equal(got["s2"], ref["s2"])
        st = srv.stats()
        assert st["last_error"] == 0 and st["max_inflight"] == 1 and st["batches"] >= 2
    finally:
        srv.close()
