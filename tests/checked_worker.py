"""Child program of tests/test_checked_gpu.py: runs a fixed set of small workloads through
the library the environment selects (LAGP_CHECKED=1: the checked build) and writes their
outputs, plus the bounds-check records, to the .npz file named on the command line."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import torch  # noqa: E402

from paper_1303_0383_gb300 import inputs, lagp  # noqa: E402
from tests.test_batch_gpu import make_batch, run_batch  # noqa: E402


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def knn(w, M):
    cand = torch.empty((w.XX.shape[0], M), dtype=torch.int32, device="cuda")
    lagp.lagp_knn_dev(dev(w.X), dev(w.XX), M, cand,
                      lagp.workspace(lagp.lagp_knn_workspace_bytes(w.N, w.XX.shape[0], M)))
    return cand


def select(w, cand, method, precision, dense=False):
    T, M = cand.shape
    out = {k: torch.empty(T, dtype=torch.float64, device="cuda") for k in ("mean", "s2", "var")}
    out["idx"] = torch.empty((T, w.n), dtype=torch.int32, device="cuda")
    out["status"] = torch.empty(T, dtype=torch.int8, device="cuda")
    X, Z, XX = dev(w.X), dev(w.Z), dev(w.XX)
    if dense:
        ws = lagp.workspace(lagp.lagp_select_dense_workspace_bytes(T, w.p, w.n, M))
        lagp.lagp_select_dense_dev(X, Z, XX, cand, w.n0, w.n, w.d, w.g, out["mean"], out["s2"],
                                   out["var"], out["idx"], out["status"], ws)
    else:
        ws = lagp.workspace(lagp.lagp_select_workspace_bytes(T, w.p, w.n, M, method, precision))
        lagp.lagp_select_dev(X, Z, XX, cand, w.n0, w.n, w.d, w.g, method, precision, out["mean"],
                             out["s2"], out["var"], out["idx"], out["status"], ws)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def cut(w, T):
    w.XX = np.ascontiguousarray(w.XX[:T])
    return w


def main(path):
    res = {}
    cases = {"tiny": inputs.tiny_2d(),
             "ragged3d": inputs.random_case(91, 3000, 3, 40, 4, 30, 333, d=0.3, g=1e-6),
             "paper2d": cut(inputs.paper_2d(), 300),     # the tensor-memory instance
             "smooth8d": cut(inputs.smooth_8d(), 48),    # the row-ring instance
             "bigM": inputs.random_case(92, 20000, 2, 3, 6, 12, 8192, d=0.05, g=1e-6)}
    for name, w in cases.items():
        cand = knn(w, w.ncand)
        res[name + "/cand"] = cand.cpu().numpy()
        for method, prec in (("alc", "fp64"), ("alc", "mixed")):
            for k, v in select(w, cand, method, prec).items():
                res["%s/%s_%s/%s" % (name, method, prec, k)] = v
        if w.n <= 128:
            for k, v in select(w, cand, "alc", "fp64", dense=True).items():
                res["%s/dense/%s" % (name, k)] = v
    ws, design_of, n, M, XX = make_batch(seed=5, T=80)
    for prec in ("fp64", "mixed"):
        out = run_batch(ws, design_of, n, M, XX, "alc", prec)[0]
        for k, v in out.items():
            res["batch/%s/%s" % (prec, k)] = v
    chk = lagp.lagp_check_take()
    for k, v in chk.items():
        res["check/" + k] = np.int64(v)
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
