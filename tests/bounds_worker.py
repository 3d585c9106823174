"""Runs the CUDA paths of the bounds-check build (GBCG_LIBRARY=check must be
set by the caller) on ragged and small cases and prints one JSON line: the
largest error of each family against the oracle (relative to its bound) and
the index faults the checked kernels counted.  Helper of test_gpu_bounds.py."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from inner_bounds import fp32, lowprec_matrix, spmv_row_bound  # noqa: E402
from paper_1107_0538_gb300 import gbcg, problems  # noqa: E402
from test_gpu_inner import SPMV_CASES  # noqa: E402

assert gbcg.LIB_PATH.endswith("libgbcg_check.so"), gbcg.LIB_PATH
dev = torch.device("cuda:0")
U = 2.0 ** -53
out = {}


def spmv_ratio(A, x, y):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    absum = np.bincount(rows, weights=np.abs(A.vals * x[A.colidx]), minlength=A.n)
    bound = 2.0 * (np.diff(A.rowptr) + 2) * U * absum
    err = np.abs(y - oracle.spmv(A, x))
    return float(np.max(np.where(err > 0, err / np.maximum(bound, 1e-300), 0.0))) if A.n else 0.0


worst = 0.0
for name, mk in SPMV_CASES.items():
    A = mk()
    x = np.random.default_rng(5).standard_normal(A.n)
    with gbcg.Solver(A) as s:
        xt = torch.from_numpy(x).to(dev)
        yt = torch.full_like(xt, float("nan"))
        s.spmv(xt, yt)
        torch.cuda.synchronize()
        worst = max(worst, spmv_ratio(A, x, yt.cpu().numpy()))
    for values, fmt in ((gbcg.CG_VALUES_FP32, oracle.FP32_FORMAT), (gbcg.CG_VALUES_BF16, oracle.BF16_FORMAT)):
        for tiled in (False, True):
            A_lo = lowprec_matrix(A, fmt)
            xl = fp32(x)
            with gbcg.Solver(A, inner_values=values, vectors_in_memory=tiled) as s:
                xt = torch.from_numpy(xl.astype(np.float32)).to(dev)
                yt = torch.full_like(xt, float("nan"))
                s.spmv_inner(xt, yt)
                err = np.abs(yt.cpu().numpy().astype(np.float64) - oracle.spmv(A_lo, xl))
                bound = spmv_row_bound(A_lo, xl)
                worst = max(worst, float(np.max(np.where(err > 0, err / np.maximum(bound, 1e-300), 0.0)))
                            if A.n else 0.0)
out["spmv_err_over_bound"] = worst

# solves through every solve kernel: the slice kernel, the tiled kernel (vectors
# in memory), the SELL memory-mode kernel (61^3 nodes), both refinement kernels
solves = []
for e, kw in ((8, {}), (8, {"vectors_in_memory": True}), (8, {"precond": 1}), (60, {}),
              (8, {"inner_values": gbcg.CG_VALUES_FP32}),
              (8, {"inner_values": gbcg.CG_VALUES_BF16, "vectors_in_memory": True, "precond": 1})):
    pr = problems.cube_blobs(e, tol=1e-8)
    with gbcg.Solver(pr.A, **kw) as s:
        b = torch.from_numpy(pr.b).to(dev)
        x = torch.zeros_like(b)
        info = s.solve(b, x, tol=pr.tol)
        xs = x.cpu().numpy()
        solves.append({"e": e, "kw": str(kw), "status": info.status, "plan": s.plan()["slice_solve"],
                       "relres_true": float(np.linalg.norm(pr.b - oracle.spmv(pr.A, xs)) / np.linalg.norm(pr.b))})
out["solves"] = solves

# the batched kernel, both tile kinds
sl = problems.batch_systems(3, 5, 9, seed0=1000)
batch = []
for gather in (0, 1):
    with gbcg.BatchSolver([s["A"] for s in sl], precond=1) as bs:
        bs.set_tuning(1e-3, gather, 2)
        B = torch.from_numpy(np.concatenate([s["B"] for s in sl], axis=1)).to(dev).contiguous()
        X = torch.zeros_like(B)
        rc, res, ms = bs.solve(B, X, 1e-8)
        batch.append(rc)
out["batch"] = batch

# the learned preconditioner applied once and one flexible-CG solve
inst = problems.learn_instance(8, 20001)
net = gbcg.Net(problems.learn_init_params())
with gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED) as s:
    s.set_learned(net, inst.grid, inst.lognu.astype(np.float32))
    r = torch.from_numpy(inst.b).to(dev)
    z = torch.empty_like(r)
    s.precond_apply(r, z)
    x = torch.zeros_like(r)
    info = s.solve(r, x, tol=1e-8)
    out["learned_status"] = info.status
net.close()
torch.cuda.synchronize()
out["faults"] = gbcg.cg_bounds_faults()
print(json.dumps(out))
