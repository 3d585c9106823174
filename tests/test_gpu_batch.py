"""GPU checks of batched solves (cg_batch_*) against the FP64 oracle.

Every (system, right-hand side) pair must stop on the true FP64 residual
(||b - A x|| <= tol ||b||, checked again with the oracle's SpMV) and lie
within the error bound the arithmetic gives against the oracle's FP64 CG
solution: ||x - x_ref|| <= (||r_x|| + ||r_ref||) / lambda_lb with
lambda_lb = 1e-2 min(M_L) <= lambda_min(A) (K is positive semidefinite).
Batched results must also be bitwise reproducible and independent of the
other systems in the batch (the same system solved alone gives the same
bits).
"""
import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()
    return torch.device("cuda:0")


_SYS = {}


def systems(n=10, emin=4, emax=14):
    key = (n, emin, emax)
    if key not in _SYS:
        _SYS[key] = problems.batch_systems(n, emin, emax, seed0=1000)
    return _SYS[key]


def stacked(sys_list, nrhs):
    return np.concatenate([s["B"][:nrhs] for s in sys_list], axis=1)


def check_pairs(sys_list, X, res, nrhs, precond=0):
    off = 0
    for si, s in enumerate(sys_list):
        A, n = s["A"], s["A"].n
        lam_lb = 1e-2 * s["mass"].min()
        for r in range(nrhs):
            rr = res[si * nrhs + r]
            b = s["B"][r]
            x = X[r, off:off + n]
            assert rr.status == gbcg.CG_OK, (si, r, rr.status)
            assert rr.relres <= TOL
            true = np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)
            assert true <= 1.05 * TOL, (si, r, true)
            ref = oracle.cg(A, b, tol=TOL, precond=precond)
            r_ref = np.linalg.norm(b - oracle.spmv(A, ref["x"]))
            assert np.linalg.norm(x - ref["x"]) <= (true * np.linalg.norm(b) + r_ref) / lam_lb
        off += n


@pytest.mark.parametrize("values,precond,nrhs", [
    (gbcg.CG_VALUES_FP32, 0, 4), (gbcg.CG_VALUES_FP32, 1, 4), (gbcg.CG_VALUES_BF16, 1, 4),
    (gbcg.CG_VALUES_FP32, 1, 1), (gbcg.CG_VALUES_FP32, 0, 3)])
def test_batch_matches_oracle(dev, values, precond, nrhs):
    sl = systems()
    with gbcg.BatchSolver([s["A"] for s in sl], inner_values=values, precond=precond) as bs:
        B = torch.from_numpy(stacked(sl, nrhs)).to(dev).contiguous()
        X = torch.zeros_like(B)
        rc, res, ms = bs.solve(B, X, TOL)
        assert rc == gbcg.CG_OK
        check_pairs(sl, X.cpu().numpy(), res, nrhs, precond)


def test_batch_reproducible_and_independent_of_neighbours(dev):
    sl = systems()
    with gbcg.BatchSolver([s["A"] for s in sl], precond=1) as bs:
        B = torch.from_numpy(stacked(sl, 4)).to(dev).contiguous()
        X1 = torch.zeros_like(B)
        X2 = torch.zeros_like(B)
        bs.solve(B, X1, TOL)
        bs.solve(B, X2, TOL)
        assert torch.equal(X1, X2)
    # the third system alone
    s = sl[2]
    off = sum(x["A"].n for x in sl[:2])
    with gbcg.BatchSolver([s["A"]], precond=1) as one:
        B1 = torch.from_numpy(np.ascontiguousarray(s["B"][:4])).to(dev)
        X3 = torch.zeros_like(B1)
        rc, res, ms = one.solve(B1, X3, TOL)
        assert rc == gbcg.CG_OK
        check_pairs([s], X3.cpu().numpy(), res, 4, 1)


def test_batch_edge_cases(dev):
    sl = systems(4)
    empty = problems.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    mats = [sl[0]["A"], empty, sl[1]["A"]]
    n = sum(m.n for m in mats)
    with gbcg.BatchSolver(mats, precond=1) as bs:
        Bn = np.zeros((2, n))
        Bn[0, :sl[0]["A"].n] = sl[0]["B"][0]
        Bn[1, :sl[0]["A"].n] = sl[0]["B"][1]
        # second system's right-hand sides stay 0: x = 0
        B = torch.from_numpy(Bn).to(dev)
        X = torch.ones_like(B)
        rc, res, ms = bs.solve(B, X, TOL)
        Xh = X.cpu().numpy()
        off = sl[0]["A"].n
        assert np.all(Xh[:, off:] == 0.0)
        assert all(r.status == gbcg.CG_OK for r in res)
        Bn[0, 3] = np.nan
        rc, res, ms = bs.solve(torch.from_numpy(Bn).to(dev), torch.zeros_like(B), TOL)
        assert res[0].status == gbcg.CG_ENAN and rc != gbcg.CG_OK


def test_batch_tuner_and_async(dev):
    sl = systems(6)
    with gbcg.BatchSolver([s["A"] for s in sl], precond=1) as bs:
        B = torch.from_numpy(stacked(sl, 4)).to(dev).contiguous()
        X = torch.zeros_like(B)
        rc, choice = bs.tune(B, X, TOL)
        assert rc == gbcg.CG_OK and choice.trials == 24 and choice.best_ms > 0
        assert choice.lanes_per_row in (1, 2, 4) and choice.gather_tiles in (0, 1)
        assert torch.count_nonzero(X) == 0  # the tuner leaves X alone
        assert bs.enqueue(B, X, TOL) == gbcg.CG_OK
        rc, res = bs.results(4)
        assert rc == gbcg.CG_OK
        check_pairs(sl, X.cpu().numpy(), res, 4, 1)


def test_batch_graph_capture_replay_matches_oracle(dev):
    """cg_batch_enqueue makes no host synchronization and allocates nothing,
    so one enqueue is captured into a CUDA graph on the handle's stream; two
    replays from x0 = 0 must each give pairs that pass the oracle checks."""
    sl = systems(6)
    stream = torch.cuda.Stream()
    with gbcg.BatchSolver([s["A"] for s in sl], precond=1, stream=stream) as bs:
        B = torch.from_numpy(stacked(sl, 4)).to(dev).contiguous()
        X = torch.zeros_like(B)
        torch.cuda.synchronize()
        assert bs.enqueue(B, X, TOL) == gbcg.CG_OK   # once outside the capture
        rc, res = bs.results(4)
        assert rc == gbcg.CG_OK
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            rcq = bs.enqueue(B, X, TOL)
        assert rcq == gbcg.CG_OK
        for _ in range(2):
            X.zero_()
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                g.replay()
            rc, res = bs.results(4)
            assert rc == gbcg.CG_OK
            check_pairs(sl, X.cpu().numpy(), res, 4, 1)
        del g


@pytest.mark.parametrize("split", [0, 1], ids=["resplit", "static"])
@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("gather", [0, 1], ids=["window", "gather"])
def test_batch_tuning_choices_match_oracle(dev, lanes, gather, split):
    """Every point the tuner can choose (tile kind x lanes per row of the
    inner SpMM), with the inner loop re-splitting the active tiles or keeping
    the creation-time split, applied with cg_batch_set_tuning, gives pairs
    that pass the oracle checks; invalid choices are refused."""
    sl = systems(5)
    with gbcg.BatchSolver([s["A"] for s in sl], precond=1) as bs:
        bs.set_tuning(3e-3, gather, lanes, split)
        B = torch.from_numpy(stacked(sl, 4)).to(dev).contiguous()
        X = torch.zeros_like(B)
        rc, res, ms = bs.solve(B, X, TOL)
        assert rc == gbcg.CG_OK
        check_pairs(sl, X.cpu().numpy(), res, 4, 1)
        for bad in (gbcg.cg_batch_tuning(inner_tol=3e-3, gather_tiles=0, lanes_per_row=3),
                    gbcg.cg_batch_tuning(inner_tol=0.0, gather_tiles=0, lanes_per_row=1),
                    gbcg.cg_batch_tuning(inner_tol=1e-3, gather_tiles=2, lanes_per_row=1),
                    gbcg.cg_batch_tuning(inner_tol=1e-3, gather_tiles=0, lanes_per_row=1, static_split=2)):
            assert gbcg.cg_batch_set_tuning(bs.h, bad) == gbcg.CG_EINVAL
