"""Parity at the full workload sizes, in the launch configuration the bench
times.

* The batch of 256 uneven Q1 boxes (edges U{20..80}, 4 source-current
  right-hand sides each, FP32 inner CG with Jacobi and FP64 refinement to
  relative residual 1e-8): the autotuner's choice on the first 32 systems
  applied to the whole batch, one plain solve, then the enqueue captured in a
  CUDA graph and replayed.  The oracle cannot solve 1024 pairs in seconds, so
  every pair is checked through what holds at any size (its status, the
  residual the kernel reports, and the true FP64 residual recomputed with the
  oracle's SpMV), the replay must reproduce the plain solve bit for bit, and
  the pairs of the three smallest systems are compared with the oracle's FP64
  Jacobi-PCG under the error bound ||x - x_ref|| <= (||r_x|| + ||r_ref||) /
  lambda_lb, lambda_lb = 1e-2 min(M_L) <= lambda_min(A).
* The learned preconditioner on the 100^3 instance (1030301 nodes): z = M r
  against the oracle's network element by element (normwise BF16 bar 3e-2,
  as for the small grids), and flexible CG to relative residual 1e-8 checked
  on the true FP64 residual.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from oracle import learn as OL
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 1e-8
NSYS, EMIN, EMAX, SEED0, NRHS = 256, 20, 80, 1000, 4


@pytest.fixture(scope="module", autouse=True)
def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()


def _batch():
    # system i depends only on seed SEED0 + i, so one task per system gives
    # the same systems as problems.batch_systems(NSYS, EMIN, EMAX, SEED0)
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda i: problems.batch_systems(1, EMIN, EMAX, seed0=SEED0 + i)[0], range(NSYS)))


def _check_against_oracle_cg(s, X, off, res0):
    A, n = s["A"], s["A"].n
    lam_lb = 1e-2 * s["mass"].min()
    for r in range(NRHS):
        b = s["B"][r]
        x = X[r, off:off + n]
        r_x = np.linalg.norm(b - oracle.spmv(A, x))
        ref = oracle.cg(A, b, tol=TOL, precond=1)
        assert ref["status"] == 0
        r_ref = np.linalg.norm(b - oracle.spmv(A, ref["x"]))
        err = np.linalg.norm(x - ref["x"])
        assert err <= (r_x + r_ref) / lam_lb, (res0, r, err)


def test_batch_256_boxes_graph_replay_matches_oracle():
    sl = _batch()
    sizes = [s["A"].n for s in sl]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    assert max(sizes) <= 81 ** 3 and min(sizes) >= 21 ** 3
    stream = torch.cuda.Stream()
    # the tuner on the first 32 systems, as the bench runs it
    sub = sl[:32]
    with gbcg.BatchSolver([s["A"] for s in sub], inner_values=gbcg.CG_VALUES_FP32,
                          precond=gbcg.CG_PRECOND_JACOBI) as tb:
        Bt = torch.from_numpy(np.concatenate([s["B"] for s in sub], axis=1)).to(DEV).contiguous()
        rc, ch = tb.tune(Bt, torch.zeros_like(Bt), TOL)
        assert rc == gbcg.CG_OK and ch.trials == 24
        choice = (ch.inner_tol, ch.gather_tiles, ch.lanes_per_row)
        del Bt
    with gbcg.BatchSolver([s["A"] for s in sl], inner_values=gbcg.CG_VALUES_FP32,
                          precond=gbcg.CG_PRECOND_JACOBI, stream=stream) as bs:
        bs.set_tuning(*choice)
        B = torch.from_numpy(np.concatenate([s["B"] for s in sl], axis=1)).to(DEV).contiguous()
        X = torch.zeros_like(B)
        torch.cuda.synchronize()
        rc, res1, _ = bs.solve(B, X, TOL)
        assert rc == gbcg.CG_OK, choice
        X1 = X.cpu().numpy()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            rcq = bs.enqueue(B, X, TOL)
        assert rcq == gbcg.CG_OK
        X.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            g.replay()
        rc, res = bs.results(NRHS)
        assert rc == gbcg.CG_OK
        Xh = X.cpu().numpy()
        del g, B, X
    torch.cuda.empty_cache()
    assert len(res) == NSYS * NRHS
    # the replay reproduces the plain solve bit for bit
    assert np.array_equal(Xh, X1)
    assert [(r.iters, r.outer) for r in res] == [(r.iters, r.outer) for r in res1]
    # every pair: status, reported and true FP64 residual
    worst = 0.0
    for i, s in enumerate(sl):
        for r in range(NRHS):
            rr = res[i * NRHS + r]
            assert rr.status == gbcg.CG_OK and rr.relres <= TOL, (i, r, rr.status, rr.relres, choice)
            b = s["B"][r]
            x = Xh[r, offs[i]:offs[i + 1]]
            true = np.linalg.norm(b - oracle.spmv(s["A"], x)) / np.linalg.norm(b)
            worst = max(worst, true)
            assert true <= 1.05 * TOL, (i, r, true, choice)
    # the three smallest systems against the oracle's FP64 Jacobi-PCG
    for i in sorted(range(NSYS), key=lambda k: sizes[k])[:3]:
        _check_against_oracle_cg(sl[i], Xh, offs[i], i)


def _theta(seed):
    # parameters as the small-grid tests draw them: BF16-representable, gate
    # weights and biases of order one so that the gates vary over the grid
    rng = np.random.default_rng(seed)
    th = problems.learn_init_params(seed=seed, noise=0.3).astype(np.float64)
    th[OL.N_W1 + OL.N_W2:OL.N_W1 + OL.N_W2 + OL.N_WG] = 0.5 * rng.standard_normal(OL.N_WG)
    th[-OL.CH:] = rng.standard_normal(OL.CH)
    return problems.bf16_representable(th)


def test_learned_apply_and_fcg_100cube():
    inst = problems.learn_instance(100, 20000)
    g = inst.grid
    shape = (g.ez + 1, g.ey + 1, g.ex + 1)
    assert inst.A.n == 101 ** 3
    th = _theta(5)
    net = gbcg.Net(th.astype(np.float32))
    s = gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED)
    try:
        s.set_learned(net, g, inst.lognu.astype(np.float32))
        rt = torch.tensor(inst.b, device=DEV)
        zt = torch.zeros_like(rt)
        s.precond_apply(rt, zt)
        z = zt.cpu().numpy()
        lognu32 = inst.lognu.astype(np.float32).astype(np.float64)
        ref = OL.apply(th, inst.b, OL.diagonal(inst.A), lognu32, shape)
        rel = float(np.linalg.norm(z - ref) / np.linalg.norm(ref))
        assert rel <= 3e-2, rel
        assert np.dot(z, inst.b) > 0
        x = torch.zeros_like(rt)
        info = s.solve(rt, x, TOL)
        assert info.status == gbcg.CG_OK, info.status
        xh = x.cpu().numpy()
        true = np.linalg.norm(inst.b - oracle.spmv(inst.A, xh)) / np.linalg.norm(inst.b)
        assert true <= 1.05 * TOL, true
        assert info.relres_true <= 1.05 * TOL
    finally:
        s.close()
        net.close()
