"""Learned preconditioner on the GPU against the FP64 oracle (oracle/learn.py).

Bars:
* z = M r: the network runs in BF16 (inputs, gates, activations rounded to
  8 significant bits, relative error <= 2^-9 each) with FP32 accumulation;
  with the parameters BF16-representable the path has 6 such roundings in
  sequence (s_hat, g, h1, h2, k1, and g again), so the normwise error is a
  small multiple of 6 * 2^-9 = 1.2e-2: the bar is 3e-2.
* gradients: relative normwise error <= 3e-2 (the same roundings, plus the
  backward fields du, dk, dh2, da1, dag in BF16).
* flexible CG: converges to the tolerance on the true residual; with the
  Jacobi fallback the iterations match Jacobi-PCG of the oracle within 2;
  with the network, within max(3, 10%) of the oracle's FCG with the same
  parameters (its preconditioner differs by the BF16 error above).
"""
import numpy as np
import pytest

import oracle
from oracle import learn as OL
from paper_1107_0538_gb300 import gbcg, problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _theta(seed, noise=0.3, gate_scale=0.5):
    rng = np.random.default_rng(seed)
    th = P.learn_init_params(seed=seed, noise=noise).astype(np.float64)
    th[OL.N_W1 + OL.N_W2:OL.N_W1 + OL.N_W2 + OL.N_WG] = gate_scale * rng.standard_normal(OL.N_WG)
    th[-OL.CH:] = rng.standard_normal(OL.CH)
    return P.bf16_representable(th)


def _learned(inst, net, **kw):
    sw = kw.pop("stall_window", 0)
    sf = kw.pop("stall_factor", 0.0)
    s = gbcg.Solver(inst.A, precond=gbcg.CG_PRECOND_LEARNED, **kw)
    s.set_learned(net, inst.grid, inst.lognu.astype(np.float32), sw, sf)
    return s


def _lognu32(inst):
    return inst.lognu.astype(np.float32).astype(np.float64)


def _shape(inst):
    g = inst.grid
    return (g.ez + 1, g.ey + 1, g.ex + 1)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _box(ex, ey, ez, seed):
    g = P.Grid(ex, ey, ez, 1.0 / max(ex, ey, ez))
    nu = P.nu_blobs(g, seed=seed, nu_iron=1e-3)
    A, _ = P.q1_matrix(nu, g.h)
    xs = 2.0 * P.uniform01(seed + 1, A.n) - 1.0
    return P.LearnInstance(f"box{ex}x{ey}x{ez}", g, A, P.csr_times(A, xs), xs, P.node_log_nu(g, nu))


@pytest.mark.parametrize("dims", [(8, 8, 8), (5, 9, 7), (30, 20, 10), (1, 1, 1)])
def test_precond_apply_matches_oracle(dims):
    inst = _box(*dims, seed=10000 + sum(dims))
    th = _theta(5)
    net = gbcg.Net(th.astype(np.float32))
    s = _learned(inst, net)
    d = OL.diagonal(inst.A)
    for k, r in enumerate([np.random.default_rng(7).standard_normal(inst.A.n), inst.b]):
        ref = OL.apply(th, r, d, _lognu32(inst), _shape(inst))
        rt = torch.tensor(r, device=DEV)
        zt = torch.zeros_like(rt)
        s.precond_apply(rt, zt)
        z = zt.cpu().numpy()
        assert _rel(z, ref) <= 3e-2, (dims, k, _rel(z, ref))
        assert np.dot(z, r) > 0
    # r = 0 gives z = 0
    zt = torch.ones(inst.A.n, dtype=torch.float64, device=DEV)
    s.precond_apply(torch.zeros_like(zt), zt)
    assert float(zt.abs().max()) == 0.0


def test_gradient_matches_oracle():
    insts = [_box(6, 5, 7, 10001), _box(6, 5, 7, 10002)]
    th = _theta(9)
    net = gbcg.Net(th.astype(np.float32))
    solvers = [_learned(i, net) for i in insts]
    rng = np.random.default_rng(3)
    pairs_r, pairs_e, pinst = [], [], []
    for k, inst in enumerate(insts):
        S = OL.csr_matrix(inst.A).toarray()
        for _ in range(2):
            r = rng.standard_normal(inst.A.n).astype(np.float32)
            e = np.linalg.solve(S, r.astype(np.float64)).astype(np.float32)
            pairs_r.append(r)
            pairs_e.append(e)
            pinst.append(k)
    R = torch.tensor(np.stack(pairs_r), device=DEV)
    E = torch.tensor(np.stack(pairs_e), device=DEV)
    lset = gbcg.LearnSet(solvers, pinst, R, E)
    idx = np.array([0, 3, 1, 2], dtype=np.int64)
    loss, grad = net.grad(lset, idx)
    samples = []
    for j in idx:
        inst = insts[pinst[j]]
        samples.append((OL.csr_matrix(inst.A), OL.diagonal(inst.A), _lognu32(inst), _shape(inst),
                        pairs_r[j].astype(np.float64), pairs_e[j].astype(np.float64)))
    lref, gref = OL.batch_loss_grad(th, samples)
    assert abs(loss - lref) <= 3e-2 * abs(lref), (loss, lref)
    assert _rel(grad, gref) <= 3e-2, _rel(grad, gref)
    # each block of the gradient on its own
    for sl in (slice(0, OL.N_W1), slice(OL.N_W1, OL.N_W1 + OL.N_W2),
               slice(OL.N_W1 + OL.N_W2, OL.N_PARAMS - OL.CH), slice(OL.N_PARAMS - OL.CH, OL.N_PARAMS)):
        assert _rel(grad[sl], gref[sl]) <= 5e-2, (sl, _rel(grad[sl], gref[sl]))
    # the parameters did not change
    assert np.array_equal(net.params(), th.astype(np.float32))


# vectors_in_memory = False: the SpMV step and the x, r update run as one
# cooperative SELL-32 kernel; True: as the tiled SpMV and the vector kernel
PATHS = [pytest.param(False, id="sell_fused"), pytest.param(True, id="tiled")]


@pytest.mark.parametrize("vim", PATHS)
def test_zero_network_falls_back_to_jacobi_pcg(vim):
    inst = P.learn_instance(10, 20000)
    net = gbcg.Net(np.zeros(gbcg.CG_LEARN_PARAMS, dtype=np.float32))
    s = _learned(inst, net, vectors_in_memory=vim)
    b = torch.tensor(inst.b, device=DEV)
    x = torch.zeros_like(b)
    info = s.solve(b, x, 1e-8)
    ref = oracle.cg(inst.A, inst.b, tol=1e-8, precond=1)
    assert info.status == gbcg.CG_OK and info.reverted_at == 0
    assert abs(info.iters - ref["iters"]) <= 2
    assert info.relres_true <= 1.05e-8
    assert _rel(x.cpu().numpy(), ref["x"]) <= 1e-6


@pytest.mark.parametrize("vim", PATHS)
def test_learned_fcg_matches_oracle_fcg(vim):
    inst = P.learn_instance(10, 20001)
    th = P.learn_init_params(seed=11, noise=0.05)
    net = gbcg.Net(th)
    s = _learned(inst, net, vectors_in_memory=vim)
    b = torch.tensor(inst.b, device=DEV)
    x = torch.zeros_like(b)
    info = s.solve(b, x, 1e-8)
    d = OL.diagonal(inst.A)
    M = lambda v: OL.apply(th.astype(np.float64), v, d, _lognu32(inst), _shape(inst))
    ref = OL.fcg(inst.A, inst.b, M, tol=1e-8)
    assert ref["status"] == OL.OK and ref["reverted_at"] == -1
    assert info.status == gbcg.CG_OK and info.reverted_at == -1, info.as_dict()
    assert abs(info.iters - ref["iters"]) <= max(3, 0.1 * ref["iters"]), (info.iters, ref["iters"])
    assert info.relres_true <= 1.05e-8
    # A = K + 1e-2 M_L with K positive semi-definite, so lambda_min(A) >=
    # 1e-2 min(M_L) = 1e-2 h^3 / 8 and ||x - x*|| <= ||b - A x|| / lambda_min
    xg = x.cpu().numpy()
    lam = 1e-2 * inst.grid.h ** 3 / 8
    assert np.linalg.norm(xg - inst.xstar) <= np.linalg.norm(inst.b - P.csr_times(inst.A, xg)) / lam


@pytest.mark.parametrize("vim", PATHS)
def test_stall_switch_matches_oracle(vim):
    inst = P.learn_instance(10, 20002)
    th = P.learn_init_params(seed=12, noise=0.05)
    net = gbcg.Net(th)
    s = _learned(inst, net, stall_window=5, stall_factor=1e-6, vectors_in_memory=vim)
    b = torch.tensor(inst.b, device=DEV)
    x = torch.zeros_like(b)
    info = s.solve(b, x, 1e-8)
    d = OL.diagonal(inst.A)
    M = lambda v: OL.apply(th.astype(np.float64), v, d, _lognu32(inst), _shape(inst))
    ref = OL.fcg(inst.A, inst.b, M, tol=1e-8, stall_window=5, stall_factor=1e-6)
    assert ref["reverted_at"] == 5
    assert info.status == gbcg.CG_OK and info.reverted_at == 5
    assert abs(info.iters - ref["iters"]) <= 3
    assert info.relres_true <= 1.05e-8


def test_fused_barrier_timeout_reports_status():
    """The grid barrier of the fused SpMV-update kernel, made to wait for a CTA
    that never arrives, gives up after the wait limit: the solve reports
    CG_ETIMEOUT, and the next solve on the same network and context works."""
    inst = P.learn_instance(8, 20003)
    net = gbcg.Net(P.learn_init_params(seed=13))
    b = torch.tensor(inst.b, device=DEV)
    s = _learned(inst, net, wait_limit_s=2e-3, debug_phantom_arrivals=1)
    x = torch.zeros_like(b)
    info = s.solve(b, x, 1e-8)
    assert info.status == gbcg.CG_ETIMEOUT, info.as_dict()
    s.close()
    s = _learned(inst, net)
    x = torch.zeros_like(b)
    info = s.solve(b, x, 1e-8)
    assert info.status == gbcg.CG_OK and info.relres_true <= 1.05e-8


@pytest.mark.parametrize("vim", PATHS)
def test_edge_cases_and_determinism(vim):
    inst = P.learn_instance(8, 20003)
    net = gbcg.Net(P.learn_init_params(seed=13))
    s = _learned(inst, net, vectors_in_memory=vim)
    b = torch.zeros(inst.A.n, dtype=torch.float64, device=DEV)
    x = torch.ones_like(b)
    info = s.solve(b, x, 1e-8)
    assert info.status == gbcg.CG_OK and info.iters == 0 and float(x.abs().max()) == 0.0
    b = torch.tensor(inst.b, device=DEV)
    x = torch.tensor(inst.xstar, device=DEV)
    info = s.solve(b, x, 1e-8)
    assert info.status == gbcg.CG_OK and info.iters == 0
    x1 = torch.zeros_like(b)
    i1 = s.solve(b, x1, 1e-9)
    x2 = torch.zeros_like(b)
    i2 = s.solve(b, x2, 1e-9)
    assert i1.iters == i2.iters and torch.equal(x1, x2)
    x3 = torch.zeros_like(b)
    i3 = s.solve(b, x3, 1e-9, maxit=7)
    assert i3.status == gbcg.CG_ENOCONV and i3.iters == 7
    xh = np.zeros(inst.A.n)
    ih = s.solve_host(inst.b, xh, 1e-9)
    assert ih.iters == i1.iters and np.array_equal(xh, x1.cpu().numpy())


def test_training_pairs_are_consistent():
    inst = P.learn_instance(8, 10003)
    net = gbcg.Net(P.learn_init_params())
    s = _learned(inst, net)
    n = inst.A.n
    R = torch.zeros((6, n), dtype=torch.float32, device=DEV)
    E = torch.zeros_like(R)
    b = torch.tensor(inst.b, device=DEV)
    xs = torch.tensor(inst.xstar, device=DEV)
    s.learn_pairs(b, xs, 4, 6, R, E)
    Rh, Eh = R.cpu().numpy().astype(np.float64), E.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(R[0].cpu().numpy(), inst.b.astype(np.float32))
    np.testing.assert_array_equal(E[0].cpu().numpy(), inst.xstar.astype(np.float32))
    for k in range(6):
        ae = P.csr_times(inst.A, Eh[k])
        assert np.linalg.norm(ae - Rh[k]) <= 1e-5 * np.linalg.norm(inst.b)
    # residuals shrink along the restarted CG segments
    norms = np.linalg.norm(Rh, axis=1)
    assert norms[-1] < 0.5 * norms[0]
    # and match the oracle's restarted CG
    x = np.zeros(n)
    for k in range(5):
        x = oracle.cg(inst.A, inst.b, x0=x, tol=0.0, maxit=4)["x"]
    assert _rel(Eh[5], inst.xstar - x) <= 1e-4


def test_training_gains_over_jacobi():
    """Trains on small random instances with the project's kernels and checks
    that the network cuts flexible-CG iterations on unseen instances below
    Jacobi-PCG's."""
    train = [P.learn_instance(12, 10000 + i) for i in range(4)]
    net = gbcg.Net(P.learn_init_params())
    solvers = [_learned(i, net) for i in train]
    n = train[0].A.n
    per = 24
    R = torch.zeros((per * len(train), n), dtype=torch.float32, device=DEV)
    E = torch.zeros_like(R)
    for k, (inst, s) in enumerate(zip(train, solvers)):
        b = torch.tensor(inst.b, device=DEV)
        xs = torch.tensor(inst.xstar, device=DEV)
        s.learn_pairs(b, xs, 16, per, R[k * per:(k + 1) * per], E[k * per:(k + 1) * per])
    pinst = np.repeat(np.arange(len(train)), per)
    lset = gbcg.LearnSet(solvers, pinst, R, E)
    held = np.arange(0, len(pinst), 3)           # a fixed set of pairs to compare the loss on
    before, _ = net.grad(lset, held)
    steps, batch = 300, 4
    order = (P.splitmix64(77, steps * batch) % np.uint64(len(pinst))).astype(np.int64)
    losses = net.train(lset, order, steps, batch, 1e-3)
    assert np.all(np.isfinite(losses))
    after, _ = net.grad(lset, held)
    assert after < before, (before, after)
    for seed, e in ((20010, 12), (20011, 16)):
        test = P.learn_instance(e, seed)
        s = _learned(test, net)
        b = torch.tensor(test.b, device=DEV)
        x = torch.zeros_like(b)
        info = s.solve(b, x, 1e-8)
        jac = oracle.cg(test.A, test.b, tol=1e-8, precond=1)
        assert info.status == gbcg.CG_OK and info.relres_true <= 1.05e-8
        assert info.reverted_at == -1
        assert info.iters < 0.7 * jac["iters"], (e, info.iters, jac["iters"])
