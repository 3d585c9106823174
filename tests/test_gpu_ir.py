"""GPU checks of the mixed-precision solve (FP32/BF16 inner CG + FP64
iterative refinement) against the FP64 oracle.

Bar: the solve stops on the true FP64 residual, so ||b - A x|| <= tol ||b||
must hold (checked again with the oracle's SpMV).  The error against the
oracle's FP64 CG solution is bounded from the arithmetic: A = K + s M_L with
K positive semidefinite, so lambda_min(A) >= s min(M_L) (Weyl) and
||x - x_ref|| <= (||b - A x|| + ||b - A x_ref||) / (s min(M_L)).  A
residual-based stop leaves the smooth, near-constant mode (eigenvalue ~1e-8)
loosely determined, so refinement and plain CG may differ there by far more
than their residuals suggest; the bound above is what both runs guarantee.
The refinement must actually refine (>= 2 steps with rounded values) and
need about as many steps as the oracle's refinement.
"""
import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_CACHE = {}


def problem(name):
    if name not in _CACHE:
        _CACHE[name] = {"small": lambda: problems.cube_blobs(8, tol=1e-10),
                        "c2": lambda: problems.cube_blobs(50),
                        "c3": lambda: problems.cube_blobs(100)}[name]()
    return _CACHE[name]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()
    return torch.device("cuda:0")


def solve(A, b, dev, tol, values, precond=0, **kw):
    with gbcg.Solver(A, precond=precond, inner_values=values, **kw) as s:
        bt = torch.from_numpy(b).to(dev)
        xt = torch.zeros_like(bt)
        info = s.solve(bt, xt, tol=tol)
        return xt.cpu().numpy(), info


def true_relres(A, b, x):
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("precond", [0, 1])
@pytest.mark.parametrize("values", [gbcg.CG_VALUES_FP32, gbcg.CG_VALUES_BF16], ids=["fp32", "bf16"])
@pytest.mark.parametrize("name", ["small", "c2"])
def test_refinement_reaches_fp64_accuracy(dev, name, values, precond):
    pr = problem(name)
    x, info = solve(pr.A, pr.b, dev, pr.tol, values, precond)
    assert info.status == gbcg.CG_OK, gbcg.cg_strerror(info.status)
    assert info.outer >= 2 and info.iters > 0
    assert info.relres <= pr.tol and info.relres_true <= pr.tol
    assert true_relres(pr.A, pr.b, x) <= 1.05 * pr.tol
    ref = oracle.cg(pr.A, pr.b, tol=pr.tol, precond=precond)
    lam_lb = 1e-2 * pr.mass.min()
    r_gpu = np.linalg.norm(pr.b - oracle.spmv(pr.A, x))
    r_ref = np.linalg.norm(pr.b - oracle.spmv(pr.A, ref["x"]))
    assert np.linalg.norm(x - ref["x"]) <= (r_gpu + r_ref) / lam_lb


@pytest.mark.parametrize("values", [gbcg.CG_VALUES_FP32, gbcg.CG_VALUES_BF16], ids=["fp32", "bf16"])
def test_refinement_tiled_kernel(dev, values):
    """vectors_in_memory selects the tiled refinement kernel (the default
    handles run the SELL-32 one): same accuracy bar on the 50^3 system."""
    pr = problem("c2")
    x, info = solve(pr.A, pr.b, dev, pr.tol, values, 1, vectors_in_memory=True)
    assert info.status == gbcg.CG_OK and info.outer >= 2
    assert info.relres_true <= pr.tol and true_relres(pr.A, pr.b, x) <= 1.05 * pr.tol
    ref = oracle.cg(pr.A, pr.b, tol=pr.tol, precond=1)
    lam_lb = 1e-2 * pr.mass.min()
    r_gpu = np.linalg.norm(pr.b - oracle.spmv(pr.A, x))
    r_ref = np.linalg.norm(pr.b - oracle.spmv(pr.A, ref["x"]))
    assert np.linalg.norm(x - ref["x"]) <= (r_gpu + r_ref) / lam_lb


@pytest.mark.parametrize("values,fmt", [(gbcg.CG_VALUES_FP32, oracle.FP32_FORMAT),
                                        (gbcg.CG_VALUES_BF16, oracle.BF16_FORMAT)], ids=["fp32", "bf16"])
def test_refinement_steps_match_oracle(dev, values, fmt):
    """The oracle's refinement (FP64 inner CG on the same rounded matrix) and
    the GPU's (FP32 inner CG) need about the same number of corrections."""
    pr = problem("small")
    lo = oracle.lowprec_values(pr.A, fmt)
    inner_tol = 1e-3 if values == gbcg.CG_VALUES_FP32 else 1e-2
    ref = oracle.cg_ir(pr.A, lo, pr.b, tol=pr.tol, inner_tol=inner_tol, max_outer=60)
    x, info = solve(pr.A, pr.b, dev, pr.tol, values)
    assert ref["status"] == oracle.OK and info.status == gbcg.CG_OK
    assert abs(info.outer - ref["outer"]) <= 2


@pytest.mark.parametrize("values", [gbcg.CG_VALUES_FP32, gbcg.CG_VALUES_BF16], ids=["fp32", "bf16"])
def test_refinement_large(dev, values):
    pr = problem("c3")
    x, info = solve(pr.A, pr.b, dev, pr.tol, values, 1)
    assert info.status == gbcg.CG_OK and info.relres_true <= pr.tol
    assert true_relres(pr.A, pr.b, x) <= 1.05 * pr.tol
    assert np.linalg.norm(x - pr.xstar) / np.linalg.norm(pr.xstar) <= 1e-4


def test_refinement_edge_cases(dev):
    pr = problem("small")
    x, info = solve(pr.A, np.zeros(pr.A.n), dev, 1e-8, gbcg.CG_VALUES_FP32)
    assert info.status == gbcg.CG_OK and np.all(x == 0) and info.outer == 0
    x, info = solve(pr.A, pr.b, dev, 1e-14, gbcg.CG_VALUES_BF16, max_outer=1)
    assert info.status == gbcg.CG_ENOCONV and info.outer == 1
    b = pr.b.copy()
    b[3] = np.inf
    x, info = solve(pr.A, b, dev, 1e-8, gbcg.CG_VALUES_FP32)
    assert info.status == gbcg.CG_ENAN
