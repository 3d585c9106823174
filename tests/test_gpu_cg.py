"""GPU parity of the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (derived from the arithmetic of each check):
  * SpMV, per row: |y - y_ref| <= 2 (m + 2) u sum_j |a_ij x_j|, m the row
    length, u = 2^-53 (the bound for two different summation orders of m terms).
  * CG iterates at a fixed iteration count k before the loss of orthogonality
    sets in (every k used here): relative 2-norm difference <= 1e-10.
  * Full solves on the 20^3 uniform cube: relative difference <= 1e-10 and
    iteration counts within +-2.
  * Full solves on the contrast-1e3 cubes, where rounding order alone moves the
    count by ~1%: both meet the tolerance, iteration counts within
    max(2, 2%), and |x - x_oracle| <= 2 |x_oracle - x*| (both within the
    error ball the stop test allows).
"""
import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()
    return torch.device("cuda:0")


_CACHE = {}


def problem(name):
    if name not in _CACHE:
        if name == "c1":
            _CACHE[name] = problems.cube_uniform(20)
        elif name == "c2":
            _CACHE[name] = problems.cube_blobs(50)
        elif name == "c3":
            _CACHE[name] = problems.cube_blobs(100)
        elif name == "c55":
            _CACHE[name] = problems.cube_blobs(55)
        elif name == "small":
            _CACHE[name] = problems.cube_blobs(7, contrast=1e2, tol=1e-10)
    return _CACHE[name]


def oracle_full(name, precond=0):
    key = ("full", name, precond)
    if key not in _CACHE:
        pr = problem(name)
        _CACHE[key] = oracle.cg(pr.A, pr.b, tol=pr.tol, precond=precond)
    return _CACHE[key]


def gpu_solve(A, b, dev, tol, maxit=0, precond=0, x0=None, **kw):
    with gbcg.Solver(A, precond=precond, **kw) as s:
        bt = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
        xt = torch.zeros_like(bt) if x0 is None else torch.from_numpy(np.array(x0, dtype=np.float64)).to(dev)
        info = s.solve(bt, xt, tol=tol, maxit=maxit)
        return xt.cpu().numpy(), info


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def check_spmv(A, x, y):
    ref = oracle.spmv(A, x)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    absum = np.bincount(rows, weights=np.abs(A.vals * x[A.colidx]), minlength=A.n)
    m = np.diff(A.rowptr)
    bound = 2.0 * (m + 2) * U * absum
    err = np.abs(y - ref)
    assert np.all(err <= bound), (err.max(), np.argmax(err - bound))


# ------------------------------------------------------------------ SpMV

def ragged_csr(n, seed, long_rows=(), long_len=0, empty=(), unsorted=False, dup=False):
    rng = np.random.default_rng(seed)
    rowptr = [0]
    cols, vals = [], []
    for i in range(n):
        if i in empty:
            m = 0
        elif i in long_rows:
            m = long_len
        else:
            m = int(rng.integers(1, 60))
        c = rng.choice(n, size=min(m, n), replace=False) if m else np.zeros(0, int)
        if not unsorted:
            c = np.sort(c)
        if dup and m > 2:
            c = np.concatenate([c, c[:2]])
        cols.extend(c.tolist())
        vals.extend(rng.standard_normal(len(c)).tolist())
        rowptr.append(len(cols))
    return problems.CSR(n, np.array(rowptr, np.int32), np.array(cols, np.int32), np.array(vals))


SPMV_CASES = {
    "n1": lambda: problems.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0])),
    "tail129": lambda: ragged_csr(129, 1),
    "empty_rows": lambda: ragged_csr(700, 2, empty=set(range(0, 700, 7)) | {699}),
    "long_row": lambda: ragged_csr(9000, 3, long_rows={4500}, long_len=8999),
    "two_long_rows": lambda: ragged_csr(6000, 4, long_rows={0, 5999}, long_len=4097),
    "unsorted_dups": lambda: ragged_csr(1000, 5, unsorted=True, dup=True),
    "tile_limit_rows": lambda: ragged_csr(3000, 6, long_rows={10, 11, 12, 2999}, long_len=1024),
    "over_tile_limit": lambda: ragged_csr(3000, 7, long_rows={0, 40, 41}, long_len=1025),
    "all_empty": lambda: problems.CSR(50, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0)),
    "c1": lambda: problem("c1").A,
    "c2": lambda: problem("c2").A,
    "c3": lambda: problem("c3").A,
}


@pytest.mark.parametrize("case", list(SPMV_CASES))
def test_spmv_parity(dev, case):
    A = SPMV_CASES[case]()
    x = np.random.default_rng(11).standard_normal(A.n)
    with gbcg.Solver(A) as s:
        xt = torch.from_numpy(x).to(dev)
        yt = torch.full_like(xt, np.nan)
        s.spmv(xt, yt)
        torch.cuda.synchronize()
        check_spmv(A, x, yt.cpu().numpy())


# -------------------------------------------------------------- CG parity

@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
def test_cg_uniform_cube_full_solve(dev, mem):
    pr = problem("c1")
    ref = oracle_full("c1")
    x, info = gpu_solve(pr.A, pr.b, dev, pr.tol, vectors_in_memory=mem)
    assert ref["status"] == oracle.OK and info.status == gbcg.CG_OK
    assert abs(info.iters - ref["iters"]) <= 2
    assert rel(x, ref["x"]) <= 1e-10
    assert info.relres <= pr.tol
    assert info.relres_true <= 1.01 * pr.tol


@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
@pytest.mark.parametrize("precond,k", [(0, 200), (0, 350), (1, 150)])
def test_cg_paper_sized_fixed_k_iterates(dev, precond, k, mem):
    pr = problem("c2")
    ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=k, precond=precond)
    x, info = gpu_solve(pr.A, pr.b, dev, 0.0, maxit=k, precond=precond, vectors_in_memory=mem)
    assert info.status == gbcg.CG_ENOCONV and ref["status"] == oracle.ENOCONV
    assert info.iters == k == ref["iters"]
    assert rel(x, ref["x"]) <= 1e-10
    assert abs(info.relres - ref["relres"]) <= 1e-6 * ref["relres"]


@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
@pytest.mark.parametrize("precond", [0, 1])
def test_cg_paper_sized_full_solve(dev, precond, mem):
    pr = problem("c2")
    ref = oracle_full("c2", precond)
    x, info = gpu_solve(pr.A, pr.b, dev, pr.tol, precond=precond, vectors_in_memory=mem)
    assert ref["status"] == oracle.OK and info.status == gbcg.CG_OK
    assert abs(info.iters - ref["iters"]) <= max(2, 0.02 * ref["iters"])
    assert info.relres <= pr.tol and info.relres_true <= 1.05 * pr.tol
    true = np.linalg.norm(pr.b - oracle.spmv(pr.A, x)) / np.linalg.norm(pr.b)
    assert true <= 1.05 * pr.tol
    assert rel(x, ref["x"]) <= 2.0 * rel(ref["x"], pr.xstar)


@pytest.mark.parametrize("precond", [0, 1])
def test_cg_large_fixed_k_and_full_solve(dev, precond):
    pr = problem("c3")
    k = 40
    ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=k, precond=precond)
    x, info = gpu_solve(pr.A, pr.b, dev, 0.0, maxit=k, precond=precond)
    assert info.iters == k and rel(x, ref["x"]) <= 1e-10
    assert abs(info.relres - ref["relres"]) <= 1e-6 * ref["relres"]
    x, info = gpu_solve(pr.A, pr.b, dev, pr.tol, precond=precond)
    assert info.status == gbcg.CG_OK and info.relres_true <= 1.05 * pr.tol
    true = np.linalg.norm(pr.b - oracle.spmv(pr.A, x)) / np.linalg.norm(pr.b)
    assert true <= 1.05 * pr.tol


def test_memory_mode_sell_kernel_small(dev):
    """On 2 CTAs the 20^3 box (290 slices) is too large for the slice kernel
    and for register rows, so its solves run the SELL-32 kernel with the
    vectors in memory: iterates, a full solve and the edge cases."""
    pr = problem("c1")
    kw = dict(grid_ctas=2)
    with gbcg.Solver(pr.A, **kw) as s:
        assert s.plan()["slice_solve"] == 2 and s.plan()["ctas"] == 2
    for precond in (0, 1):
        ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=60, precond=precond)
        x, info = gpu_solve(pr.A, pr.b, dev, 0.0, maxit=60, precond=precond, **kw)
        assert info.status == gbcg.CG_ENOCONV and info.iters == 60
        assert rel(x, ref["x"]) <= 1e-10
    ref = oracle_full("c1")
    x, info = gpu_solve(pr.A, pr.b, dev, pr.tol, **kw)
    assert info.status == gbcg.CG_OK and abs(info.iters - ref["iters"]) <= 2
    assert rel(x, ref["x"]) <= 1e-10 and info.relres_true <= 1.01 * pr.tol
    x, info = gpu_solve(pr.A, np.zeros(pr.A.n), dev, 1e-8, x0=np.ones(pr.A.n), **kw)
    assert info.status == gbcg.CG_OK and info.iters == 0 and np.all(x == 0)
    x0 = ref["x"] + 1e-3
    r2 = oracle.cg(pr.A, pr.b, x0=x0, tol=pr.tol)
    x, info = gpu_solve(pr.A, pr.b, dev, pr.tol, x0=x0, **kw)
    assert abs(info.iters - r2["iters"]) <= 2 and rel(x, r2["x"]) <= 1e-10
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-10, wait_limit_s=2e-3, debug_phantom_arrivals=1, **kw)
    assert info.status == gbcg.CG_ETIMEOUT


@pytest.mark.parametrize("precond", [0, 1])
def test_cg_tiled_register_kernel_fixed_k_iterates(dev, precond):
    """A 55^3 box has more than one 32-row slice per warp, so its solves run
    the tiled kernel with rows held in registers."""
    pr = problem("c55")
    k = 120
    ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=k, precond=precond)
    with gbcg.Solver(pr.A, precond=precond) as s:
        assert s.plan()["slice_solve"] == 0 and s.plan()["reg_rows"] > 0
    x, info = gpu_solve(pr.A, pr.b, dev, 0.0, maxit=k, precond=precond)
    assert info.status == gbcg.CG_ENOCONV and info.iters == k == ref["iters"]
    assert rel(x, ref["x"]) <= 1e-10
    assert abs(info.relres - ref["relres"]) <= 1e-6 * ref["relres"]


def test_slice_kernel_with_fewer_ctas(dev):
    """grid_ctas limits the slice kernel to 31 slices per CTA: 20^3 (290
    slices) runs it on 10 CTAs and falls back to the tiled kernel on 8."""
    pr = problem("c1")
    ref = oracle.cg(pr.A, pr.b, tol=0.0, maxit=60)
    for ctas, sliced in ((10, 1), (8, 0)):
        with gbcg.Solver(pr.A, grid_ctas=ctas) as s:
            assert s.plan()["slice_solve"] == sliced and s.plan()["ctas"] == ctas
        x, info = gpu_solve(pr.A, pr.b, dev, 0.0, maxit=60, grid_ctas=ctas)
        assert info.iters == 60 and rel(x, ref["x"]) <= 1e-10


# ------------------------------------------------------------- edge cases

@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
def test_zero_rhs(dev, mem):
    pr = problem("small")
    x, info = gpu_solve(pr.A, np.zeros(pr.A.n), dev, 1e-8, x0=np.ones(pr.A.n), vectors_in_memory=mem)
    assert info.status == gbcg.CG_OK and info.iters == 0 and np.all(x == 0)


def test_nan_rhs(dev):
    pr = problem("small")
    b = pr.b.copy()
    b[5] = np.nan
    x, info = gpu_solve(pr.A, b, dev, 1e-8)
    assert info.status == gbcg.CG_ENAN


@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
def test_maxit_returns_last_iterate(dev, mem):
    pr = problem("small")
    ref = oracle.cg(pr.A, pr.b, tol=1e-14, maxit=7)
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-14, maxit=7, vectors_in_memory=mem)
    assert info.status == gbcg.CG_ENOCONV == ref["status"] and info.iters == 7
    assert rel(x, ref["x"]) <= 1e-12


def test_indefinite_breakdown(dev):
    A = problems.CSR(3, np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32),
                     np.array([1.0, -1.0, 2.0]))
    x, info = gpu_solve(A, np.array([0.0, 1.0, 0.0]), dev, 1e-12)
    assert info.status == gbcg.CG_EBREAKDOWN
    assert oracle.cg(A, np.array([0.0, 1.0, 0.0]), tol=1e-12)["status"] == oracle.EBREAKDOWN


def test_single_unknown(dev):
    A = problems.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    x, info = gpu_solve(A, np.array([2.0]), dev, 1e-12)
    assert info.status == gbcg.CG_OK and info.iters == 1 and x[0] == 0.5


@pytest.mark.parametrize("mem", [False, True], ids=["regs", "memory"])
def test_nonzero_initial_guess_and_already_converged(dev, mem):
    pr = problem("small")
    ref = oracle.cg(pr.A, pr.b, tol=1e-12)
    x0 = ref["x"] + 1e-3
    r2 = oracle.cg(pr.A, pr.b, x0=x0, tol=1e-12)
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-12, x0=x0, vectors_in_memory=mem)
    assert abs(info.iters - r2["iters"]) <= 2 and rel(x, r2["x"]) <= 1e-10
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-2, x0=ref["x"], vectors_in_memory=mem)
    assert info.status == gbcg.CG_OK and info.iters == 0


def test_empty_matrix(dev):
    A = problems.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with gbcg.Solver(A) as s:
        info = s.solve(torch.zeros(0, dtype=torch.float64, device=dev),
                       torch.zeros(0, dtype=torch.float64, device=dev), tol=1e-8)
        assert info.status == gbcg.CG_OK and info.iters == 0


def test_bounded_barrier_timeout_reports_status(dev):
    """Grid barriers that wait for a CTA that never arrives give up after the
    wait limit and report CG_ETIMEOUT; the context stays usable."""
    pr = problem("small")
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-10, wait_limit_s=2e-3, debug_phantom_arrivals=1)
    assert info.status == gbcg.CG_ETIMEOUT
    x, info = gpu_solve(pr.A, pr.b, dev, 1e-10)
    assert info.status == gbcg.CG_OK


# ----------------------------------------------------- boundary behaviour

def test_host_path_matches_device_path_bitwise(dev):
    pr = problem("c1")
    with gbcg.Solver(pr.A) as s:
        bt = torch.from_numpy(pr.b).to(dev)
        xt = torch.zeros_like(bt)
        i1 = s.solve(bt, xt, tol=pr.tol)
        xh = np.zeros(pr.A.n)
        i2 = s.solve_host(pr.b.copy(), xh, tol=pr.tol)
        assert i1.iters == i2.iters and i1.status == i2.status == gbcg.CG_OK
        assert np.array_equal(xt.cpu().numpy(), xh)


def test_deterministic_bitwise(dev):
    pr = problem("c2")
    x1, i1 = gpu_solve(pr.A, pr.b, dev, pr.tol)
    x2, i2 = gpu_solve(pr.A, pr.b, dev, pr.tol)
    assert i1.iters == i2.iters and np.array_equal(x1, x2)


def test_device_resident_csr_input(dev):
    pr = problem("small")
    A = pr.A
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    va = torch.from_numpy(A.vals).to(dev)
    c = gbcg.cg_csr(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), gbcg.CG_MEM_DEVICE)
    rc, h = gbcg.cg_create(c, None, torch.cuda.current_stream().cuda_stream)
    assert rc == gbcg.CG_OK
    try:
        bt = torch.from_numpy(pr.b).to(dev)
        xt = torch.zeros_like(bt)
        rc, info = gbcg.cg_solve(h, bt.data_ptr(), xt.data_ptr(), 1e-10, 0)
        x_host, _ = gpu_solve(A, pr.b, dev, 1e-10)
        assert rc == gbcg.CG_OK and np.array_equal(xt.cpu().numpy(), x_host)
    finally:
        gbcg.cg_destroy(h)


def test_plan_and_vector_modes(dev):
    with gbcg.Solver(problem("c3").A) as s:
        assert s.plan()["reg_rows"] == 0          # too many rows per thread
        assert s.plan()["slice_solve"] == 2       # SELL-32 with the vectors in memory
    with gbcg.Solver(problem("c2").A, vectors_in_memory=True) as s:
        assert s.plan()["reg_rows"] == 0 and s.plan()["slice_solve"] == 0
    with gbcg.Solver(problem("c55").A) as s:
        assert s.plan()["slice_solve"] == 0 and s.plan()["reg_rows"] in (1, 2, 4)
    pr = problem("c2")
    with gbcg.Solver(pr.A) as s:
        p = s.plan()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert p["slice_solve"] == (1 if (pr.A.n + 31) // 32 <= 31 * p["ctas"] else 0)
    assert p["reg_rows"] in (1, 2, 4)
    assert p["window_tiles"] == p["tiles"]  # every stencil tile stages its x-window
    assert 1 <= p["ctas"] <= sms and p["tiles"] >= p["ctas"]
    assert p["tile_nnz"] <= 896 and p["n"] == pr.A.n and p["nnz"] == pr.A.nnz


def test_solve_argument_errors(dev):
    pr = problem("small")
    with gbcg.Solver(pr.A) as s:
        bt = torch.from_numpy(pr.b).to(dev)
        rc, _ = gbcg.cg_solve(s.h, bt.data_ptr(), bt.data_ptr(), 1e-8, 0)  # b aliases x
        assert rc == gbcg.CG_EINVAL
        rc, _ = gbcg.cg_solve(s.h, bt.data_ptr(), 0, 1e-8, 0)
        assert rc == gbcg.CG_EINVAL
        rc, _ = gbcg.cg_solve(s.h, bt.data_ptr(), torch.zeros_like(bt).data_ptr(), -1.0, 0)
        assert rc == gbcg.CG_EINVAL
