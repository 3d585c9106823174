"""The allocation-free solve, cg_solve_noalloc, against cg_solve and the oracle.

cg_solve_noalloc exists for callers that may not allocate device memory:
code inside a framework whose caching allocator owns the device memory,
real-time loops that cannot take the device-wide synchronization of an
allocation, plug-ins with a fixed device-memory budget.  It keeps its
workspace in one fixed array inside the library, shared by all calls, so the
first test calls it twice in a row on the same inputs: the second call must
clear what the first left behind.  Its result must match cg_solve's within
the bar the other full-solve tests use on this system (relative difference
<= 1e-10, iterations within 2), match the FP64 oracle within the same bar,
and the device's free memory must not change across a call.  The other
tests cover the statuses the kernel and the host checks give: a malformed
matrix, the iteration cap, b = 0, a nonzero x0, and host memory passed where
device memory is required.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()
    return torch.device("cuda:0")


def device_csr(A, dev, rowptr=None, colidx=None):
    """cg_csr over device copies of A's arrays (returned too, to keep them alive)."""
    rp = torch.from_numpy(np.asarray(A.rowptr if rowptr is None else rowptr, np.int32)).to(dev)
    ci = torch.from_numpy(np.asarray(A.colidx if colidx is None else colidx, np.int32)).to(dev)
    va = torch.from_numpy(np.asarray(A.vals, np.float64)).to(dev)
    return gbcg.cg_csr(A.n, A.nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), gbcg.CG_MEM_DEVICE), (rp, ci, va)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_cg_solve_on_two_calls_in_a_row(dev):
    pr = problems.cube_uniform(20)  # 9261 unknowns, tol 1e-10
    A = pr.A
    b = torch.from_numpy(pr.b).to(dev)

    with gbcg.Solver(A) as s:
        x_ref = torch.zeros_like(b)
        ref = s.solve(b, x_ref, tol=pr.tol)
    assert ref.status == gbcg.CG_OK
    orc = oracle.cg(A, pr.b, tol=pr.tol)
    assert orc["status"] == oracle.OK

    csr, keep = device_csr(A, dev)
    stream = torch.cuda.current_stream().cuda_stream
    xr = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc, info = gbcg.cg_solve_noalloc(csr, b.data_ptr(), x.data_ptr(), pr.tol, 0, stream)
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == gbcg.CG_OK == info.status, (call, gbcg.cg_strerror(rc))
        assert abs(info.iters - ref.iters) <= 2, (call, info.iters, ref.iters)
        assert abs(info.iters - orc["iters"]) <= 2, (call, info.iters, orc["iters"])
        xn = x.cpu().numpy()
        assert rel(xn, xr) <= 1e-10, call
        assert rel(xn, orc["x"]) <= 1e-10, call
        assert info.relres <= pr.tol
        if call == 1:
            assert free_after == free_before


def test_noalloc_cap_zero_rhs_and_start_vector(dev):
    """maxit = 3 gives CG_ENOCONV with the oracle's third iterate; b = 0 gives
    x = 0 after 0 iterations; a nonzero x0 gives the oracle's solve from it."""
    pr = problems.cube_blobs(7, contrast=1e2, tol=1e-10)
    A = pr.A
    csr, keep = device_csr(A, dev)
    stream = torch.cuda.current_stream().cuda_stream
    b = torch.from_numpy(pr.b).to(dev)

    x = torch.zeros_like(b)
    rc, info = gbcg.cg_solve_noalloc(csr, b.data_ptr(), x.data_ptr(), pr.tol, 3, stream)
    orc = oracle.cg(A, pr.b, tol=pr.tol, maxit=3)
    assert rc == gbcg.CG_ENOCONV == orc["status"] and info.iters == 3
    assert rel(x.cpu().numpy(), orc["x"]) <= 1e-10

    x = torch.full_like(b, 7.0)
    zero = torch.zeros_like(b)
    rc, info = gbcg.cg_solve_noalloc(csr, zero.data_ptr(), x.data_ptr(), pr.tol, 0, stream)
    assert rc == gbcg.CG_OK and info.iters == 0 and torch.count_nonzero(x) == 0

    x0 = np.random.default_rng(3).standard_normal(A.n)
    x = torch.from_numpy(x0.copy()).to(dev)
    rc, info = gbcg.cg_solve_noalloc(csr, b.data_ptr(), x.data_ptr(), pr.tol, 0, stream)
    orc = oracle.cg(A, pr.b, x0=x0, tol=pr.tol)
    assert rc == gbcg.CG_OK == orc["status"] and abs(info.iters - orc["iters"]) <= 2
    assert rel(x.cpu().numpy(), orc["x"]) <= 1e-10


@pytest.mark.parametrize("case", ["column_past_n", "rowptr_past_nnz"])
def test_noalloc_malformed_matrix_is_einval(dev, case):
    """The kernel checks every row range and column before using it; entries
    out of bounds are skipped (never read) and the call returns CG_EINVAL."""
    pr = problems.cube_blobs(6, contrast=1e2)
    A = pr.A
    rowptr, colidx = A.rowptr.copy(), A.colidx.copy()
    if case == "column_past_n":
        colidx[A.rowptr[5] + 1] = A.n + 3
    else:
        rowptr[7] = A.nnz + 50   # row 6 ends past nnz, row 7 starts after it ends
    csr, keep = device_csr(A, dev, rowptr, colidx)
    stream = torch.cuda.current_stream().cuda_stream
    b = torch.from_numpy(pr.b).to(dev)
    x = torch.zeros_like(b)
    rc, info = gbcg.cg_solve_noalloc(csr, b.data_ptr(), x.data_ptr(), 1e-8, 0, stream)
    assert rc == gbcg.CG_EINVAL == info.status
    # the context is intact: a well-formed call on the same device still solves
    good, keep2 = device_csr(A, dev)
    rc, info = gbcg.cg_solve_noalloc(good, b.data_ptr(), x.data_ptr(), 1e-8, 0, stream)
    assert rc == gbcg.CG_OK


def test_noalloc_host_vector_is_einval_before_any_launch(dev):
    pr = problems.cube_blobs(6, contrast=1e2)
    csr, keep = device_csr(pr.A, dev)
    stream = torch.cuda.current_stream().cuda_stream
    b_host = np.ascontiguousarray(pr.b)
    x = torch.zeros(pr.A.n, dtype=torch.float64, device=dev)
    rc, info = gbcg.cg_solve_noalloc(csr, b_host.ctypes.data, x.data_ptr(), 1e-8, 0, stream)
    assert rc == gbcg.CG_EINVAL
    b_pinned = torch.from_numpy(b_host).pin_memory()
    rc, info = gbcg.cg_solve_noalloc(csr, b_pinned.data_ptr(), x.data_ptr(), 1e-8, 0, stream)
    assert rc == gbcg.CG_EINVAL
    assert torch.count_nonzero(x) == 0
