"""The allocation-free solve, cg_solve_noalloc, against cg_solve.

cg_solve_noalloc exists for callers that may not allocate device memory (a
stream being captured into a graph, a framework whose allocator owns the
device memory, a real-time loop that cannot take an allocation's
synchronization).  It keeps its workspace in one fixed array inside the
library, shared by all calls, so this test calls it twice in a row on the
same inputs: the second call must clear what the first left behind.  Its
result must match cg_solve's within the bar the other full-solve tests use
on this system (relative difference <= 1e-10, iterations within 2), and the
device's free memory must not change across a call.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_matches_cg_solve_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    pr = problems.cube_uniform(20)  # 9261 unknowns, tol 1e-10
    A = pr.A
    b = torch.from_numpy(pr.b).to(dev)

    with gbcg.Solver(A) as s:
        x_ref = torch.zeros_like(b)
        ref = s.solve(b, x_ref, tol=pr.tol)
    assert ref.status == gbcg.CG_OK

    rowptr = torch.from_numpy(A.rowptr).to(dev)
    colidx = torch.from_numpy(A.colidx).to(dev)
    vals = torch.from_numpy(A.vals).to(dev)
    csr = gbcg.cg_csr(A.n, A.nnz, rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(),
                      gbcg.CG_MEM_DEVICE)
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
        xn = x.cpu().numpy()
        assert np.linalg.norm(xn - xr) / np.linalg.norm(xr) <= 1e-10, call
        assert info.relres <= pr.tol
        if call == 1:
            assert free_after == free_before
