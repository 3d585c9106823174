"""GPU parity of the low-precision inner path of iterative refinement, entry
by entry, against the FP64 oracle on the same rounded matrix.

Refinement corrects itself: a wrong inner SpMV, a wrong compensated diagonal
or a wrong inner beta would still reach the FP64 outer tolerance, only more
slowly, so the refinement tests alone cannot see such a mistake.  These
tests look at the inner path directly:

* the inner SpMV alone (cg_spmv_inner: y = A_lo x through the device routine
  of the handle's refinement kernel, SELL-32 slices or staged tiles) against
  oracle.spmv on oracle.lowprec_values(A, fmt), per row, within the bound of
  FP32 accumulation: |y - y_ref| <= 2 (m + 2) 2^-24 sum_j |a_ij x_j|;
* the inner CG iterate after exactly k steps (max_outer = 1, max_inner = k,
  x0 = 0, so the solution returned is the correction d_k of the first
  refinement step) against the oracle's CG on A_lo d = fl32(b) after k steps,
  for cg_irsell_kernel, cg_ir_kernel and the batched kernel (one system,
  1 to 4 right-hand sides), with and without Jacobi: element by element at
  k = 1, in the max norm at k > 1, within the bounds derived in
  inner_bounds.py.
"""
import numpy as np
import pytest

import oracle
from inner_bounds import check_inner_iterate, fp32, lowprec_matrix, spmv_row_bound
from paper_1107_0538_gb300 import gbcg, problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMATS = {gbcg.CG_VALUES_FP32: oracle.FP32_FORMAT, gbcg.CG_VALUES_BF16: oracle.BF16_FORMAT}
VALUE_IDS = {gbcg.CG_VALUES_FP32: "fp32", gbcg.CG_VALUES_BF16: "bf16"}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbcg.lib()
    return torch.device("cuda:0")


def ragged_csr(n, seed, long_rows=(), long_len=0, empty=(), unsorted=False, dup=False, diag=True):
    """Random CSR with given row lengths; every non-empty row holds its
    diagonal (when diag) so that the compensated diagonal is exercised."""
    rng = np.random.default_rng(seed)
    rowptr, cols, vals = [0], [], []
    for i in range(n):
        m = 0 if i in empty else (long_len if i in long_rows else int(rng.integers(1, 60)))
        c = rng.choice(n, size=min(m, n), replace=False) if m else np.zeros(0, int)
        if diag and m and i not in c:
            c[0] = i
        if not unsorted:
            c = np.sort(c)
        if dup and m > 2:
            c = np.concatenate([c, c[:2]])
        cols.extend(c.tolist())
        vals.extend((rng.standard_normal(len(c)) * np.exp(rng.uniform(-3, 3, len(c)))).tolist())
        rowptr.append(len(cols))
    return problems.CSR(n, np.array(rowptr, np.int32), np.array(cols, np.int32), np.array(vals))


_CACHE = {}


def cached(key, fn):
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


SPMV_CASES = {
    "n1": lambda: problems.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0])),
    "tail129": lambda: ragged_csr(129, 1),
    "empty_rows": lambda: ragged_csr(700, 2, empty=set(range(0, 700, 7)) | {699}),
    "long_row": lambda: ragged_csr(9000, 3, long_rows={4500}, long_len=8999),
    "unsorted_dups": lambda: ragged_csr(1000, 5, unsorted=True, dup=True),
    "over_tile_limit": lambda: ragged_csr(3000, 7, long_rows={0, 40, 41}, long_len=1025),
    "no_diagonal": lambda: ragged_csr(500, 8, diag=False),
    "all_empty": lambda: problems.CSR(50, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0)),
    "blobs8": lambda: cached("blobs8", lambda: problems.cube_blobs(8, tol=1e-10)).A,
    "c1": lambda: cached("c1", lambda: problems.cube_uniform(20)).A,
    "c2": lambda: cached("c2", lambda: problems.cube_blobs(50)).A,
}


@pytest.mark.parametrize("tiled", [False, True], ids=["default", "tiled"])
@pytest.mark.parametrize("values", list(FORMATS), ids=lambda v: VALUE_IDS[v])
@pytest.mark.parametrize("case", list(SPMV_CASES))
def test_inner_spmv_per_row(dev, case, values, tiled):
    A = SPMV_CASES[case]()
    A_lo = lowprec_matrix(A, FORMATS[values])
    x = fp32(np.random.default_rng(13).standard_normal(A.n))
    with gbcg.Solver(A, inner_values=values, vectors_in_memory=tiled) as s:
        if tiled:
            assert s.plan()["inner_solve"] == 0
        xt = torch.from_numpy(x.astype(np.float32)).to(dev)
        yt = torch.full_like(xt, float("nan"))
        s.spmv_inner(xt, yt)
        y = yt.cpu().numpy().astype(np.float64)
    ref = oracle.spmv(A_lo, x)
    err = np.abs(y - ref)
    bound = spmv_row_bound(A_lo, x)
    assert np.all(err <= bound), (float(err.max()), int(np.argmax(err - bound)))


def test_inner_spmv_large_default_layout(dev):
    """The 100^3 system (27.3M entries): the handle's inner layout, every row."""
    A = cached("c3", lambda: problems.cube_blobs(100)).A
    for values in FORMATS:
        A_lo = lowprec_matrix(A, FORMATS[values])
        x = fp32(np.random.default_rng(17).standard_normal(A.n))
        with gbcg.Solver(A, inner_values=values, precond=gbcg.CG_PRECOND_JACOBI) as s:
            xt = torch.from_numpy(x.astype(np.float32)).to(dev)
            yt = torch.full_like(xt, float("nan"))
            s.spmv_inner(xt, yt)
            y = yt.cpu().numpy().astype(np.float64)
        err = np.abs(y - oracle.spmv(A_lo, x))
        assert np.all(err <= spmv_row_bound(A_lo, x)), VALUE_IDS[values]


def test_inner_spmv_rejects_fp64_handle(dev):
    A = SPMV_CASES["tail129"]()
    with gbcg.Solver(A) as s:
        x = torch.zeros(A.n, dtype=torch.float32, device=dev)
        assert gbcg.cg_spmv_inner(s.h, x.data_ptr(), x.data_ptr()) == gbcg.CG_EINVAL


INNER_SYSTEMS = {
    "blobs8": lambda: cached("blobs8", lambda: problems.cube_blobs(8, tol=1e-10)),
    "blobs12c10": lambda: cached("blobs12c10", lambda: problems.cube_blobs(12, contrast=10.0)),
}


@pytest.mark.parametrize("k", [1, 3, 10])
@pytest.mark.parametrize("precond", [0, 1], ids=["plain", "jacobi"])
@pytest.mark.parametrize("tiled", [False, True], ids=["irsell", "ir_tiled"])
@pytest.mark.parametrize("values", list(FORMATS), ids=lambda v: VALUE_IDS[v])
@pytest.mark.parametrize("name", list(INNER_SYSTEMS))
def test_inner_iterates_fixed_k(dev, name, values, tiled, precond, k):
    pr = INNER_SYSTEMS[name]()
    A_lo = lowprec_matrix(pr.A, FORMATS[values])
    b32 = fp32(pr.b)
    with gbcg.Solver(pr.A, inner_values=values, precond=precond, vectors_in_memory=tiled, max_outer=1,
                     max_inner=k, inner_tol=1e-30) as s:
        assert s.plan()["inner_solve"] == (0 if tiled else 1)
        bt = torch.from_numpy(pr.b).to(dev)
        xt = torch.zeros_like(bt)
        info = s.solve(bt, xt, tol=0.0)
        d = xt.cpu().numpy()
    assert info.status == gbcg.CG_ENOCONV and info.outer == 1 and info.iters == k, info.as_dict()
    check_inner_iterate(d, A_lo, b32, k, precond)


@pytest.mark.parametrize("k", [1, 3, 10])
@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
@pytest.mark.parametrize("precond", [0, 1], ids=["plain", "jacobi"])
@pytest.mark.parametrize("values", list(FORMATS), ids=lambda v: VALUE_IDS[v])
def test_batch_inner_iterates_fixed_k(dev, values, precond, nrhs, k):
    sysl = cached("batch1", lambda: problems.batch_systems(1, 7, 11, seed0=1000))
    s0 = sysl[0]
    A_lo = lowprec_matrix(s0["A"], FORMATS[values])
    with gbcg.BatchSolver([s0["A"]], inner_values=values, precond=precond, max_outer=1, max_inner=k,
                          inner_tol=1e-30) as bs:
        B = torch.from_numpy(np.ascontiguousarray(s0["B"][:nrhs])).to(dev)
        X = torch.zeros_like(B)
        rc, res, _ = bs.solve(B, X, 0.0)
        Xh = X.cpu().numpy()
    for r in range(nrhs):
        assert res[r].status == gbcg.CG_ENOCONV and res[r].outer == 1 and res[r].iters == k, (r, res[r].iters)
        check_inner_iterate(Xh[r], A_lo, fp32(s0["B"][r]), k, precond)
