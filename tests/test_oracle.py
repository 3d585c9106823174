"""Pins for the CPU FP64 oracle.

The oracle is checked against what the mathematics of CG fixes rather than
against itself: dense Cholesky solves (a library routine) on small SPD
systems, a manufactured solution, the A-orthogonality of the search
directions, the orthogonality of the residuals, the monotone decrease of the
A-norm error, finite termination in at most N (or m distinct eigenvalue)
steps, the Chebyshev bound, the exact equivalence of Jacobi-PCG with CG on
the symmetrically scaled matrix, and brute-force enumeration of a
floating-point format for the rounding routine.  A dropped term, a wrong sign
or a transposed operand anywhere in the recurrence breaks at least one.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1107_0538_gb300 import problems as P


def dense_to_csr(D, keep_zeros=False):
    n = D.shape[0]
    rowptr = [0]
    cols, vals = [], []
    for i in range(n):
        for j in range(n):
            if keep_zeros or D[i, j] != 0.0:
                cols.append(j)
                vals.append(D[i, j])
        rowptr.append(len(cols))
    return P.CSR(n, np.array(rowptr, np.int32), np.array(cols, np.int32), np.array(vals))


def random_spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    D = (Q * ev) @ Q.T
    return 0.5 * (D + D.T)


def random_csr(n, density, seed, long_row=None, empty_rows=()):
    rng = np.random.default_rng(seed)
    D = np.where(rng.random((n, n)) < density, rng.standard_normal((n, n)), 0.0)
    for r in empty_rows:
        D[r, :] = 0.0
    if long_row is not None:
        D[long_row, :] = rng.standard_normal(n)
    return D, dense_to_csr(D)


# ------------------------------------------------------------------- SpMV

@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (37, 0.2, 1), (200, 0.05, 2)])
def test_spmv_matches_dense_product(n, density, seed):
    D, A = random_csr(n, density, seed, long_row=n // 2, empty_rows=(0,) if n > 2 else ())
    x = np.random.default_rng(seed + 10).standard_normal(n)
    np.testing.assert_allclose(oracle.spmv(A, x), D @ x, rtol=1e-13, atol=1e-13)


def test_spmv_q1_grid_bruteforce():
    pr = P.cube_blobs(4)
    x = np.random.default_rng(0).standard_normal(pr.A.n)
    np.testing.assert_allclose(oracle.spmv(pr.A, x), pr.A.to_dense() @ x, rtol=1e-13, atol=1e-16)


# ------------------------------------------------------ CG solution pins

@pytest.mark.parametrize("n,cond,seed", [(8, 10.0, 0), (33, 1e3, 1), (64, 1e2, 2)])
def test_cg_matches_cholesky(n, cond, seed):
    D = random_spd(n, cond, seed)
    A = dense_to_csr(D, keep_zeros=True)
    b = np.random.default_rng(seed).standard_normal(n)
    r = oracle.cg(A, b, tol=1e-13, maxit=10 * n)
    assert r["status"] == oracle.OK
    x_ref = sla.cho_solve(sla.cho_factor(D), b)
    assert np.linalg.norm(r["x"] - x_ref) / np.linalg.norm(x_ref) <= 10 * cond * 1e-13


@pytest.mark.parametrize("e", [2, 3])
def test_cg_q1_grid_matches_cholesky(e):
    pr = P.cube_blobs(e)
    D = pr.A.to_dense()
    r = oracle.cg(pr.A, pr.b, tol=1e-14, maxit=10 * pr.A.n)
    x_ref = sla.cho_solve(sla.cho_factor(D), pr.b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(r["x"] - x_ref) / np.linalg.norm(x_ref) <= 10 * kappa * 1e-14


def test_manufactured_solution():
    pr = P.cube_blobs(8)
    kappa = np.linalg.cond(pr.A.to_dense())
    r = oracle.cg(pr.A, pr.b, tol=1e-12)
    assert r["status"] == oracle.OK
    err = np.linalg.norm(r["x"] - pr.xstar) / np.linalg.norm(pr.xstar)
    assert err <= kappa * 1e-12


def test_exact_termination_within_n_steps():
    # moderate conditioning so that rounding does not delay termination
    n = 48
    D = random_spd(n, 10.0, 7)
    A = dense_to_csr(D, keep_zeros=True)
    b = np.random.default_rng(7).standard_normal(n)
    r = oracle.cg(A, b, tol=1e-10, maxit=n)
    assert r["status"] == oracle.OK and r["iters"] <= n


def test_scaled_identity_one_iteration():
    n = 20
    c = 3.5
    A = dense_to_csr(c * np.eye(n))
    b = np.random.default_rng(1).standard_normal(n)
    r = oracle.cg(A, b, tol=1e-14)
    assert r["status"] == oracle.OK and r["iters"] == 1
    np.testing.assert_allclose(r["x"], b / c, rtol=1e-15)


@pytest.mark.parametrize("m", [1, 3, 7])
def test_m_distinct_eigenvalues_m_iterations(m):
    n = 40
    eig = np.repeat(np.linspace(1.0, 5.0, m), int(np.ceil(n / m)))[:n]
    rng = np.random.default_rng(m)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = (Q * eig) @ Q.T
    A = dense_to_csr(0.5 * (D + D.T), keep_zeros=True)
    b = rng.standard_normal(n)
    r = oracle.cg(A, b, tol=1e-11, maxit=n)
    assert r["status"] == oracle.OK
    assert r["iters"] == m


# ------------------------------------------------------ iterate invariants

def _small_traced_problem():
    pr = P.cube_blobs(4, contrast=10.0)
    D = pr.A.to_dense()
    xs = np.linalg.solve(D, pr.b)
    tr = oracle.cg(pr.A, pr.b, tol=0.0, maxit=15, trace=True)
    return pr, D, xs, tr


def test_search_directions_a_orthogonal():
    pr, D, xs, tr = _small_traced_problem()
    Pm = tr["ptrace"]
    G = Pm @ D @ Pm.T
    d = np.sqrt(np.diag(G))
    C = G / np.outer(d, d)
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() <= 1e-8


def test_residuals_orthogonal_and_consistent():
    pr, D, xs, tr = _small_traced_problem()
    R = tr["rtrace"]
    G = R @ R.T
    d = np.sqrt(np.diag(G))
    C = G / np.outer(d, d)
    assert np.abs(C - np.diag(np.diag(C))).max() <= 1e-8
    # the recursive residual is the true residual of each iterate
    for k in range(R.shape[0]):
        true = pr.b - D @ tr["xtrace"][k]
        assert np.linalg.norm(true - R[k]) <= 1e-12 * np.linalg.norm(pr.b)


def test_a_norm_error_monotone_and_chebyshev():
    pr, D, xs, tr = _small_traced_problem()
    E = tr["xtrace"] - xs
    anorm = np.sqrt(np.einsum("ki,ij,kj->k", E, D, E))
    assert np.all(np.diff(anorm) <= 1e-12 * anorm[0])
    ev = np.linalg.eigvalsh(D)
    kappa = ev[-1] / ev[0]
    rate = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    bound = 2 * rate ** np.arange(len(anorm)) * anorm[0]
    assert np.all(anorm <= bound * (1 + 1e-10))


def test_krylov_optimality_first_steps():
    """x_k minimises the A-norm error over x0 + K_k(A, r0) (checked for k <= 4)."""
    pr, D, xs, tr = _small_traced_problem()
    b = pr.b
    basis = [b]
    for k in range(1, 5):
        Kmat = np.array(basis).T  # n x k
        # minimise ||x - xs||_A over x = K c: normal equations K^T A K c = K^T b
        c = np.linalg.solve(Kmat.T @ D @ Kmat, Kmat.T @ b)
        x_opt = Kmat @ c
        rel = np.linalg.norm(x_opt - tr["xtrace"][k]) / np.linalg.norm(x_opt)
        assert rel <= 1e-8
        basis.append(D @ basis[-1])


# --------------------------------------------------------- Jacobi-PCG pins

def test_jacobi_pcg_on_diagonal_matrix_one_iteration():
    n = 30
    d = np.linspace(1.0, 100.0, n)
    A = dense_to_csr(np.diag(d))
    b = np.random.default_rng(2).standard_normal(n)
    r = oracle.cg(A, b, tol=1e-14, precond=1)
    assert r["iters"] == 1 and r["status"] == oracle.OK
    np.testing.assert_allclose(r["x"], b / d, rtol=1e-14)
    assert oracle.cg(A, b, tol=1e-14, precond=0)["iters"] > 1


def test_jacobi_pcg_equals_cg_on_scaled_system():
    """PCG with M = diag(A) produces x_k = D^-1/2 y_k, y_k the CG iterates of
    D^-1/2 A D^-1/2 y = D^-1/2 b (the same Krylov recurrence, exact arithmetic)."""
    pr = P.cube_blobs(5, contrast=1e2)
    D = pr.A.to_dense()
    s = 1.0 / np.sqrt(np.diag(D))
    As = dense_to_csr(D * np.outer(s, s), keep_zeros=True)
    k = 25
    xp = oracle.cg(pr.A, pr.b, tol=0.0, maxit=k, precond=1)["x"]
    y = oracle.cg(As, s * pr.b, tol=0.0, maxit=k, precond=0)["x"]
    np.testing.assert_allclose(xp, s * y, rtol=1e-9, atol=1e-12 * np.abs(xp).max())


# ------------------------------------------------------------ edge cases

def test_zero_rhs_gives_zero_solution():
    pr = P.cube_uniform(3)
    r = oracle.cg(pr.A, np.zeros(pr.A.n), x0=np.ones(pr.A.n), tol=1e-10)
    assert r["status"] == oracle.OK and r["iters"] == 0
    assert np.all(r["x"] == 0)


def test_maxit_reached_returns_last_iterate():
    pr = P.cube_blobs(5)
    r5 = oracle.cg(pr.A, pr.b, tol=1e-14, maxit=5)
    assert r5["status"] == oracle.ENOCONV and r5["iters"] == 5
    tr = oracle.cg(pr.A, pr.b, tol=0.0, maxit=5, trace=True)
    np.testing.assert_array_equal(r5["x"], tr["xtrace"][5])


def test_indefinite_breaks_down():
    A = dense_to_csr(np.diag([1.0, -1.0, 2.0]))
    r = oracle.cg(A, np.array([0.0, 1.0, 0.0]), tol=1e-12)
    assert r["status"] == oracle.EBREAKDOWN


def test_nan_rhs():
    pr = P.cube_uniform(2)
    b = pr.b.copy()
    b[3] = np.nan
    assert oracle.cg(pr.A, b)["status"] == oracle.ENAN


def test_empty_system():
    A = P.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    r = oracle.cg(A, np.zeros(0))
    assert r["status"] == oracle.OK and r["iters"] == 0


def test_nonzero_initial_guess():
    pr = P.cube_blobs(4)
    x_ref = np.linalg.solve(pr.A.to_dense(), pr.b)
    r = oracle.cg(pr.A, pr.b, x0=x_ref + 1e-3, tol=1e-12)
    np.testing.assert_allclose(r["x"], x_ref, rtol=1e-8)


# ------------------------------------------------------- rounding routine

def _all_bf16_values():
    bits = np.arange(65536, dtype=np.uint32) << np.uint32(16)
    with np.errstate(invalid="ignore"):
        v = bits.view(np.float32).astype(np.float64)
    pattern = np.arange(65536)
    keep = np.isfinite(v)
    return v[keep], pattern[keep]


def test_round_bf16_bruteforce_nearest_even():
    vals, pats = _all_bf16_values()
    order = np.argsort(vals, kind="stable")
    vals, pats = vals[order], pats[order]
    # drop -0 so each value appears once (keep +0, pattern 0)
    keep = ~((vals == 0) & (pats != 0))
    vals, pats = vals[keep], pats[keep]
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-40, 38, 20000),
                        (vals[1:-1] + vals[2:]) / 2.0])  # exact midpoints: ties
    v = v[np.abs(v) < vals.max()]
    got = oracle.round_to_format(v, oracle.BF16_FORMAT)
    i = np.clip(np.searchsorted(vals, v), 1, len(vals) - 1)
    lo, hi = vals[i - 1], vals[i]
    want = np.where(v - lo < hi - v, lo, hi)
    tie = (v - lo) == (hi - v)
    want = np.where(tie, np.where(pats[i - 1] % 2 == 0, lo, hi), want)
    want = np.where(v == hi, hi, want)
    np.testing.assert_array_equal(got, want)


def test_round_fp32_matches_ieee_cast():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(50000) * 10.0 ** rng.integers(-46, 39, 50000)
    v = np.concatenate([v, [1e-46, 3e-45, 3.4e38, 3.5e38, -1e39, 0.0]])
    with np.errstate(over="ignore"):
        want = v.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(oracle.round_to_format(v, oracle.FP32_FORMAT), want)


# ----------------------------------------------- iterative refinement pins

def test_ir_with_exact_values_is_one_correction():
    pr = P.cube_blobs(5)
    r = oracle.cg_ir(pr.A, pr.A.vals, pr.b, tol=1e-9, inner_tol=1e-12, max_outer=10)
    assert r["status"] == oracle.OK and r["outer"] == 1
    x_ref = oracle.cg(pr.A, pr.b, tol=1e-12)["x"]
    np.testing.assert_allclose(r["x"], x_ref, rtol=1e-8)


@pytest.mark.parametrize("fmt,inner_tol", [(oracle.FP32_FORMAT, 1e-3), (oracle.BF16_FORMAT, 1e-2)])
def test_ir_reaches_fp64_accuracy_with_rounded_values(fmt, inner_tol):
    pr = P.cube_blobs(6)
    D = pr.A.to_dense()
    lo = oracle.lowprec_values(pr.A, fmt)
    r = oracle.cg_ir(pr.A, lo, pr.b, tol=1e-10, inner_tol=inner_tol, max_outer=60)
    assert r["status"] == oracle.OK and r["outer"] >= 2
    true = np.linalg.norm(pr.b - D @ r["x"]) / np.linalg.norm(pr.b)
    assert true <= 1e-10
    x_ref = sla.cho_solve(sla.cho_factor(D), pr.b)
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(r["x"] - x_ref) / np.linalg.norm(x_ref) <= 10 * kappa * 1e-10


@pytest.mark.parametrize("fmt", [oracle.FP32_FORMAT, oracle.BF16_FORMAT])
def test_lowprec_values_rowsums_format_and_spd(fmt):
    pr = P.cube_blobs(6)
    lo = oracle.lowprec_values(pr.A, fmt)
    rows = np.repeat(np.arange(pr.A.n), np.diff(pr.A.rowptr))
    diag = pr.A.colidx == rows
    # off-diagonals are exactly the rounded values
    np.testing.assert_array_equal(lo[~diag], oracle.round_to_format(pr.A.vals[~diag], fmt))
    # the diagonal is an FP32 number
    assert np.array_equal(lo[diag], lo[diag].astype(np.float32).astype(np.float64))
    # row sums agree with A's to one FP32 rounding of the diagonal
    rs = np.bincount(rows, weights=pr.A.vals)
    rs_lo = np.bincount(rows, weights=lo)
    assert np.all(np.abs(rs_lo - rs) <= 2.0 ** -24 * np.abs(lo[diag]) * 1.01)
    D = P.CSR(pr.A.n, pr.A.rowptr, pr.A.colidx, lo).to_dense()
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    # plain rounding of every value (the diagonal included) is not enough in BF16
    if fmt == oracle.BF16_FORMAT:
        Dn = P.CSR(pr.A.n, pr.A.rowptr, pr.A.colidx, oracle.round_to_format(pr.A.vals, fmt)).to_dense()
        assert np.linalg.eigvalsh(Dn).min() < 0


def test_openmp_baseline_matches_serial_oracle():
    """The multi-core CPU baseline (timed by the bench, not a parity
    reference) computes the same CG: on the 20^3 uniform cube at rtol 1e-10
    its solution is within 1e-10 of the serial oracle's and its iteration
    count within 2 (it only sums its dot products in another order)."""
    pr = P.cube_uniform(20)
    ref = oracle.cg(pr.A, pr.b, tol=pr.tol)
    omp = oracle.cg_omp(pr.A, pr.b, tol=pr.tol)
    assert omp["status"] == oracle.OK == ref["status"]
    assert abs(omp["iters"] - ref["iters"]) <= 2
    assert np.linalg.norm(omp["x"] - ref["x"]) <= 1e-10 * np.linalg.norm(ref["x"])
    assert oracle.omp_threads() >= 1
    z = oracle.cg_omp(pr.A, np.zeros(pr.A.n), tol=1e-8)
    assert z["status"] == oracle.OK and z["iters"] == 0 and not np.any(z["x"])
    capped = oracle.cg_omp(pr.A, pr.b, tol=1e-14, maxit=5)
    assert capped["status"] == oracle.ENOCONV and capped["iters"] == 5
