"""Error bounds for the FP32 inner CG of iterative refinement against the
FP64 oracle run on the same rounded matrix (helpers of test_gpu_inner.py).

The inner solve of refinement runs CG on A_lo d = fl32(r) with FP32 vectors,
FP32 products and FP32 per-thread sums (the per-CTA partial sums are then
added in FP64).  The oracle runs the same recurrence (Section IV's CG, with
Jacobi when asked) in FP64 on the same rounded values, so the two differ only
by the FP32 rounding of the GPU side.  u = 2^-24 is the FP32 unit roundoff.

One step, d_1 = alpha z_0 with z_0 = M r_0 and alpha = rho_0 / sigma_0,
rho_0 = r_0 . z_0, sigma_0 = z_0 . A_lo z_0:
  * z_0,i carries at most 3u relative error (1 / diag rounded to FP32, the
    product rounded; the oracle forms 1 / diag in FP64);
  * rho_0 is a sum of positive terms, each rounded once, accumulated by one
    thread over at most L rows in FP32: relative error <= (L + 5) u;
  * sigma_0: each q_i = (A_lo z)_i is an FP32 sum of m_i + 1 products plus
    the diagonal FMA, error <= (m_i + 2) u (|A_lo| |z|)_i; the products
    z_i q_i and their FP32 accumulation add (L + 4) u sum |z_i q_i|; so
    |d sigma| / sigma <= [(m + 2) u |z|^T |A_lo| |z| + (L + 4) u sum |z_i q_i|] / sigma;
  * alpha = rho / sigma is formed in FP64 and rounded to FP32 (u), and
    d_1,i = fl(alpha z_0,i) adds one rounding (u) to z_0's 3u.
So |d_1,i - d_1,i_ref| <= |d_1,i_ref| (e_rho + e_sigma + 5u).

After k steps the same rounding terms enter once per step (alpha, beta from
two sums, the SpMV, three vector updates); the test uses k times the
one-step relative bound as a norm-wise bound on the iterate, and checks that
the oracle's iterates k - 1 and k + 1 are farther from iterate k than that,
so an off-by-one in the iteration count, a wrong beta or a wrong inner matrix
cannot pass.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1107_0538_gb300 import problems

U32 = 2.0 ** -24
L_ROWS = 64   # rows one thread accumulates in FP32 before the FP64 sums (at most, for the test sizes)


def lowprec_matrix(A, fmt) -> problems.CSR:
    """A_lo as the oracle defines it (off-diagonals rounded, diagonal compensated)."""
    return problems.CSR(A.n, A.rowptr, A.colidx, oracle.lowprec_values(A, fmt))


def fp32(v) -> np.ndarray:
    """FP32 rounding of FP64 values (IEEE nearest-even), back as FP64."""
    return oracle.round_to_format(np.asarray(v, dtype=np.float64), oracle.FP32_FORMAT)


def diag_of(A) -> np.ndarray:
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return np.bincount(rows, weights=np.where(A.colidx == rows, A.vals, 0.0), minlength=A.n)


def abs_matrix(A) -> problems.CSR:
    return problems.CSR(A.n, A.rowptr, A.colidx, np.abs(A.vals))


def spmv_row_bound(A_lo, x) -> np.ndarray:
    """Per-row bound of an FP32 SpMV (FMA chain of the row's m entries, the
    split accumulators joined, then the diagonal FMA: at most m + 2
    roundings) against the FP64 product of the same FP32 inputs, plus the
    FP64 oracle's own rounding."""
    m = np.diff(A_lo.rowptr).astype(np.float64)
    absax = oracle.spmv(abs_matrix(A_lo), np.abs(x))
    return 2.0 * (m + 2) * (U32 + 2.0 ** -53) * absax


def one_step_rel_bound(A_lo, b32, precond: int) -> float:
    """e_rho + e_sigma + 5u of the module docstring for the first inner step."""
    if precond:
        z = b32 / diag_of(A_lo)
    else:
        z = b32.copy()
    q = oracle.spmv(A_lo, z)
    sigma = float(np.dot(z, q))
    m_max = float(np.max(np.diff(A_lo.rowptr)))
    e_rho = (L_ROWS + 5) * U32
    e_sigma = ((m_max + 2) * U32 * float(np.dot(np.abs(z), oracle.spmv(abs_matrix(A_lo), np.abs(z))))
               + (L_ROWS + 4) * U32 * float(np.sum(np.abs(z * q)))) / sigma
    return e_rho + e_sigma + 5 * U32


def oracle_inner_iterates(A_lo, b32, k: int, precond: int):
    """The oracle's CG iterates k - 1, k, k + 1 on A_lo d = b32 from d = 0."""
    out = []
    for kk in (k - 1, k, k + 1):
        if kk == 0:
            out.append(np.zeros(A_lo.n))
            continue
        r = oracle.cg(A_lo, b32, tol=0.0, maxit=kk, precond=precond)
        assert r["status"] == oracle.ENOCONV and r["iters"] == kk, (r["status"], r["iters"], kk)
        out.append(r["x"])
    return out


def check_inner_iterate(d_gpu, A_lo, b32, k: int, precond: int) -> dict:
    """Compares the GPU inner iterate d_k with the oracle's, element by element
    (k = 1) or in the max norm (k > 1), and checks that the bound separates
    iterate k from its neighbours."""
    prev, ref, nxt = oracle_inner_iterates(A_lo, b32, k, precond)
    b1 = one_step_rel_bound(A_lo, b32, precond)
    scale = float(np.max(np.abs(ref)))
    err = np.abs(d_gpu - ref)
    if k == 1:
        bound = b1 * np.abs(ref) + 4 * 2.0 ** -53 * scale
        assert np.all(err <= bound), (float(np.max(err / np.maximum(bound, 1e-300))), int(np.argmax(err - bound)))
    tau = k * b1
    gap = min(float(np.max(np.abs(prev - ref))), float(np.max(np.abs(nxt - ref)))) / scale
    assert gap >= 4 * tau, ("the bound cannot see an off-by-one here", gap, tau)
    rel = float(np.max(err)) / scale
    assert rel <= tau, (rel, tau)
    return {"rel_err_max": rel, "bound": tau, "gap": gap}
