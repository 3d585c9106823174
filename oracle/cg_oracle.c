/*
 * Plain, serial, FP64 CPU oracle for the conjugate-gradient hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs use it.  It shares no code, header, table or
 * constant with the CUDA library under paper_1107_0538_gb300/.
 *
 * What it computes (paper, Section IV "Case Study"): the conjugate gradient
 * method on a symmetric positive definite matrix stored in Compressed Sparse
 * Row form, iterated until a continue-condition on the residual fails or the
 * loop has run N times.  One iteration is one sparse matrix-vector product
 * ("DGEMV(sparse)"), two dot products and three axpy updates, which is the
 * operation count that reproduces the GFLOPS column of Table I
 * (2*NNZ + 10*N flops per iteration).  The recurrence is the standard
 * Hestenes-Stiefel form of the textbook the paper cites for CG (Golub and
 * Van Loan):
 *
 *     r0 = b - A x0,  p0 = z0 = M^-1 r0,  rho0 = r0.z0
 *     for k = 1, 2, ...
 *         q     = A p
 *         alpha = rho / (p.q)
 *         x    += alpha p
 *         r    -= alpha q
 *         stop when ||r||_2 <= tol ||b||_2
 *         z     = M^-1 r          (M = I for plain CG, M = diag(A) for Jacobi)
 *         beta  = (r.z) / rho,  rho = r.z
 *         p     = z + beta p
 *
 * Readings where the paper is silent:
 *   - the stop test is the recursive residual 2-norm relative to ||b||_2
 *     (Table I gives only "tol=1e-10");
 *   - the iteration count is the number of products A p inside the loop;
 *   - the default maximum is N iterations ("a 132651 loop", Section IV);
 *   - b = 0 gives x = 0 after zero iterations;
 *   - p.q <= 0 is a breakdown, a non-finite scalar is reported as NaN.
 *
 * Arithmetic: every sum runs left to right in index order, and the file is
 * compiled with -ffp-contract=off so no multiply-add is fused; results are
 * the same on x86-64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Status codes of this oracle (defined here on their own; the CUDA library
 * has its own header). */
#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2
#define ORACLE_ENOCONV 4
#define ORACLE_EBREAKDOWN 5
#define ORACLE_ENAN 6

/* y = A x: for each row, the sum over its stored entries, in storage order.
 * This is the "DGEMV(sparse)" task of Section IV. */
void oracle_spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                 const double *vals, const double *x, double *y)
{
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s = s + vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

/* a.b summed left to right. */
double oracle_dot(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i)
        s = s + a[i] * b[i];
    return s;
}

/* The diagonal entry of row i (sum of the entries whose column is i). */
static double row_diagonal(const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, int32_t i)
{
    double d = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (colidx[k] == i)
            d = d + vals[k];
    return d;
}

/* z = M^-1 r: the identity for plain CG, division by diag(A) for Jacobi. */
static void apply_preconditioner(int32_t n, int32_t precond, const double *diag,
                                 const double *r, double *z)
{
    for (int32_t i = 0; i < n; ++i)
        z[i] = precond ? r[i] / diag[i] : r[i];
}

/*
 * Conjugate gradient (precond = 0) or Jacobi-preconditioned CG (precond = 1)
 * on A x = b, following the recurrence in the header above.
 *
 *   x        in: x0, out: the last iterate
 *   tol      relative tolerance on ||r||_2 / ||b||_2 (>= 0)
 *   maxit    maximum iterations; <= 0 means n
 *   iters    out: iterations completed (products A p whose update was applied)
 *   relres   out: ||r_k||_2 / ||b||_2 of the recursive residual at exit
 *   xtrace   optional (may be NULL): (maxit + 1) * n doubles; row k holds x_k
 *   ptrace   optional: maxit * n doubles; row k holds the direction p_k
 *   rtrace   optional: (maxit + 1) * n doubles; row k holds r_k
 *
 * Returns ORACLE_OK on convergence, ORACLE_ENOCONV after maxit iterations,
 * ORACLE_EBREAKDOWN when p.q <= 0 (or r.z <= 0 with a preconditioner),
 * ORACLE_ENAN when a scalar is not finite, ORACLE_EINVAL on bad arguments.
 */
int oracle_cg(int32_t n, const int32_t *rowptr, const int32_t *colidx,
              const double *vals, const double *b, double *x, double tol,
              int32_t maxit, int32_t precond, int32_t *iters, double *relres,
              double *xtrace, double *ptrace, double *rtrace)
{
    if (n < 0 || !(tol >= 0.0) || (precond != 0 && precond != 1))
        return ORACLE_EINVAL;
    if (maxit <= 0)
        maxit = n;
    *iters = 0;
    *relres = 0.0;
    if (n == 0)
        return ORACLE_OK;

    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    int status = ORACLE_OK;
    if (!r || !z || !p || !q || !diag) {
        status = ORACLE_ENOMEM;
        goto done;
    }
    for (int32_t i = 0; i < n; ++i) {
        diag[i] = row_diagonal(rowptr, colidx, vals, i);
        if (precond && !(diag[i] > 0.0)) {
            status = ORACLE_EINVAL;
            goto done;
        }
    }

    /* r0 = b - A x0 */
    oracle_spmv(n, rowptr, colidx, vals, x, q);
    for (int32_t i = 0; i < n; ++i)
        r[i] = b[i] - q[i];
    double bb = oracle_dot(n, b, b);
    if (!isfinite(bb)) {
        status = ORACLE_ENAN;
        goto done;
    }
    double bnorm = sqrt(bb);
    if (bnorm == 0.0) { /* b = 0: the solution is x = 0 */
        for (int32_t i = 0; i < n; ++i)
            x[i] = 0.0;
        if (xtrace)
            memcpy(xtrace, x, sizeof(double) * (size_t)n);
        goto done;
    }
    apply_preconditioner(n, precond, diag, r, z);
    double rr = oracle_dot(n, r, r);
    double rho = oracle_dot(n, r, z);
    if (xtrace)
        memcpy(xtrace, x, sizeof(double) * (size_t)n);
    if (rtrace)
        memcpy(rtrace, r, sizeof(double) * (size_t)n);
    *relres = sqrt(rr) / bnorm;
    if (!isfinite(rr) || !isfinite(rho)) {
        status = ORACLE_ENAN;
        goto done;
    }
    if (sqrt(rr) <= tol * bnorm)
        goto done;
    if (!(rho > 0.0)) {
        status = ORACLE_EBREAKDOWN;
        goto done;
    }
    for (int32_t i = 0; i < n; ++i)
        p[i] = z[i];

    for (int32_t k = 1; k <= maxit; ++k) {
        if (ptrace)
            memcpy(ptrace + (size_t)(k - 1) * n, p, sizeof(double) * (size_t)n);
        oracle_spmv(n, rowptr, colidx, vals, p, q);
        double sigma = oracle_dot(n, p, q);
        if (!isfinite(sigma)) {
            status = ORACLE_ENAN;
            goto done;
        }
        if (!(sigma > 0.0)) {
            status = ORACLE_EBREAKDOWN;
            goto done;
        }
        double alpha = rho / sigma;
        for (int32_t i = 0; i < n; ++i)
            x[i] = x[i] + alpha * p[i];
        for (int32_t i = 0; i < n; ++i)
            r[i] = r[i] - alpha * q[i];
        *iters = k;
        if (xtrace)
            memcpy(xtrace + (size_t)k * n, x, sizeof(double) * (size_t)n);
        if (rtrace)
            memcpy(rtrace + (size_t)k * n, r, sizeof(double) * (size_t)n);
        rr = oracle_dot(n, r, r);
        *relres = sqrt(rr) / bnorm;
        if (!isfinite(rr)) {
            status = ORACLE_ENAN;
            goto done;
        }
        if (sqrt(rr) <= tol * bnorm)
            goto done;
        apply_preconditioner(n, precond, diag, r, z);
        double rho_new = oracle_dot(n, r, z);
        if (!isfinite(rho_new)) {
            status = ORACLE_ENAN;
            goto done;
        }
        if (!(rho_new > 0.0)) {
            status = ORACLE_EBREAKDOWN;
            goto done;
        }
        double beta = rho_new / rho;
        for (int32_t i = 0; i < n; ++i)
            p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
    status = ORACLE_ENOCONV;

done:
    free(r);
    free(z);
    free(p);
    free(q);
    free(diag);
    return status;
}

/*
 * Round v to the nearest value of a binary floating-point format with a
 * p-bit significand (hidden bit included), minimum normal exponent emin and
 * maximum exponent emax; ties go to the even significand (IEEE 754
 * round-to-nearest-even).  Below 2^emin the spacing stays 2^(emin - p + 1)
 * (gradual underflow); a result past the largest finite value becomes
 * infinite.  fp32 is (24, -126, 127); bf16 is (8, -126, 127).
 */
double oracle_round_to_format(double v, int32_t p, int32_t emin, int32_t emax)
{
    if (v == 0.0 || !isfinite(v))
        return v;
    int e;
    (void)frexp(v, &e);     /* v = m 2^e with 0.5 <= |m| < 1 */
    int E = e - 1;          /* v = (2m) 2^E with 1 <= |2m| < 2 */
    if (E < emin)
        E = emin;
    int shift = E - p + 1;  /* the spacing of the format near v is 2^shift */
    double scaled = ldexp(v, -shift);      /* exact: a power-of-two scale */
    double r = ldexp(nearbyint(scaled), shift);
    double max_finite = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
    if (fabs(r) > max_finite)
        return copysign(INFINITY, v);
    return r;
}

void oracle_round_array(int64_t count, const double *in, double *out, int32_t p,
                        int32_t emin, int32_t emax)
{
    for (int64_t i = 0; i < count; ++i)
        out[i] = oracle_round_to_format(in[i], p, emin, emax);
}

/*
 * The low-precision inner matrix of iterative refinement, written out as
 * doubles.  Off-diagonal values are rounded to the format (p, emin, emax).
 * Rounding them alone would move every row sum by up to half an ulp per
 * entry, which for a stiffness matrix K (rows summing to zero) plus a small
 * mass shift destroys the smallest eigenvalues and can make the rounded
 * matrix indefinite.  So the diagonal entry of each row is set to
 *     fp32( sum_j a_ij  -  sum_{j != i} lo(a_ij) )
 * (both sums in FP64, left to right in storage order): the rounded matrix has
 * the same row sums as A up to one FP32 rounding, and a symmetric matrix with
 * non-positive off-diagonals and positive row sums stays diagonally dominant,
 * hence SPD.  The diagonal is kept in FP32 (p = 24) whatever the off-diagonal
 * format.  With several entries in column i the first one takes the value and
 * the others become 0; a row without a diagonal entry is rounded as is.
 */
void oracle_lowprec_values(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                           const double *vals, int32_t p, int32_t emin, int32_t emax,
                           double *vals_lo)
{
    for (int32_t i = 0; i < n; ++i) {
        double rowsum = 0.0, offsum = 0.0;
        int32_t dpos = -1;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            rowsum = rowsum + vals[k];
            if (colidx[k] == i) {
                if (dpos < 0)
                    dpos = k;
                vals_lo[k] = 0.0;
            } else {
                vals_lo[k] = oracle_round_to_format(vals[k], p, emin, emax);
                offsum = offsum + vals_lo[k];
            }
        }
        if (dpos >= 0)
            vals_lo[dpos] = oracle_round_to_format(rowsum - offsum, 24, -126, 127);
    }
}

/*
 * Mixed-precision iterative refinement around CG.  The outer loop keeps the
 * solution and the residual in FP64 with the FP64 matrix:
 *
 *     r = b - A x;  stop when ||r||_2 <= tol ||b||_2
 *     solve A_lo d = r by CG until ||r_in||_2 <= inner_tol ||r||_2
 *     x += d
 *
 * where A_lo holds the matrix values rounded to the low precision (the caller
 * passes them already rounded, as doubles).  The inner solve here runs in
 * FP64 arithmetic; only the matrix copy is rounded.
 *
 *   outer     out: outer corrections applied
 *   inner     out: inner CG iterations summed over all corrections
 *   relres    out: ||b - A x||_2 / ||b||_2 with the FP64 matrix at exit
 */
int oracle_cg_ir(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                 const double *vals, const double *vals_lo, const double *b,
                 double *x, double tol, double inner_tol, int32_t max_outer,
                 int32_t max_inner, int32_t *outer, int32_t *inner,
                 double *relres)
{
    *outer = 0;
    *inner = 0;
    *relres = 0.0;
    if (n < 0 || !(tol >= 0.0) || !(inner_tol > 0.0) || max_outer < 0)
        return ORACLE_EINVAL;
    if (n == 0)
        return ORACLE_OK;
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    int status = ORACLE_OK;
    if (!r || !d) {
        status = ORACLE_ENOMEM;
        goto done;
    }
    double bb = oracle_dot(n, b, b);
    if (!isfinite(bb)) {
        status = ORACLE_ENAN;
        goto done;
    }
    double bnorm = sqrt(bb);
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; ++i)
            x[i] = 0.0;
        goto done;
    }
    for (int32_t o = 0;; ++o) {
        oracle_spmv(n, rowptr, colidx, vals, x, r);
        for (int32_t i = 0; i < n; ++i)
            r[i] = b[i] - r[i];
        double rnorm = sqrt(oracle_dot(n, r, r));
        *relres = rnorm / bnorm;
        if (!isfinite(rnorm)) {
            status = ORACLE_ENAN;
            goto done;
        }
        if (rnorm <= tol * bnorm)
            goto done;
        if (o == max_outer) {
            status = ORACLE_ENOCONV;
            goto done;
        }
        for (int32_t i = 0; i < n; ++i)
            d[i] = 0.0;
        int32_t it = 0;
        double rel_in = 0.0;
        int st = oracle_cg(n, rowptr, colidx, vals_lo, r, d, inner_tol, max_inner,
                           0, &it, &rel_in, NULL, NULL, NULL);
        *inner += it;
        if (st == ORACLE_ENAN || st == ORACLE_EBREAKDOWN || st == ORACLE_EINVAL ||
            st == ORACLE_ENOMEM) {
            status = st;
            goto done;
        }
        for (int32_t i = 0; i < n; ++i)
            x[i] = x[i] + d[i];
        *outer = o + 1;
    }

done:
    free(r);
    free(d);
    return status;
}
