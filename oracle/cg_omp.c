/*
 * cg_omp.c -- the timed multi-core CPU baseline (TEST INFRASTRUCTURE).
 *
 * Plain FP64 conjugate gradient, the recurrence of the paper's Section IV
 * (one CSR SpMV, two dot products and three axpys per iteration; stop when
 * ||r||_2 <= tol ||b||_2), with the row loop of the SpMV and the vector
 * loops split over the host's cores by OpenMP.  It exists to be timed beside
 * the GPU solve on all host cores; it is NOT the parity reference: its dot
 * products add per-thread partial sums, so its rounding differs from the
 * serial oracle in cg_oracle.c (which stays the reference every parity test
 * uses).  Its own test checks it against that serial oracle.
 *
 * Same conventions as oracle_cg: x holds x0 on entry and the last iterate on
 * exit; maxit <= 0 means n; returns 0 (converged), 4 (maxit reached),
 * 5 (p.q <= 0), 6 (non-finite scalar), 1 (invalid arguments).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include <omp.h>

int cpu_omp_threads(void) { return omp_get_max_threads(); }

static void spmv(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals, const double *x,
                 double *y)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s += vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

static double dot(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int32_t i = 0; i < n; ++i)
        s += a[i] * b[i];
    return s;
}

int cpu_cg_omp(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *vals, const double *b,
               double *x, double tol, int32_t maxit, int32_t *iters, double *relres)
{
    *iters = 0;
    *relres = 0.0;
    if (n < 0 || !(tol >= 0.0))
        return 1;
    if (n == 0)
        return 0;
    if (maxit <= 0)
        maxit = n;
    double *r = malloc(sizeof(double) * (size_t)n);
    double *p = malloc(sizeof(double) * (size_t)n);
    double *q = malloc(sizeof(double) * (size_t)n);
    int status = 4;
    if (!r || !p || !q) {
        status = 2;
        goto done;
    }
    spmv(n, rowptr, colidx, vals, x, q);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        r[i] = b[i] - q[i];
        p[i] = r[i];
    }
    const double bnorm = sqrt(dot(n, b, b));
    double rho = dot(n, r, r);
    if (!isfinite(bnorm) || !isfinite(rho)) {
        status = 6;
        goto done;
    }
    if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i)
            x[i] = 0.0;
        status = 0;
        goto done;
    }
    *relres = sqrt(rho) / bnorm;
    if (sqrt(rho) <= tol * bnorm) {
        status = 0;
        goto done;
    }
    for (int32_t k = 1; k <= maxit; ++k) {
        spmv(n, rowptr, colidx, vals, p, q);
        const double sigma = dot(n, p, q);
        if (!isfinite(sigma)) {
            status = 6;
            break;
        }
        if (!(sigma > 0.0)) {
            status = 5;
            break;
        }
        const double alpha = rho / sigma;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        const double rho_new = dot(n, r, r);
        *iters = k;
        *relres = sqrt(rho_new) / bnorm;
        if (!isfinite(rho_new)) {
            status = 6;
            break;
        }
        if (sqrt(rho_new) <= tol * bnorm) {
            status = 0;
            break;
        }
        const double beta = rho_new / rho;
        rho = rho_new;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i)
            p[i] = r[i] + beta * p[i];
    }
done:
    free(r);
    free(p);
    free(q);
    return status;
}
