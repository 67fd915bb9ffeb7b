/*
 * The oracle's Table I sequences run over all host cores.  TEST
 * INFRASTRUCTURE ONLY (the benchmark's CPU baseline and the reference arm):
 * nothing in the product path may call, link or load this file.
 *
 * Every routine computes exactly what the routine of the same name in
 * bto_oracle.c computes, bit for bit: the work is divided among OpenMP
 * threads over independent outputs only (rows of A p, columns of A^T r,
 * elements of the vector kernels), and every output is formed by one thread
 * with the same operations in the same order as the serial loop nest (sums
 * in ascending index order, each multiply and add rounded on its own; build
 * with -ffp-contract=off).  The one sum over all of a vector, AXPYDOT's
 * r = z^T u, stays on one thread.  tests/test_oracle_par.py checks the bit
 * equality against bto_oracle.c.
 */
#include <stdint.h>
#include <stdlib.h>

#define AT(A, lda, i, j) ((A)[(size_t)(i) + (size_t)(j) * (size_t)(lda)])

/* out[i] = sum_j A(i,j) v[j], ascending j, for every row i. */
static void rows_dot(int64_t m, int64_t n, const double *A, int64_t lda, const double *v, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; j++)
            acc += AT(A, lda, i, j) * v[j];
        out[i] = acc;
    }
}

/* out[j] = sum_i A(i,j) v[i], ascending i, for every column j. */
static void cols_dot(int64_t m, int64_t n, const double *A, int64_t lda, const double *v, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++) {
        double acc = 0.0;
        for (int64_t i = 0; i < m; i++)
            acc += AT(A, lda, i, j) * v[i];
        out[j] = acc;
    }
}

void oracle_par_bicgk(int64_t m, int64_t n, const double *A, int64_t lda,
                      const double *p, const double *r, double *q, double *s)
{
    rows_dot(m, n, A, lda, p, q);
    cols_dot(m, n, A, lda, r, s);
}

int oracle_par_atax(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                    const double *x, double *y)
{
    double *t0 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t0) return -1;
    rows_dot(m, n, A, lda, x, t0);
    cols_dot(m, n, A, lda, t0, y);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        y[j] = y[j] * beta;
    free(t0);
    return 0;
}

int oracle_par_gemver(int64_t m, int64_t n, double alpha, double beta,
                      const double *A, int64_t lda,
                      const double *u1, const double *v1,
                      const double *u2, const double *v2,
                      const double *y, const double *z,
                      double *B, int64_t ldb, double *x, double *w)
{
    double *t2 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t2) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            double b = AT(A, lda, i, j);
            b = b + u1[i] * v1[j];
            AT(B, ldb, i, j) = b + u2[i] * v2[j];
        }
    cols_dot(m, n, B, ldb, y, x);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        x[j] = beta * x[j] + z[j];
    rows_dot(m, n, B, ldb, x, t2);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++)
        w[i] = alpha * t2[i];
    free(t2);
    return 0;
}

int oracle_par_gesummv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                       double beta, const double *B, int64_t ldb,
                       const double *x, double *y)
{
    double *ta = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *tb = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!ta || !tb) { free(ta); free(tb); return -1; }
    rows_dot(m, n, A, lda, x, ta);
    rows_dot(m, n, B, ldb, x, tb);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++)
        y[i] = alpha * ta[i] + beta * tb[i];
    free(ta); free(tb);
    return 0;
}

int oracle_par_dgemv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                     const double *x, double beta, const double *y, double *z)
{
    double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t) return -1;
    rows_dot(m, n, A, lda, x, t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++)
        z[i] = alpha * t[i] + beta * y[i];
    free(t);
    return 0;
}

int oracle_par_dgemvt(int64_t m, int64_t n, double alpha, double beta,
                      const double *A, int64_t lda, const double *y, const double *z,
                      double *x, double *w)
{
    double *t2 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t2) return -1;
    cols_dot(m, n, A, lda, y, x);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
        x[j] = beta * x[j] + z[j];
    rows_dot(m, n, A, lda, x, t2);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++)
        w[i] = alpha * t2[i];
    free(t2);
    return 0;
}

void oracle_par_axpydot(int64_t n, double alpha, const double *w, const double *v,
                        const double *u, double *z, double *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        z[i] = w[i] - alpha * v[i];
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++)
        acc += z[i] * u[i];
    *r = acc;
}

void oracle_par_waxpby(int64_t n, double alpha, const double *x, double beta,
                       const double *y, double *w)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        w[i] = alpha * x[i] + beta * y[i];
}

void oracle_par_vadd(int64_t n, const double *w, const double *y, const double *z,
                     double *x)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        x[i] = (w[i] + y[i]) + z[i];
}
