/*
 * Oracle for the fused BLAS-1/2 sequences of "Reliable Generation of
 * High-Performance Matrix Algebra" (Belter, Jessup, Nelson, Norris, Siek;
 * the Build to Order BLAS).  TEST INFRASTRUCTURE ONLY: nothing in the product
 * path may call, link or load this file; only the tests, the package smoke
 * check and the benchmark's CPU-baseline leg do.
 *
 * Every routine is the plain mathematical definition of one kernel of
 * Table I, written as the unfused loop nests of the running example (the
 * BATAX pseudocode of Section III-D: an accumulation loop nest per product,
 * then a separate scaling loop), in FP64, ascending index order, one loop
 * nest per statement of the table.  Compile with -ffp-contract=off so that
 * every multiply and add rounds on its own.
 *
 * The CSR routines at the end define BICGK and BATAX on a matrix in
 * compressed sparse rows (the sparse format of Section VII) as loops over the
 * stored entries, in storage order; the band routines after them define
 * BICGK and BATAX on banded and triangular matrices (the other formats
 * planned there) as the same loops restricted to the band.
 *
 * Matrices are column-major: element (i, j) of A is A[i + j*lda].
 * Sizes m, n may be zero; empty sums are zero.  No BLAS-style shortcut is
 * taken for zero scalars: alpha*s is always evaluated, so NaN/Inf propagate.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define AT(A, lda, i, j) ((A)[(size_t)(i) + (size_t)(j) * (size_t)(lda)])

/* BICGK (Table I):  q <- A p ;  s <- A^T r.
 * The two statements are the two dgemv calls of the paper's BLAS listing
 * for BICGK (Section V-A): a non-transposed and a transposed product. */
void oracle_bicgk(int64_t m, int64_t n, const double *A, int64_t lda,
                  const double *p, const double *r, double *q, double *s)
{
    for (int64_t i = 0; i < m; i++) q[i] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            q[i] += AT(A, lda, i, j) * p[j];
    for (int64_t j = 0; j < n; j++) s[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            s[j] += AT(A, lda, i, j) * r[i];
}

/* BATAX (Section II, Fig. 1 and the operation listing of Section III-D):
 * t0 = A x ; t1 = A^T t0 ; y = t1 * beta.  ATAX of Table I is beta = 1. */
int oracle_atax(int64_t m, int64_t n, double beta, const double *A, int64_t lda,
                const double *x, double *y)
{
    double *t0 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *t1 = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!t0 || !t1) { free(t0); free(t1); return -1; }
    for (int64_t i = 0; i < m; i++) t0[i] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t0[i] += AT(A, lda, i, j) * x[j];
    for (int64_t j = 0; j < n; j++) t1[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t1[j] += AT(A, lda, i, j) * t0[i];
    for (int64_t j = 0; j < n; j++)
        y[j] = t1[j] * beta;
    free(t0); free(t1);
    return 0;
}

/* GEMVER (Table I):  B <- A + u1 v1^T + u2 v2^T ;  x <- beta B^T y + z ;
 * w <- alpha B x.  B is its own buffer (ldb); the rank-1 terms are added
 * in the order written, (A + u1 v1^T) + u2 v2^T.  x uses the new B and w
 * uses the new x. */
int oracle_gemver(int64_t m, int64_t n, double alpha, double beta,
                  const double *A, int64_t lda,
                  const double *u1, const double *v1,
                  const double *u2, const double *v2,
                  const double *y, const double *z,
                  double *B, int64_t ldb, double *x, double *w)
{
    double *t = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *t2 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t || !t2) { free(t); free(t2); return -1; }
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++)
            AT(B, ldb, i, j) = AT(A, lda, i, j);
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++)
            AT(B, ldb, i, j) = AT(B, ldb, i, j) + u1[i] * v1[j];
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++)
            AT(B, ldb, i, j) = AT(B, ldb, i, j) + u2[i] * v2[j];
    for (int64_t j = 0; j < n; j++) t[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t[j] += AT(B, ldb, i, j) * y[i];
    for (int64_t j = 0; j < n; j++)
        x[j] = beta * t[j] + z[j];
    for (int64_t i = 0; i < m; i++) t2[i] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t2[i] += AT(B, ldb, i, j) * x[j];
    for (int64_t i = 0; i < m; i++)
        w[i] = alpha * t2[i];
    free(t); free(t2);
    return 0;
}

/* GESUMMV (Table I):  y <- alpha A x + beta B x. */
int oracle_gesummv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                   double beta, const double *B, int64_t ldb,
                   const double *x, double *y)
{
    double *ta = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *tb = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!ta || !tb) { free(ta); free(tb); return -1; }
    for (int64_t i = 0; i < m; i++) { ta[i] = 0.0; tb[i] = 0.0; }
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            ta[i] += AT(A, lda, i, j) * x[j];
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            tb[i] += AT(B, ldb, i, j) * x[j];
    for (int64_t i = 0; i < m; i++)
        y[i] = alpha * ta[i] + beta * tb[i];
    free(ta); free(tb);
    return 0;
}

/* DGEMV (Table I):  z <- alpha A x + beta y. */
int oracle_dgemv(int64_t m, int64_t n, double alpha, const double *A, int64_t lda,
                 const double *x, double beta, const double *y, double *z)
{
    double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t) return -1;
    for (int64_t i = 0; i < m; i++) t[i] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t[i] += AT(A, lda, i, j) * x[j];
    for (int64_t i = 0; i < m; i++)
        z[i] = alpha * t[i] + beta * y[i];
    free(t);
    return 0;
}

/* DGEMVT (Table I):  x <- beta A^T y + z ;  w <- alpha A x  (with the new x). */
int oracle_dgemvt(int64_t m, int64_t n, double alpha, double beta,
                  const double *A, int64_t lda, const double *y, const double *z,
                  double *x, double *w)
{
    double *t = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *t2 = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t || !t2) { free(t); free(t2); return -1; }
    for (int64_t j = 0; j < n; j++) t[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t[j] += AT(A, lda, i, j) * y[i];
    for (int64_t j = 0; j < n; j++)
        x[j] = beta * t[j] + z[j];
    for (int64_t i = 0; i < m; i++) t2[i] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++)
            t2[i] += AT(A, lda, i, j) * x[j];
    for (int64_t i = 0; i < m; i++)
        w[i] = alpha * t2[i];
    free(t); free(t2);
    return 0;
}

/* AXPYDOT (Table I):  z <- w - alpha v ;  r <- z^T u.  (The table names the
 * output scalar beta; it is r here so it does not clash with the input
 * scalars of the other kernels.)  Plain ascending-order sum. */
void oracle_axpydot(int64_t n, double alpha, const double *w, const double *v,
                    const double *u, double *z, double *r)
{
    for (int64_t i = 0; i < n; i++)
        z[i] = w[i] - alpha * v[i];
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++)
        acc += z[i] * u[i];
    *r = acc;
}

/* WAXPBY (Table I):  w <- alpha x + beta y. */
void oracle_waxpby(int64_t n, double alpha, const double *x, double beta,
                   const double *y, double *w)
{
    for (int64_t i = 0; i < n; i++)
        w[i] = alpha * x[i] + beta * y[i];
}

/* VADD (Table I):  x <- w + y + z, evaluated left to right: (w + y) + z. */
void oracle_vadd(int64_t n, const double *w, const double *y, const double *z,
                 double *x)
{
    for (int64_t i = 0; i < n; i++)
        x[i] = (w[i] + y[i]) + z[i];
}

/* Compensated dot product "Dot2" of Ogita, Rump and Oishi ("Accurate sum and
 * dot product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm 5.3), built from
 * the error-free transformations TwoSum (Knuth) and TwoProduct (here with a
 * fused multiply-add, which returns the exact product error).  Its result is
 * as accurate as if computed in twice the working precision and then rounded:
 * |res - x^T y| <= u |x^T y| + gamma_n^2 |x|^T |y|.  Used as the reference for
 * dot products of length >= 2^20, where the plain ascending sum's own error is
 * near the comparison tolerance. */
static void two_sum(double a, double b, double *x, double *y)
{
    double s = a + b;
    double z = s - a;
    *x = s;
    *y = (a - (s - z)) + (b - z);
}

static void two_product(double a, double b, double *x, double *y)
{
    double p = a * b;
    *x = p;
    *y = fma(a, b, -p);
}

double oracle_dot2(int64_t n, const double *x, const double *y)
{
    if (n <= 0) return 0.0;
    double p, s, h, r, q;
    two_product(x[0], y[0], &p, &s);
    for (int64_t i = 1; i < n; i++) {
        two_product(x[i], y[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    return p + s;
}

/* Dot2 applied to the AXPYDOT dot: z is formed exactly as in oracle_axpydot,
 * then r = Dot2(z, u). */
void oracle_axpydot_dot2(int64_t n, double alpha, const double *w, const double *v,
                         const double *u, double *z, double *r)
{
    for (int64_t i = 0; i < n; i++)
        z[i] = w[i] - alpha * v[i];
    *r = oracle_dot2(n, z, u);
}

/* Multi-right-hand-side BICGK: the BICGK statements applied to k column
 * pairs at once, Q <- A P and S <- A^T R, with P (n x k, ldp) and
 * R (m x k, ldr) column-major, Q (m x k, ldq) and S (n x k, lds). */
void oracle_bicgk_mrhs(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                       const double *P, int64_t ldp, const double *R, int64_t ldr,
                       double *Q, int64_t ldq, double *S, int64_t lds)
{
    for (int64_t c = 0; c < k; c++)
        oracle_bicgk(m, n, A, lda, P + (size_t)c * (size_t)ldp, R + (size_t)c * (size_t)ldr,
                     Q + (size_t)c * (size_t)ldq, S + (size_t)c * (size_t)lds);
}

/* Sampled outputs for full-size checks: q_i = sum_j A(i,j) p_j for one row
 * given as a contiguous vector, in ascending j (identical order to
 * oracle_bicgk).  Used where the whole matrix does not fit the host budget. */
double oracle_row_dot(int64_t n, const double *row, const double *p)
{
    double acc = 0.0;
    for (int64_t j = 0; j < n; j++)
        acc += row[j] * p[j];
    return acc;
}

/* Sparse BICGK on compressed sparse rows (the sparse format the paper plans
 * in Section VII): q_i = sum over the stored entries k of row i of
 * val[k] p[col[k]], taken in storage order; s_j = sum over every stored
 * entry in column j of val[k] r_i, taken in row order then storage order.
 * Duplicated (row, column) entries add. */
void oracle_csr_bicgk(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val, const double *p, const double *r, double *q, double *s)
{
    for (int64_t j = 0; j < n; j++) s[j] = 0.0;
    for (int64_t i = 0; i < m; i++) {
        double acc = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            acc += val[k] * p[col[k]];
            s[col[k]] += val[k] * r[i];
        }
        q[i] = acc;
    }
}

/* Sparse BATAX: t = A x (row by row), then y = beta A^T t, as the dense
 * oracle_atax orders it. */
int oracle_csr_atax(int64_t m, int64_t n, double beta, const int64_t *row_ptr, const int32_t *col,
                    const double *val, const double *x, double *y)
{
    double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t) return 1;
    for (int64_t i = 0; i < m; i++) {
        double acc = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) acc += val[k] * x[col[k]];
        t[i] = acc;
    }
    for (int64_t j = 0; j < n; j++) y[j] = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) y[col[k]] += val[k] * t[i];
    for (int64_t j = 0; j < n; j++) y[j] *= beta;
    free(t);
    return 0;
}

/* Structured storage (the banded and triangular formats the paper plans in
 * Section VII).  A is m x n with A(i, j) = 0 outside the band
 * j - ku <= i <= j + kl (kl sub-diagonals, ku super-diagonals); a triangle
 * is the band with kl = 0 (upper, ku = n - 1) or ku = 0 (lower,
 * kl = m - 1).  With unit != 0 the diagonal entries are taken as 1 and never
 * read.  Only entries inside the band are read, whatever the storage holds
 * elsewhere, and only they enter the sums (an entry outside the band is
 * structurally zero, so a NaN or Inf in p or r meets no product there).
 * Storage kinds:
 *   0 full:   A(i, j) at A[i + j*ld] (ld >= m);
 *   1 band:   A(i, j) at A[(ku + i - j) + j*ld] (ld >= kl + ku + 1): column
 *             j of the band array holds the band's part of column j, the
 *             diagonal in row ku;
 *   2 packed: a square triangle stored column after column with no gaps:
 *             column j holds rows 0..j (upper) or rows j..n-1 (lower).
 */
typedef struct {
    int storage;
    int64_t m, n, kl, ku;
    int unit;
    const double *A;
    int64_t ld;
    int64_t *colstart;   /* packed: offset of column j's first stored entry */
} band_mat;

static int band_open(band_mat *b, int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit,
                     const double *A, int64_t ld)
{
    b->storage = storage; b->m = m; b->n = n; b->kl = kl; b->ku = ku; b->unit = unit;
    b->A = A; b->ld = ld; b->colstart = NULL;
    if (storage == 2) {
        /* Column j starts after every stored entry of columns 0..j-1;
         * column c holds c + 1 entries (upper) or n - c entries (lower). */
        b->colstart = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!b->colstart) return 1;
        int64_t off = 0;
        for (int64_t c = 0; c < n; c++) {
            b->colstart[c] = off;
            off += (kl == 0) ? c + 1 : n - c;
        }
    }
    return 0;
}

static void band_close(band_mat *b) { free(b->colstart); }

/* A(i, j) for (i, j) inside the band. */
static double band_get(const band_mat *b, int64_t i, int64_t j)
{
    if (b->unit && i == j) return 1.0;
    if (b->storage == 0) return b->A[(size_t)i + (size_t)j * (size_t)b->ld];
    if (b->storage == 1) return b->A[(size_t)(b->ku + i - j) + (size_t)j * (size_t)b->ld];
    /* packed: upper column j holds rows 0..j, lower column j rows j..n-1 */
    return b->A[b->colstart[j] + (b->kl == 0 ? i : i - j)];
}

/* Structured BICGK: q_i = sum over the band's columns of row i of
 * A(i, j) p_j, ascending j; s_j = sum over the band's rows of column j of
 * A(i, j) r_i, ascending i. */
int oracle_band_bicgk(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit,
                      const double *A, int64_t ld, const double *p, const double *r, double *q, double *s)
{
    band_mat b;
    if (band_open(&b, storage, m, n, kl, ku, unit, A, ld)) return 1;
    for (int64_t i = 0; i < m; i++) {
        double acc = 0.0;
        for (int64_t j = (i - kl > 0 ? i - kl : 0); j <= i + ku && j < n; j++)
            acc += band_get(&b, i, j) * p[j];
        q[i] = acc;
    }
    for (int64_t j = 0; j < n; j++) {
        double acc = 0.0;
        for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < m; i++)
            acc += band_get(&b, i, j) * r[i];
        s[j] = acc;
    }
    band_close(&b);
    return 0;
}

/* Structured BATAX: t = A x, then y = beta (A^T t), in the order of the
 * dense oracle_atax (the scale is its own loop). */
int oracle_band_atax(int storage, int64_t m, int64_t n, int64_t kl, int64_t ku, int unit, double beta,
                     const double *A, int64_t ld, const double *x, double *y)
{
    band_mat b;
    double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    if (!t || band_open(&b, storage, m, n, kl, ku, unit, A, ld)) { free(t); return 1; }
    for (int64_t i = 0; i < m; i++) {
        double acc = 0.0;
        for (int64_t j = (i - kl > 0 ? i - kl : 0); j <= i + ku && j < n; j++)
            acc += band_get(&b, i, j) * x[j];
        t[i] = acc;
    }
    for (int64_t j = 0; j < n; j++) {
        double acc = 0.0;
        for (int64_t i = (j - ku > 0 ? j - ku : 0); i <= j + kl && i < m; i++)
            acc += band_get(&b, i, j) * t[i];
        y[j] = acc;
    }
    for (int64_t j = 0; j < n; j++) y[j] = y[j] * beta;
    band_close(&b);
    free(t);
    return 0;
}
