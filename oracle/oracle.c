/*
 * FP64 reference ("oracle") for the sparse products of Eckstein & Matyasfalvi,
 * "Efficient Distributed-Memory Parallel Matrix-Vector Multiplication with
 * Wide or Tall Unstructured Sparse Matrices" (arXiv 1812.00904).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * links, includes or calls it, and this file shares no code with it.
 *
 * Every routine is the plain definition written out as straight loops over the
 * compressed arrays, in double precision, one nonzero at a time, in storage
 * order.  Inputs of narrower types are widened exactly by the caller before
 * they reach these loops.
 *
 * Problem statement (Sec. I): A is m x n with Z nonzeros,
 *     SpMV   y = A x,        y_i = sum_j A_ij x_j        (x in R^n, y in R^m)
 *     SpVTM  u^T = v^T A,    u_j = sum_i v_i A_ij        (v in R^m, u in R^n)
 * Storage (Sec. II): a wide matrix is kept column-major (CSC: ptr has n+1
 * entries, column j owns positions ptr[j] .. ptr[j+1]-1 with row ids in idx);
 * a tall matrix is kept row-major (CSR), i.e. the same arrays with the roles
 * of rows and columns reversed.  Indices are 0-based.  Repeated indices inside
 * one column (row) simply contribute several terms.
 */
#include <stdint.h>

/* Sec. I, y = A x with A in CSC (Sec. II): every nonzero A_ij adds A_ij x_j to y_i. */
void oracle_csc_matvec(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                       const double *val, const double *x, double *y)
{
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) {
            y[idx[k]] += val[k] * x[j];
        }
    }
}

/* Sec. I, u^T = v^T A with A in CSC: u_j is the dot product of column j with v. */
void oracle_csc_vecmat(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                       const double *val, const double *v, double *u)
{
    (void)m;
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) {
            s += v[idx[k]] * val[k];
        }
        u[j] = s;
    }
}

/* Sec. I/II, y = A x with A in CSR (tall, roles reversed): y_i is the dot product of row i with x. */
void oracle_csr_matvec(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                       const double *val, const double *x, double *y)
{
    (void)n;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            s += val[k] * x[idx[k]];
        }
        y[i] = s;
    }
}

/* Sec. I/II, u^T = v^T A with A in CSR: every nonzero A_ij adds v_i A_ij to u_j. */
void oracle_csr_vecmat(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                       const double *val, const double *v, double *u)
{
    for (int64_t j = 0; j < n; ++j) u[j] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            u[idx[k]] += v[i] * val[k];
        }
    }
}

/*
 * Gradient of y = A x with respect to the stored values: for the nonzero at
 * position k holding A_ij, d(r^T A x)/dA_ij = r_i x_j.  CSC: i = idx[k],
 * j = column of k.
 */
void oracle_csc_dvalues(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                        const double *r, const double *x, double *g)
{
    (void)m;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t k = ptr[j]; k < ptr[j + 1]; ++k) {
            g[k] = r[idx[k]] * x[j];
        }
    }
}

/* Same with A in CSR: i = row of k, j = idx[k]. */
void oracle_csr_dvalues(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx,
                        const double *r, const double *x, double *g)
{
    (void)n;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            g[k] = r[i] * x[idx[k]];
        }
    }
}
