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
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

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

/*
 * All-core variants of the four product loops, for timing the CPU baseline on
 * every host core.  Each is the serial loop above run over a contiguous range of
 * the major index (columns for CSC, rows for CSR) per thread; the ranges split
 * the nonzeros evenly (the Sec. II rule applied to whole columns/rows).
 *  - dot-product directions (CSC vecmat, CSR matvec): every output entry is
 *    computed by one thread with the serial loop, so the result equals the
 *    serial one bit for bit;
 *  - scatter directions (CSC matvec, CSR vecmat): every thread adds into its own
 *    zeroed copy of the output, and the copies are then summed in thread order
 *    (a different rounding order from the serial loop).
 * Returns 0, or -1 if a thread or its buffer could not be created.
 */
typedef struct {
    int csr, scatter;
    int64_t lo, hi, len_out;
    const int32_t *ptr, *idx;
    const double *val, *vin;
    double *out;
} oracle_job;

static void *oracle_job_run(void *arg)
{
    const oracle_job *J = (const oracle_job *)arg;
    if (J->scatter) {
        for (int64_t i = 0; i < J->len_out; ++i) J->out[i] = 0.0;
        for (int64_t a = J->lo; a < J->hi; ++a) {
            for (int64_t k = J->ptr[a]; k < J->ptr[a + 1]; ++k) {
                if (J->csr)
                    J->out[J->idx[k]] += J->vin[a] * J->val[k];
                else
                    J->out[J->idx[k]] += J->val[k] * J->vin[a];
            }
        }
    } else {
        for (int64_t a = J->lo; a < J->hi; ++a) {
            double s = 0.0;
            for (int64_t k = J->ptr[a]; k < J->ptr[a + 1]; ++k) {
                if (J->csr)
                    s += J->val[k] * J->vin[J->idx[k]];
                else
                    s += J->vin[J->idx[k]] * J->val[k];
            }
            J->out[a] = s;
        }
    }
    return NULL;
}

/* first major index a with ptr[a] >= target (a in [0, n_major]) */
static int64_t oracle_lower_major(const int32_t *ptr, int64_t n_major, int64_t target)
{
    int64_t lo = 0, hi = n_major;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (ptr[mid] < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

static int oracle_parallel(int csr, int scatter, int64_t n_major, int64_t len_out, const int32_t *ptr,
                           const int32_t *idx, const double *val, const double *vin, double *out, int threads)
{
    if (threads < 1) threads = 1;
    const int64_t nnz = ptr[n_major];
    oracle_job *jobs = (oracle_job *)calloc((size_t)threads, sizeof(oracle_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    double *priv = scatter ? (double *)malloc((size_t)threads * (size_t)(len_out > 0 ? len_out : 1) * sizeof(double))
                           : NULL;
    if (!jobs || !tids || (scatter && !priv)) {
        free(jobs);
        free(tids);
        free(priv);
        return -1;
    }
    int started = 0, rc = 0;
    for (int t = 0; t < threads; ++t) {
        oracle_job *J = &jobs[t];
        J->csr = csr;
        J->scatter = scatter;
        J->lo = oracle_lower_major(ptr, n_major, nnz * t / threads);
        J->hi = (t == threads - 1) ? n_major : oracle_lower_major(ptr, n_major, nnz * (t + 1) / threads);
        if (t > 0) J->lo = jobs[t - 1].hi;
        J->len_out = len_out;
        J->ptr = ptr;
        J->idx = idx;
        J->val = val;
        J->vin = vin;
        J->out = scatter ? priv + (size_t)t * (size_t)len_out : out;
    }
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tids[t], NULL, oracle_job_run, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        started = t;
    }
    if (rc == 0) oracle_job_run(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tids[t], NULL);
    if (rc == 0 && scatter) {
        for (int64_t i = 0; i < len_out; ++i) {
            double s = 0.0;
            for (int t = 0; t < threads; ++t) s += priv[(size_t)t * (size_t)len_out + i];
            out[i] = s;
        }
    }
    free(jobs);
    free(tids);
    free(priv);
    return rc;
}

int oracle_csc_matvec_mt(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx, const double *val,
                         const double *x, double *y, int threads)
{
    return oracle_parallel(0, 1, n, m, ptr, idx, val, x, y, threads);
}

int oracle_csc_vecmat_mt(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx, const double *val,
                         const double *v, double *u, int threads)
{
    (void)m;
    return oracle_parallel(0, 0, n, n, ptr, idx, val, v, u, threads);
}

int oracle_csr_matvec_mt(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx, const double *val,
                         const double *x, double *y, int threads)
{
    (void)n;
    return oracle_parallel(1, 0, m, m, ptr, idx, val, x, y, threads);
}

int oracle_csr_vecmat_mt(int64_t m, int64_t n, const int32_t *ptr, const int32_t *idx, const double *val,
                         const double *v, double *u, int threads)
{
    return oracle_parallel(1, 1, m, n, ptr, idx, val, v, u, threads);
}
