/*
 * spmv_gb300.h -- C ABI of the GB300 (sm_103a) wide/tall sparse product library.
 *
 * Implements the two products of Eckstein & Matyasfalvi, "Efficient
 * Distributed-Memory Parallel Matrix-Vector Multiplication with Wide or Tall
 * Unstructured Sparse Matrices" (arXiv 1812.00904):
 *
 *   SpMV   y = A x          (Sec. I)        A is m x n with Z nonzeros
 *   SpVTM  u^T = v^T A      (Sec. I)
 *
 * for a wide matrix stored column-major (CSC, m << n) or a tall matrix stored
 * row-major (CSR, m >> n; Sec. II, "reversing the roles of rows and columns").
 * The nonzeros are split into P contiguous, equally sized chunks whatever the
 * column boundaries (Sec. II); chunks that share a column (an "overlap zone")
 * combine their partial dot products through per-chunk carry records and a
 * fixed-order reduction (Sec. IV-A), with the zones numbered by the set-up
 * scans of Sec. IV-B.  On the GPU the same rule is applied twice: the P
 * reporting chunks (whose set-up quantities spmv_plan_chunks returns) and the
 * execution tiles of tile_items nonzeros, each tile a processor of the kernels
 * with its own carry records.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Indices are 0-based int32.  ptr has (n+1) entries for CSC, (m+1) for CSR;
 *    ptr[0] = 0, ptr non-decreasing, ptr[last] = nnz < 2^31.  idx entries lie in
 *    [0, m) for CSC and [0, n) for CSR.  Repeated indices in one column (row)
 *    add up; indices need not be sorted; empty columns (rows) are allowed.
 *  - Element types (spmv_dtype): values and vectors are one of the pairs
 *    (F64, F64), (F32, F32), (BF16, F32), (F16, F32).  Accumulation inside a
 *    chunk is FP32 for the last three and FP64 for the first; the cross-chunk
 *    combines (the sum of the per-CTA partial vectors of spmv, the overlap-zone
 *    fix-up of spvtm) add in FP64 for every pair, in a fixed order.
 *  - Infinities and NaNs in the values or vectors give what the plain sum gives
 *    (an infinity of one sign, or NaN where infinities of both signs or a NaN
 *    meet), also through the compensated carries of split columns; subnormal
 *    values and sums are kept (nothing is flushed to zero).
 *  - A plan BORROWS the caller's device arrays ptr/idx/vals: they must stay
 *    allocated and unchanged (values may change between calls) until
 *    spmv_plan_destroy.  The plan owns only its workspace.
 *  - The products of one plan share its workspace (partial vectors, carry records,
 *    staging buffers): calls on the same plan must not overlap on the device, i.e.
 *    issue them on one stream or order the streams (spmv_pair runs its two products
 *    side by side itself).  Different plans are independent.
 *  - Device pointers must be 16-byte aligned (cudaMalloc and torch allocations
 *    are); a misaligned pointer is rejected with SPMV_ERR_INVALID_ARG.
 *  - Vector arguments of spmv, spvtm and spmv_dvalues may be device pointers or
 *    host pointers (pinned or pageable).  With device pointers the call is
 *    asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *    With host pointers the library copies through its own device buffers and
 *    the call returns after the result has landed in host memory.
 *  - Outputs are overwritten (no alpha/beta).
 *  - No call aborts the process.  Failures return a status; spmv_last_error()
 *    gives a thread-local message.  Kernels never trap: a device-side failure
 *    (an index out of range, a staging wait that timed out) sets an error word
 *    that spmv_check() reports as SPMV_ERR_DEVICE; the outputs of the call that
 *    set it are unspecified (out-of-range indices are never dereferenced).
 */
#ifndef SPMV_GB300_H
#define SPMV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, bad size or dtype pair */
    SPMV_ERR_BAD_MATRIX = 2,   /* ptr/idx fail the structural checks above */
    SPMV_ERR_OOM = 3,          /* a device or host allocation failed */
    SPMV_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    SPMV_ERR_DEVICE = 5,       /* a kernel reported a failure through the error word */
    SPMV_ERR_TIMEOUT = 6,      /* serve_wait ran out of time */
    SPMV_ERR_BUSY = 7,         /* serving: no room (HBM budget / queue) right now */
    SPMV_ERR_UNSUPPORTED = 8,  /* valid request this build does not implement */
    SPMV_ERR_NOT_FOUND = 9     /* unknown matrix or request id */
} spmv_status;

typedef enum { SPMV_CSC_WIDE = 0, SPMV_CSR_TALL = 1 } spmv_layout;            /* Sec. II */
typedef enum { SPMV_F64 = 0, SPMV_F32 = 1, SPMV_BF16 = 2, SPMV_F16 = 3 } spmv_dtype;
typedef enum { SPMV_OP_AX = 0, SPMV_OP_VTA = 1 } spmv_op;                       /* Sec. I */

typedef struct spmv_plan_s *spmv_plan_t;

/* Plan flags. */
#define SPMV_PLAN_NO_VALIDATE 0x1u  /* skip the structural checks of ptr/idx at plan time; the kernels then
                                       check every index (an out-of-range one is clamped and reported by
                                       spmv_check).  A validated plan relies on idx staying unchanged. */
#define SPMV_PLAN_PROFILE 0x2u      /* time every kernel launch with CUDA events (spmv_profile_read) */
#define SPMV_PLAN_SHORT_IN_GLOBAL 0x4u /* keep the short vector in global memory even when it fits on chip */
#define SPMV_PLAN_BANK_ORDER 0x8u   /* keep a plan-owned copy of idx and vals in which the nonzeros of every
                                       column (row for CSR) are permuted so that the short-vector entries one
                                       warp instruction touches fall into distinct shared-memory banks.  Costs
                                       nnz x (4 + value size) bytes for the plan's life and as much again for
                                       scratch during spmv_plan; idx and vals are not read after spmv_plan
                                       returns; results equal the stored order's up to the order of rounding;
                                       spmv_dvalues answers SPMV_ERR_UNSUPPORTED (its g would be permuted). */
#define SPMV_PLAN_ROW_BLOCKS 0x20u   /* keep a second plan-owned copy of the nonzeros for the product that
                                       accumulates into the short vector (y = A x of a wide CSC matrix,
                                       u^T = v^T A of a tall CSR one): the nonzeros are cut into blocks of
                                       whole tiles (a multiple of the SM count; a CTA runs one or more in
                                       turn) and sorted inside
                                       each block by their short-vector index, so that product runs as
                                       segmented dot products over each block's window of the long vector in
                                       shared memory, without atomics and bitwise reproducibly, and the
                                       per-block vectors are added in FP64 in block order.  Costs
                                       nnz x (4 + value size) bytes plus (blocks x short length) vector
                                       entries for the plan's life and about nnz x 36 bytes of scratch
                                       during spmv_plan.  Ignored (spmv_plan_info: row_blocks = 0) when the
                                       plan skips validation, when the windows would not fit in shared
                                       memory, or when the blocks would hold fewer than 8 nonzeros per
                                       short-vector entry. */
#define SPMV_PLAN_COO_UNSORTED 0x10u /* spmv_plan_coo only: the triples may come in any order; the plan sorts
                                       them on the device by (major, minor) index, stably (duplicates keep
                                       their input order), into its own copy of the minor indices and values
                                       (nnz x (4 + value size) bytes; about 3 x nnz x 12 bytes of scratch
                                       during the call).  Both indices are range-checked even with
                                       SPMV_PLAN_NO_VALIDATE. */

/* Optional tuning of a plan; zero fields take the defaults. */
typedef struct {
    int32_t chunks;        /* P, the number of reporting chunks (Sec. II); 0 = min(tiles, 16 per SM) */
    int32_t warps_per_cta; /* most warps per CTA, 1..24 (at most 16 run the multi-vector passes);
                              0 = 24; every pass runs as many as its staging slots fit in shared
                              memory (up to 16 warps with 128 registers a thread, more with 80) */
    int32_t tile_items;    /* nonzeros per execution tile, a multiple of 8 in [8, 992]; 0 = 512, or
                              down to 64 when nnz < 32 x 512 per SM (about two tiles per warp) */
    int32_t stages;        /* staging slots per warp (tiles in flight + 1), 2..4; 0 = 2 */
    int32_t chunk_tiles;   /* consecutive tiles a warp streams as one processor, 1..64 (segments that
                              run on between them are carried in registers; overlap zones arise only
                              between chunks); 0 = 8.  The last MAX(24 (C + 1)) tiles of every CTA
                              are single-tile chunks, which balance the warps. */
} spmv_plan_opts;

/* Summary of a plan (spmv_plan_info). */
typedef struct {
    int64_t m, n, nnz;
    int32_t layout, val_dtype, vec_dtype;
    int32_t chunks;            /* P */
    int32_t ctas, warps_per_cta, tile_items, stages;
    int32_t tiles;             /* execution tiles */
    int32_t zones;             /* z, overlap zones (Sec. II), z <= P-1 */
    int32_t max_zone_size;     /* V = max |S_k| (Sec. IV-A) */
    int32_t short_on_chip;     /* 1 if the short vector lives in shared memory */
    int32_t batch_width;       /* vectors per pass of the accumulating direction of spmv_batch (1..8) */
    int64_t max_chunk_nnz, min_chunk_nnz;
    double imbalance;          /* Delta = P (max - min) / Z (Sec. VI), 0 when Z = 0 */
    int64_t workspace_bytes;   /* device bytes owned by the plan */
    double setup_ms;           /* device time of the set-up kernels */
    int32_t row_blocks;        /* blocks of the row-sorted copy (SPMV_PLAN_ROW_BLOCKS), 0 if none */
    int32_t row_block_window;  /* widest window of the long vector a block reads (elements) */
} spmv_plan_info_t;

/* Per-chunk set-up values (spmv_plan_chunks), one per chunk p_c (Sec. IV-B, Table III). */
typedef struct {
    int64_t nz_begin, nz_end;   /* nonzeros [begin, end) of the chunk (Sec. II rule) */
    int32_t jf, jl;             /* first / last column (row for CSR) j^f, j^l; -1 if the chunk is empty */
    int32_t needLeft, needRight, leftGroupEnd, rightGroup, leftGroup, procsOnLeft, procsOnRight;
} spmv_chunk_t;

/*
 * spmv_plan -- build the execution plan of one matrix (Sec. II partition and
 * Sec. IV-B overlap-zone set-up, computed on the device).
 *   out        receives the plan handle (owned by the caller; free with spmv_plan_destroy)
 *   m, n, nnz  matrix shape and nonzero count (0 <= nnz < 2^31; m, n < 2^31)
 *   layout     SPMV_CSC_WIDE or SPMV_CSR_TALL
 *   ptr, idx   device arrays (int32), see conventions; borrowed
 *   vals       device array of nnz values of type val_dtype; borrowed
 *   vec_dtype  element type of the dense vectors
 *   stream     cudaStream_t for the set-up kernels; the call synchronizes it (after
 *              validation, after the bank-order copy when asked for, and at the end)
 *              and returns with the plan ready
 *   flags      SPMV_PLAN_* bits
 * Errors: SPMV_ERR_INVALID_ARG, SPMV_ERR_BAD_MATRIX (checked unless
 * SPMV_PLAN_NO_VALIDATE), SPMV_ERR_OOM, SPMV_ERR_CUDA, SPMV_ERR_UNSUPPORTED.
 * On error *out is set to NULL and nothing is leaked.
 */
spmv_status spmv_plan(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                      const int32_t *ptr, const int32_t *idx, const void *vals,
                      int32_t val_dtype, int32_t vec_dtype, void *stream, uint32_t flags);

/* spmv_plan with explicit tuning (opts may be NULL). */
spmv_status spmv_plan_ex(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                         const int32_t *ptr, const int32_t *idx, const void *vals,
                         int32_t val_dtype, int32_t vec_dtype, void *stream, uint32_t flags,
                         const spmv_plan_opts *opts);

/*
 * spmv_plan_coo -- a plan from coordinate triples in storage order: sorted by
 * column for SPMV_CSC_WIDE (the column-major triple stream of Sec. V), by row for
 * SPMV_CSR_TALL; order inside a column (row) is free and repeated (i, j) add up.
 *   rows, cols (nnz int32 each), vals (nnz, val_dtype): device arrays, BORROWED like
 *   idx/vals of spmv_plan (the minor indices serve as idx); the plan builds and owns
 *   the pointer array on the device.  Other arguments as for spmv_plan_ex.
 * With SPMV_PLAN_COO_UNSORTED the triples may come in any order: a stable device
 * radix sort by (major, minor) puts them in storage order in a plan-owned copy, and
 * rows, cols and vals are not read after the call returns.
 * Synchronizes `stream` once for the triples, then as spmv_plan_ex does.  Errors:
 * SPMV_ERR_BAD_MATRIX when a major index (or, unsorted, either index) is out of
 * range or a sorted stream is not sorted by the major index, SPMV_ERR_OOM, then the
 * errors of spmv_plan_ex.
 */
spmv_status spmv_plan_coo(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                          const int32_t *rows, const int32_t *cols, const void *vals, int32_t val_dtype,
                          int32_t vec_dtype, void *stream, uint32_t flags, const spmv_plan_opts *opts);

/* Release the plan's workspace.  Accepts NULL.  The caller's arrays are untouched. */
spmv_status spmv_plan_destroy(spmv_plan_t plan);

/* Copy the plan summary into *info (host memory). */
spmv_status spmv_plan_info(spmv_plan_t plan, spmv_plan_info_t *info);

/* Copy the per-chunk set-up values of chunks [0, count) into out[] (host), count <= P. Synchronous. */
spmv_status spmv_plan_chunks(spmv_plan_t plan, spmv_chunk_t *out, int32_t count);

/*
 * spmv -- y = A x (Sec. I; Sec. III for the chunked computation: every chunk
 * accumulates A_(i) x_(i) into an on-chip copy of the short vector, and the
 * per-CTA partial vectors are summed in FP64 in a fixed order).
 *   x  n values of vec_dtype (device or host);  y  m values of vec_dtype (device or host), overwritten.
 */
spmv_status spmv(spmv_plan_t plan, const void *x, void *y, void *stream);

/*
 * spvtm -- u^T = v^T A (Sec. I; Sec. IV-A: every chunk dots its partial
 * columns with v; columns split between chunks are completed from carry
 * records, u_j = sum over S_k of v^T A_j^p, in FP64 and a fixed order).
 *   v  m values of vec_dtype (device or host);  u  n values of vec_dtype (device or host), overwritten.
 */
spmv_status spvtm(spmv_plan_t plan, const void *v, void *u, void *stream);

/*
 * spmv_batch -- k products of the same kind.  op = SPMV_OP_AX: Y = A X, vector b
 * of X at in + b*ld_in (length n), of Y at out + b*ld_out (length m);
 * op = SPMV_OP_VTA: U^T = V^T A with lengths m in, n out.  ld in elements,
 * ld >= vector length and ld * element size a multiple of 16.  Device pointers
 * only.  1 <= k <= 4096.  The segmented direction (SpVTM of a wide CSC plan,
 * SpMV of a tall CSR one, and the SpMV of a plan with SPMV_PLAN_ROW_BLOCKS)
 * streams the matrix once per 8 vectors, and every vector's result equals its
 * single-vector product bit for bit, whatever k and the vector's place in the
 * batch.  The accumulating direction runs batch_width vectors (spmv_plan_info)
 * per pass; its results equal the single-vector products within the stated
 * tolerances (floating-point atomic additions, in no fixed order).  The paper
 * multiplies one vector at a time; the multi-vector form has no counterpart
 * there (each vector's product is the Sec. III / Sec. IV-A computation).
 */
spmv_status spmv_batch(spmv_plan_t plan, int32_t op, int32_t k, const void *in, int64_t ld_in,
                       void *out, int64_t ld_out, void *stream);

/*
 * spmv_dvalues -- gradient of r^T A x with respect to the stored values:
 * g[p] = r_i x_j for the nonzero at position p holding A_ij.  r has m entries,
 * x has n (vec_dtype); g has nnz entries of the plan's val_dtype.  This is the
 * d(values) part of the backward pass of y = A x (with r = dL/dy); the dx part
 * is spvtm(plan, r).  Device or host pointers.  No counterpart in the paper
 * (the gradient of the product, computed with the plan's Sec. II partition).
 */
spmv_status spmv_dvalues(spmv_plan_t plan, const void *r, const void *x, void *g, void *stream);

/*
 * spmv_plan_export -- copy the nonzeros the plan multiplies by into caller buffers:
 * idx_out (nnz int32) and vals_out (nnz values of val_dtype), device or host
 * pointers, in the plan's storage order (the caller's order, or the plan's bank
 * order under SPMV_PLAN_BANK_ORDER).  Synchronizes `stream`.
 * Errors: SPMV_ERR_INVALID_ARG (null plan or buffer), SPMV_ERR_CUDA.
 */
spmv_status spmv_plan_export(spmv_plan_t plan, int32_t *idx_out, void *vals_out, void *stream);

/* Synchronize `stream`, then read and clear the plan's device error word.
 * Returns SPMV_ERR_DEVICE (with a message) if any kernel flagged a failure. */
spmv_status spmv_check(spmv_plan_t plan, void *stream);

/* Kernel timers of a plan created with SPMV_PLAN_PROFILE (or switched on with
 * spmv_profile_enable).  kernel: 0 = chunk scatter (SpMV local), 1 = partial
 * combine, 2 = chunk dot (SpVTM local), 3 = zone fixup, 4 = dvalues,
 * 5 = row-block dot (the SpMV local step over the row-sorted copy), 6 = its zone fixup.
 * Synchronizes the device.  *ms = summed event time, *launches = number of
 * timed launches.  Timing brackets every launch with two events, which waits
 * for each kernel to drain before the next starts: a profiled sequence of
 * launches runs a little slower than an unprofiled one. */
spmv_status spmv_profile_read(spmv_plan_t plan, int32_t kernel, double *ms, int64_t *launches);
spmv_status spmv_profile_reset(spmv_plan_t plan);
/* Switch the kernel timers of a plan on (on != 0) or off for the launches that follow;
 * the sums read by spmv_profile_read are kept.  Errors: SPMV_ERR_INVALID_ARG. */
spmv_status spmv_profile_enable(spmv_plan_t plan, int32_t on);

/*
 * spmv_noalloc -- y = A x for a wide CSC matrix (FP32 values and vectors)
 * without any device allocation, for callers that may not allocate device
 * memory when they multiply: code inside a memory pool or runtime that hands
 * the library only pre-sized buffers.  The paper has no counterpart; this is
 * a convenience path beside spmv_plan/spmv.
 *   m, n, nnz, ptr, idx, vals  the CSC matrix (device arrays, conventions above); m <= 49152
 *   x (n floats), y (m floats)  device vectors; y is overwritten
 *   stream                      cudaStream_t; the call is asynchronous on it
 * Scratch: the per-CTA partial vectors live in a 16 MiB array in the
 * library's static device memory, held by every device that loads the
 * library until the process exits.  All calls share it, so calls that
 * overlap on the GPU race and give wrong results; serialize them (one stream,
 * or events).  The first call on a device resolves the array's device address
 * (a host-side query, once per device).  Nothing is allocated; an m above 49152 or a bad size is rejected with
 * SPMV_ERR_INVALID_ARG before any launch.  The matrix is not validated and
 * device-side problems are not reported (there is no error word to read back):
 * a nonzero whose row index lies outside [0, m) is skipped, and a malformed ptr
 * never makes the kernel read outside ptr[0..n], idx, vals or x[0..n), but the
 * result is then unspecified.
 */
spmv_status spmv_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *ptr, const int32_t *idx,
                         const float *vals, const float *x, float *y, void *stream);

/*
 * spmv_pair -- y = A x (Sec. III) and u = v^T A (Sec. IV-A) for independent x and v in one
 * call: the paper's SpMV-SpVTM pair (Sec. V) where the second product does not consume the
 * first's result.  No counterpart in the paper beyond the two products.
 *   x (n), y (m), v (m), u (n): vectors of the plan's vector type, each on the device (16-byte
 *   aligned) or in host memory (pinned or pageable); y and u are overwritten.  The four must not
 *   overlap: the two products may run at the same time.
 * With device pointers only, the call is asynchronous: the SpMV runs on `stream` and the SpVTM
 * beside it on a stream of the plan, forked after the work already queued on `stream` and joined
 * back into it (work queued on `stream` after the call sees both results).  Otherwise the
 * library stages the host vectors through its own device buffers on `stream` and on a copy
 * stream of its own: v's copy is queued first, the copy of x to the device overlaps the SpVTM
 * kernels and the copy of u to the host overlaps the SpMV kernels, and the call returns after y
 * and u have landed (work queued on `stream` before the call completes first).  Errors as for
 * spmv and spvtm.
 */
spmv_status spmv_pair(spmv_plan_t plan, const void *x, void *y, const void *v, void *u, void *stream);

/*
 * spmv_normal -- u = A^T (A x), the normal-equation operator of least squares:
 * one SpMV (Sec. III) whose result feeds one SpVTM (Sec. IV-A), the pairing the
 * paper measures (Sec. V) with the SpVTM consuming the SpMV's output.
 *   x (n), u (n): 16-byte aligned device vectors of the plan's vector type; u is overwritten
 *   y (m): device buffer that receives A x, or NULL (the plan keeps its own, allocated once)
 * Asynchronous on `stream`.  Errors as for spmv/spvtm.
 */
spmv_status spmv_normal(spmv_plan_t plan, const void *x, void *u, void *y, void *stream);

/*
 * spmv_cgls -- least squares min ||A x - b||_2 by conjugate gradients on the
 * normal equations (CGLS), the kind of first-order method the SpMV-SpVTM pairs of
 * the paper serve (Sec. V, Sec. VII); there is no such solver in the paper.  Every
 * product and vector operation runs on the device; the iteration's scalars stay in
 * device memory and the host reads them every 8 iterations to stop.
 *   b (m), x (n)    16-byte aligned device vectors of the plan's vector type; x holds
 *                   the start on entry (zeros for the minimum-norm solution of an
 *                   underdetermined problem) and the last iterate on return
 *   max_iters, tol  stop after max_iters iterations or once ||A^T r|| <= tol ||A^T r_0||
 *   iters_done, rel_grad  (may be NULL) iterations run and ||A^T r|| / ||A^T r_0||
 * Synchronizes `stream`; allocates its work vectors (4 vectors and a few scalars)
 * for the duration of the call.
 */
spmv_status spmv_cgls(spmv_plan_t plan, const void *b, void *x, int32_t max_iters, double tol, void *stream,
                      int32_t *iters_done, double *rel_grad);

/* Thread-local message for the last failing call of this thread ("" if none). */
const char *spmv_last_error(void);

/* Library version string. */
const char *spmv_version(void);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of single products over resident matrices.
 * The paper has no serving layer; every product a server runs is the spmv /
 * spvtm / spmv_batch computation above. */

typedef struct serve_s *serve_t;

/*
 * serve_create -- start a serving runtime with its own scheduler thread.
 *   hbm_budget_bytes  device bytes the resident matrices (and their plans) may use
 *   k_max             most vectors coalesced into one multi-vector launch (1..64)
 *   n_streams         CUDA streams that run launches concurrently (1..16)
 */
spmv_status serve_create(serve_t *out, uint64_t hbm_budget_bytes, int32_t k_max, int32_t n_streams);

/* Register an existing plan (its arrays already on the device; never evicted).
 * Its footprint counts against the budget: SPMV_ERR_BUSY if it does not fit. */
spmv_status serve_register(serve_t srv, spmv_plan_t plan, int32_t *mat_id);

/* Register a matrix held in HOST memory (borrowed until serve_destroy).  It is
 * copied to the device and planned when a request needs it and the budget
 * allows; idle host-registered matrices are evicted (least recently used) to
 * admit others.  The copy and the planning run on the runtime's admission
 * thread, so requests on resident matrices keep running meanwhile. */
spmv_status serve_register_host(serve_t srv, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                                const int32_t *ptr, const int32_t *idx, const void *vals,
                                int32_t val_dtype, int32_t vec_dtype, int32_t *mat_id);

/*
 * serve_submit -- queue k products of matrix mat_id: op = SPMV_OP_AX computes
 * out_b = A in_b, SPMV_OP_VTA computes out_b^T = in_b^T A, vector b at
 * in + b*len_in and out + b*len_out (device memory, vec_dtype, contiguous).
 * Returns at once with *req_id.  The request joins the next launch of the same
 * (matrix, op) with room; the buffers must stay valid until it completes.
 * The runtime reads `in` on its own streams with no ordering against the
 * caller's: `in` must be complete on the device when serve_submit is called
 * (synchronize the stream that produced it first).  `out` holds the results
 * once serve_poll or serve_wait reports the request done.
 */
spmv_status serve_submit(serve_t srv, int32_t mat_id, int32_t op, int32_t k,
                         const void *in, void *out, uint64_t *req_id);

/* Non-blocking status: *done = 1 once the results are in `out`; *latency_ms =
 * submit-to-completion time (valid when done).  A finished request that failed
 * returns its error status.  The first serve_poll or serve_wait that reports a
 * request finished retires it from the runtime's request table into a window of
 * the 65,536 most recently reported requests, which later calls still answer;
 * after that its id is unknown (SPMV_ERR_NOT_FOUND).  A request whose completion
 * is never asked for stays in the table until serve_destroy. */
spmv_status serve_poll(serve_t srv, uint64_t req_id, int32_t *done, double *latency_ms);

/* Block until the request completes or timeout_ms passes (SPMV_ERR_TIMEOUT); on
 * completion the request is retired as by serve_poll. */
spmv_status serve_wait(serve_t srv, uint64_t req_id, int32_t timeout_ms);

/* Counters of a serving runtime. */
typedef struct {
    int64_t submitted, completed, failed, vectors, launches;
    int64_t admissions, evictions, resident_matrices;
    uint64_t resident_bytes;
    int32_t max_inflight_launches;
    int64_t tracked_requests;  /* requests in the table: queued, running, or finished and not yet reported */
} serve_stats_t;

spmv_status serve_stats(serve_t srv, serve_stats_t *out);

/* Stop the scheduler after the queued requests finish and free everything. */
spmv_status serve_destroy(serve_t srv);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_GB300_H */
