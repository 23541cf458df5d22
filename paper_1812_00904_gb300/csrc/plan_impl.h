// The plan object behind spmv_plan_t, shared by the C ABI and the serving runtime.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/spmv_gb300.h"
#include "internal.h"

struct spmv_plan_s {
    int device = 0;
    int64_t m = 0, n = 0, nnz = 0;
    int layout = 0, val_t = 0, vec_t = 0;
    uint32_t flags = 0;
    int n_major = 0, n_minor = 0;
    const int32_t *ptr = nullptr, *idx = nullptr;
    const void *vals = nullptr;
    int sv = 4, sx = 4, sa = 4;

    // launch configuration
    int P = 0;          // reporting chunks (the paper's P; spmv_plan_chunks)
    int ntiles = 0;     // execution tiles (every tile a processor of the kernels)
    int ctas = 0, W = 0, T = 0, S = 0;  // W: most warps per CTA (each pass fits what shared memory holds)
    int W_info = 0;                       // warps of the single-vector scatter pass (spmv_plan_info)
    int mwp = 0, x_cap = 0, pptr_len = 0, smem_max = 0;  // masks words per tile, window elements per tile
    int mwq = 0;                // entries per tile of the head-count prefix table (a multiple of 8)
    int chunk_tiles = 1;  // tiles per chunk of the streaming kernels' full rounds
    int bpc = 1;          // blocks (Sec. II ranges of whole tiles) each CTA runs in turn
    bool onchip = false;
    int batch_width = 1;

    // plan-owned device memory
    void *ws = nullptr;     // pointer copy, reporting chunks, counters
    void *ws2 = nullptr;    // tile descriptors, masks, zones, records, partials
    size_t ws_bytes = 0;
    int32_t *pptr = nullptr;
    gbk::ChunkAux *aux = nullptr;          // reporting chunks (P)
    gbk::ChunkDev *chunks = nullptr;
    gbk::ZoneDev *zones = nullptr;
    int32_t *counts = nullptr;
    int32_t *err = nullptr;
    gbk::TileMeta *meta = nullptr;         // execution tiles (ntiles + 1)
    uint32_t *masks = nullptr;
    uint16_t *pfx = nullptr;    // per tile: segment starts before each mask word (then the total)
    // Overlap zones among the processors of the streaming passes: the chunks of whole tiles
    // (contiguous Sec. II groups) every CTA's tile range is cut into.
    struct ProcZones {
        int nproc = 0;  // processors (chunks), the stride of the carry records
        int z = 0;      // overlap zones among them
        gbk::ZoneDev *zones = nullptr;
    };
    ProcZones pz;
    int max_nproc = 0;
    void *rec_left = nullptr, *rec_right = nullptr;  // (hi, lo) pairs of the accumulation type
    void *part = nullptr;
    int z = 0, vmax = 0;
    double setup_ms = 0.0;
    int64_t max_chunk = 0, min_chunk = 0;

    // staging buffers for host-pointer calls (allocated on first use)
    std::mutex host_mu;
    void *hin = nullptr, *hout = nullptr, *hg = nullptr;
    // spmv_pair with host vectors: device copies of v and u, and a copy stream of the plan's own
    // with its two events (made on first use)
    void *hv = nullptr, *hu = nullptr;
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_x = nullptr, ev_u = nullptr;
    void *ynorm = nullptr;  // A x of spmv_normal when the caller passes no buffer
    void *owned_ptr = nullptr;  // pointer array built by spmv_plan_coo (the other arrays stay borrowed)
    void *owned_nz = nullptr;   // plan-owned idx and vals: bank order, or triples sorted by spmv_plan_coo
    size_t owned_bytes = 0;

    // row-sorted blocks (SPMV_PLAN_ROW_BLOCKS): the sub-plan over the sorted copy and its buffers
    spmv_plan_s *tplan = nullptr;
    int blocks = 0, block_window = 0;
    void *bws = nullptr;        // windows, the copy's pointer array, per-block short vectors
    size_t bws_bytes = 0;
    void *bown = nullptr;       // the sorted copy's indices and values (when the sub-plan borrows them)
    size_t bown_bytes = 0;
    void *ypart = nullptr;      // per-block short vectors [block][n_minor]
    void *ypart_k = nullptr;    // the same for several vectors, [vector][block][n_minor] (made on first use)
    size_t ypart_k_bytes = 0;
    void *vt = nullptr;         // up to VL_MAX input vectors interleaved, for multi-vector segmented passes
    size_t vt_bytes = 0;        // over vectors that stay in global memory (made on first use)
    const int2 *win = nullptr;  // sub-plan: per CTA window of the long vector

    // kernel timers (SPMV_PLAN_PROFILE)
    struct Prof {
        int kernel;
        cudaEvent_t a, b;
    };
    std::atomic<bool> prof_on{false};  // SPMV_PLAN_PROFILE at creation; spmv_profile_enable later
    std::mutex prof_mu;
    std::vector<Prof> prof;
    double prof_ms[7] = {0, 0, 0, 0, 0, 0, 0};
    int64_t prof_n[7] = {0, 0, 0, 0, 0, 0, 0};
};

namespace gbk {

// Internal overrides of a plan made by the library itself.
struct PlanInternal {
    int ctas = 0;             // CTAs of every pass (0: one per SM, at most one per tile)
    int blocks_per_cta = 1;   // blocks of tiles each CTA runs in turn
    bool segdot_only = false; // only single-vector segmented passes will run
};
spmv_status plan_create(spmv_plan_s **out, int64_t m, int64_t n, int64_t nnz, int32_t layout, const int32_t *ptr,
                        const int32_t *idx, const void *vals, int32_t val_dtype, int32_t vec_dtype, cudaStream_t s,
                        uint32_t flags, const spmv_plan_opts *opts, const PlanInternal *pi);
void plan_free(spmv_plan_s *p);
// Build the row-sorted block copy of a finished plan (blocks.cu); leaves the plan unchanged
// when the copy would not pay or its windows do not fit on chip.
spmv_status build_row_blocks(spmv_plan_s *p, int sms, cudaStream_t s);

// Internal entry points on device pointers (no host staging).  `in`/`out`
// hold kb <= plan->batch_width vector pointers (kb == 1 off chip).
spmv_status run_scatter(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s);
spmv_status run_segdot(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s);
// op product on device vectors, any k (split into passes of batch_width)
spmv_status run_op(spmv_plan_s *p, int op, int k, const void *const *in, void *const *out, cudaStream_t s);
size_t plan_footprint(const spmv_plan_s *p);
// Plan-owned copy of idx/vals, permuted within each segment so that one warp instruction of the
// streaming kernels meets distinct shared-memory banks (banks: 32, or 16 for 8-byte vectors).
cudaError_t launch_bank_order(const int32_t *ptr, int n_major, int nnz, const int32_t *idx, const void *vals,
                              int val_bytes, int32_t *oidx, void *ovals, int32_t *slots, int T, int banks,
                              cudaStream_t s);
spmv_status set_error(spmv_status st, const std::string &msg);

// Device buffers of one stable (major, minor) sort of coordinate triples (coo.cu; freed together).
struct CooSort {
    void *tmp = nullptr;   // keys x2, payloads x2, histogram, block sums
    void *own = nullptr;   // sorted minor indices + values (handed to the plan)
    size_t own_bytes = 0;
    ~CooSort();
};
// Stable LSD radix sort of the triples by (major, minor) on `s`: sorted minor indices and values
// in cs.own, sorted major indices in a buffer inside cs.tmp.  Range errors set bits 1 / 4 of err.
spmv_status coo_sort(CooSort &cs, const int32_t *major, const int32_t *minor, const void *vals, int sv, int64_t nnz,
                     int n_major, int n_minor, int grid, int32_t *err, cudaStream_t s, const int32_t **major_sorted,
                     int32_t **minor_sorted, void **vals_sorted);
// ptr[j] = number of entries of the sorted major-index array below j, j = 0..n_major.
cudaError_t launch_coo_ptr(const int32_t *major_sorted, int64_t nnz, int n_major, int32_t *ptr, int grid,
                           cudaStream_t s);

}  // namespace gbk
