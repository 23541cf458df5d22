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
    // Overlap zones among the processors of the segmented passes (the warps that hold
    // tiles, Sec. II groups of whole tiles), one table per vector-slot template of the
    // passes (index log2 kbt: 1, 2, 4, 8 vectors), since the warp count can differ.
    struct ProcZones {
        int W = 0;      // warps per CTA of those passes
        int nproc = 0;  // processors, the stride of the carry records
        int z = 0;      // overlap zones among them
        gbk::ZoneDev *zones = nullptr;
    };
    ProcZones pz[4];
    int max_nproc = 0;
    void *rec_left = nullptr, *rec_right = nullptr;  // (hi, lo) pairs of the accumulation type
    void *part = nullptr;
    int z = 0, vmax = 0;
    double setup_ms = 0.0;
    int64_t max_chunk = 0, min_chunk = 0;

    // staging buffers for host-pointer calls (allocated on first use)
    std::mutex host_mu;
    void *hin = nullptr, *hout = nullptr, *hg = nullptr;
    void *ynorm = nullptr;  // A x of spmv_normal when the caller passes no buffer
    void *owned_ptr = nullptr;  // pointer array built by spmv_plan_coo (the other arrays stay borrowed)
    void *owned_nz = nullptr;   // plan-owned idx and vals: bank order, or triples sorted by spmv_plan_coo
    size_t owned_bytes = 0;

    // kernel timers (SPMV_PLAN_PROFILE)
    struct Prof {
        int kernel;
        cudaEvent_t a, b;
    };
    std::atomic<bool> prof_on{false};  // SPMV_PLAN_PROFILE at creation; spmv_profile_enable later
    std::mutex prof_mu;
    std::vector<Prof> prof;
    double prof_ms[5] = {0, 0, 0, 0, 0};
    int64_t prof_n[5] = {0, 0, 0, 0, 0};
};

namespace gbk {

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

}  // namespace gbk
