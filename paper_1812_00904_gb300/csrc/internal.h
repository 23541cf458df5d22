// Internal declarations shared by the CUDA translation units of libspmv_gb300.
// Not part of the public ABI (include/spmv_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbk {

// Kernel modes of the streaming kernel (one staged pass over a chunk's nonzeros).
enum Mode : int {
    MODE_SCATTER = 0,  // acc[idx[k]] += val[k] * w[major(k)]   (CSC A x, CSR v^T A)
    MODE_SEGDOT = 1,   // out[j] = sum_{k in segment j} val[k] * w[idx[k]]   (CSC v^T A, CSR A x)
    MODE_DVALUES = 2,  // g[k] = minor[idx[k]] * major[seg(k)]
};

constexpr int KB_MAX = 8;        // vectors per pass of the multi-vector kernels
constexpr int MAX_WARPS = 16;    // warps (chunks) per CTA
constexpr int MAX_STAGES = 8;

// Per-chunk descriptor read by the streaming kernels (32 bytes).
struct ChunkDev {
    int32_t nz_begin, nz_end;   // nonzeros [nz_begin, nz_end) (Sec. II rule)
    int32_t e_begin, e_end;     // segments whose end event the chunk owns: [e_begin, e_end)
    int32_t jf;                 // first segment j^f (-1 if empty)
    int32_t flags;              // bit0 needLeft, bit1 needRight
    int32_t tile_begin, tile_end;
};

// Per-chunk quantities of the set-up (Sec. IV-B), device side.
struct ChunkAux {
    int32_t nz_begin, nz_end, jf, jl, e_begin, e_end, ntiles;
    int32_t needLeft, needRight, leftGroupEnd, rightGroup, leftGroup, procsOnLeft, procsOnRight;
};

struct ZoneDev {
    int32_t first, last, col, pad;  // S_k = chunks [first, last], column j_k
};

// Parameters of the streaming kernel.
struct StreamParams {
    const int32_t *idx;
    const void *vals;
    const int32_t *pptr;   // plan-owned padded copy of the pointer array
    int32_t nnz, n_major, n_minor, P;
    const ChunkDev *chunks;
    const int4 *tiles;     // per tile: start (k, i), flags (bit0: an empty segment ends in the tile), 0
    const uint32_t *masks; // per tile: mwp words of segment-start bits (plan-time), 16-byte aligned blocks
    int32_t mwp;           // mask words per tile (multiple of 4)
    int32_t stage_bytes, warp_bytes, vec_region_bytes, stages;
    int32_t pptr_len, table_bytes;
    int32_t kb;            // vectors in this pass (<= KB template)
    const void *vin[KB_MAX];   // SCATTER: major vectors; SEGDOT: minor vectors; DVALUES: vin[0] minor, vin[1] major
    void *vout[KB_MAX];        // SEGDOT: major outputs; DVALUES: vout[0] = g
    void *part;            // SCATTER: per-CTA partials [cta][kb][n_minor] (on-chip mode) or FP64 accumulator [kb][n_minor]
    double *rec_left, *rec_right;  // SEGDOT carry records [b * P + c]
    int32_t *err;
};

struct LaunchArgs {
    StreamParams sp;
    int grid, block, smem;
    bool smemv;
    cudaStream_t stream;
};

// Dispatchers implemented in the per-value-type translation units.
cudaError_t launch_stream_f64(int mode, int kb, const LaunchArgs &a);
cudaError_t launch_stream_f32(int mode, int kb, const LaunchArgs &a);
cudaError_t launch_stream_bf16(int mode, int kb, const LaunchArgs &a);
cudaError_t launch_stream_f16(int mode, int kb, const LaunchArgs &a);

// Small kernels (small_kernels.cu).
cudaError_t launch_combine(bool vec_f64, bool part_f64, const void *part, int nparts, int n_minor, int kb,
                           void *const *out, cudaStream_t s);
cudaError_t launch_fixup(bool vec_f64, const ZoneDev *zones, int z, const double *rec_left, const double *rec_right,
                         int P, int kb, void *const *out, cudaStream_t s);

// Plan kernels (plan.cu).
cudaError_t launch_validate(const int32_t *ptr, const int32_t *idx, int n_major, int nnz, int n_minor, int32_t *err,
                            cudaStream_t s);
cudaError_t launch_pad_ptr(const int32_t *ptr, int32_t *pptr, int n_major, int nnz, int padded, cudaStream_t s);
cudaError_t launch_chunks(const int32_t *pptr, int n_major, int nnz, int P, int D, ChunkAux *aux, cudaStream_t s);
cudaError_t launch_setup(ChunkAux *aux, int P, ChunkDev *chunks, ZoneDev *zones, int32_t *counts, cudaStream_t s);
cudaError_t launch_tiles(const int32_t *pptr, int n_major, const ChunkAux *aux, const ChunkDev *chunks, int P, int D,
                         int ntiles, int4 *tiles, cudaStream_t s);
cudaError_t launch_masks(const int32_t *pptr, const ChunkDev *chunks, int P, int ntiles, int mwp, int4 *tiles,
                         uint32_t *masks, cudaStream_t s);

}  // namespace gbk
