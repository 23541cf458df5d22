// Internal declarations shared by the CUDA translation units of libspmv_gb300.
// Not part of the public ABI (include/spmv_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

namespace gbk {

// Kernel modes of the streaming kernel (one staged pass over the nonzeros).
enum Mode : int {
    MODE_SCATTER = 0,  // acc[idx[k]] += val[k] * w[major(k)]   (CSC A x, CSR v^T A)
    MODE_SEGDOT = 1,   // out[j] = sum_{k in segment j} val[k] * w[idx[k]]   (CSC v^T A, CSR A x)
    MODE_DVALUES = 2,  // g[k] = minor[idx[k]] * major[seg(k)]
    MODE_VSEG = 3,     // MODE_SEGDOT for several vectors, one per lane of a lane group
};

constexpr int KB_MAX = 8;        // vectors per pass of the multi-vector kernels (but MODE_VSEG)
constexpr int VL_MAX = 8;        // vectors per pass of MODE_VSEG (lane group width)
constexpr int MAX_WARPS = 24;    // warps per CTA of the single-vector passes (80 registers a thread beyond 16)
constexpr int MAX_WARPS_KB = 16; // warps per CTA of the multi-vector passes
constexpr int WARPS_VSEG = 16;   // warps per CTA of MODE_VSEG (up to 128 registers a thread)
constexpr int WARPS_REGS = 16;   // warps per CTA up to which a kernel may use 128 registers a thread
constexpr int MAX_STAGES = 4;    // slots per warp
constexpr int BAR_BYTES = 1024;  // slot barriers at the start of the staging area

// Per-chunk descriptor produced by the set-up (24 bytes).
struct ChunkDev {
    int32_t nz_begin, nz_end;   // nonzeros [nz_begin, nz_end) (Sec. II rule)
    int32_t e_begin, e_end;     // segments whose end event the chunk owns: [e_begin, e_end)
    int32_t jf;                 // first segment j^f (-1 if empty)
    int32_t flags;              // bit0 needLeft, bit1 needRight
};

// Per-chunk quantities of the set-up (Sec. IV-B), device side.
struct ChunkAux {
    int32_t nz_begin, nz_end, jf, jl, e_begin, e_end, ntiles;
    int32_t needLeft, needRight, leftGroupEnd, rightGroup, leftGroup, procsOnLeft, procsOnRight;
};

struct ZoneDev {
    int32_t first, last, col, pad;  // S_k = chunks [first, last], column j_k
};

// What the streaming kernel reads per execution tile (16 bytes).  Tile t covers
// nonzeros [meta[t].nzb, meta[t+1].nzb) and owns the segment end events
// [meta[t].e_begin, meta[t+1].e_begin); meta[ntiles] is the sentinel {nnz, n_major}.
struct alignas(16) TileMeta {
    int32_t nzb, e_begin;
    int32_t flags;  // bit0 needLeft, bit1 needRight, bit2 an empty segment ends in the tile
    int32_t pad;
};

// Parameters of the streaming kernel.
struct StreamParams {
    const int32_t *idx;
    const void *vals;
    const int32_t *pptr;     // plan-owned padded copy of the pointer array (general path)
    int32_t nnz, n_major, n_minor;
    const TileMeta *meta;    // ntiles + 1 entries
    const uint32_t *masks;   // per tile: mwp words of segment-start bits
    const uint16_t *pfx;     // per tile: mwq entries, the segment starts before word j (j >= mwp: all of them)
    int32_t ntiles, mwp, mwq;
    int32_t slot_bytes, vec_region_bytes, slots, x_cap;  // per-warp slot bytes, slots per warp, window elements
    int32_t tile_cap, off_val, off_mask, off_x, off_hdr;  // slot layout: indices at 0, values, masks, windows, header
    int32_t off_pfx;         // segmented modes: the tile's head-count prefix table in the slot (at off_x)
    int32_t checked;         // 1: indices not validated by the plan, checked (clamped) on every step
    int32_t kb;              // vectors in this pass (<= KB template)
    const void *vin[KB_MAX]; // SCATTER: major vectors; SEGDOT: minor vectors; DVALUES: vin[0] minor, vin[1] major;
                             // VSEG: vin[0] = the minor vectors interleaved [entry][VL]
    void *vout[VL_MAX];      // SEGDOT, VSEG: major outputs; DVALUES: vout[0] = g
    void *part;              // SCATTER: per-CTA partials [cta][kb][n_minor] (on chip) or FP64 accumulator [kb][n_minor]
    void *rec_left, *rec_right;  // SEGDOT carry records [b * nproc + proc]: (hi, lo) pairs of the accumulation type
    int32_t nproc;           // processors (chunks of tiles) of the plan: the record stride
    int32_t chunk_tiles;     // C, tiles per chunk (before the single-tile tail of every block)
    int32_t blocks_per_cta;  // BPC: the tiles form gridDim.x BPC blocks; a CTA runs BPC of them in turn
    const int2 *win;         // SEGDOT over row-sorted blocks: per CTA (first element, length) of its window of
                             // the input vector; the indices are offsets into the window (NULL: whole vector)
    int32_t *err;
};

// Dynamic shared-memory limit of one kernel, raised at most once per device and
// size: the value set so far on each device, read without a lock, raised under it.
constexpr int MAX_DEVICES = 64;
struct SmemLimit {
    std::atomic<int> bytes[MAX_DEVICES];
    std::mutex mu;
    SmemLimit() {
        for (auto &b : bytes) b.store(0, std::memory_order_relaxed);
    }
};
// Make `kern` launchable with `smem` bytes of dynamic shared memory on the current device.
template <typename K>
cudaError_t ensure_smem_limit(K kern, SmemLimit &lim, int smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (lim.bytes[dev].load(std::memory_order_acquire) >= smem) return cudaSuccess;
    std::lock_guard<std::mutex> lk(lim.mu);
    if (lim.bytes[dev].load(std::memory_order_relaxed) >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) lim.bytes[dev].store(smem, std::memory_order_release);
    return e;
}

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
// out_b[i] = sum over parts q of part[q * qstride + b * bstride + i], in FP64, in part order
// (qstride = 0: the layout [part][vector][element]).
cudaError_t launch_combine(bool vec_f64, bool part_f64, const void *part, int nparts, int n_minor, int kb,
                           void *const *out, cudaStream_t s, size_t qstride = 0, size_t bstride = 0);
// out[i * kbt + b] = in[b][i] (zeros for kb <= b < kbt), i < len: vectors interleaved for the
// multi-vector segmented passes (kbt = 2, 4 or 8).
cudaError_t launch_interleave(bool f64, int kbt, int kb, const void *const *in, int64_t len, void *out,
                              cudaStream_t s);
cudaError_t launch_fixup(bool vec_f64, const ZoneDev *zones, int z, const void *rec_left, const void *rec_right,
                         int P, int kb, void *const *out, cudaStream_t s);
// Processors of the streaming launches: the chunks of tiles of every CTA's tile range, in
// order (the kernel's numbering, whatever the warp count).  Fills nzb[0..nproc] (if not
// NULL) with their nonzero boundaries; returns nproc.
int stream_processors(int ntiles, int T, int nnz, int ctas, int C, int32_t *nzb);

// Plan kernels (plan.cu).
cudaError_t launch_validate(const int32_t *ptr, const int32_t *idx, int n_major, int nnz, int n_minor, int32_t *err,
                            cudaStream_t s);
cudaError_t launch_pad_ptr(const int32_t *ptr, int32_t *pptr, int n_major, int nnz, int padded, cudaStream_t s);
// Per chunk: bounds by the Sec. II rule over P chunks (nzb == nullptr) or from nzb[0..P], first/last
// segments, owned end events, and the number of execution tiles of at most tmax nonzeros.
cudaError_t launch_chunks(const int32_t *pptr, int n_major, int nnz, int P, const int32_t *nzb, int tmax, ChunkAux *aux,
                          cudaStream_t s);
// The Sec. IV-B set-up over P chunks (multi-block scans): flags, groups, extents, descriptors,
// zones; counts[0] = z, counts[2] = V (must be zero on entry).  scratch: setup_scratch_bytes(P).
cudaError_t launch_setup(ChunkAux *aux, int P, ChunkDev *chunks, ZoneDev *zones, int32_t *counts, void *scratch,
                         cudaStream_t s);
size_t setup_scratch_bytes(int P);
// Execution tile boundaries tile_nzb[t] = min(t * T, nnz), t = 0..ntiles.
cudaError_t launch_tile_bounds(int ntiles, int T, int nnz, int32_t *tile_nzb, cudaStream_t s);
// Per tile: segment-start masks and the kernel's tile descriptors (needLeft / needRight of
// every tile from its neighbours' first and last segments).
cudaError_t launch_masks(const int32_t *pptr, const ChunkAux *tiles, int ntiles, int nnz, int n_major, int mwp,
                         uint32_t *masks, int mwq, uint16_t *pfx, TileMeta *meta, cudaStream_t s);

}  // namespace gbk
