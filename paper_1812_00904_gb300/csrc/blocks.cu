// Row-sorted blocks: a second plan-owned copy of the nonzeros for the product
// that accumulates into the short vector (y = A x of a wide CSC matrix, u^T =
// v^T A of a tall CSR one), so that it runs without atomics.
//
// Sec. III step 1 has every processor form A_(i) x_(i), the product of its
// contiguous group of nonzeros with the entries of x it needs, and step 2 adds
// the processors' short vectors.  Here the groups are G "blocks" of whole
// execution tiles (the Sec. II rule over the tiles, G a multiple of the SM
// count), one per CTA of the pass.  Inside a block the nonzeros are re-sorted
// by their short-vector index (row of a wide matrix), so the block's
// contribution to y_i is the dot product of its row-i nonzeros with the
// block's window of x -- the segmented pass of Sec. IV-A over segments
// (block, row), reading x from a shared-memory copy of the block's window; each
// CTA runs G / (SM count) blocks in turn, restaging the window between them.
// The per-block short vectors are then added in FP64 in block order (Sec. III
// step 2).  The copy is laid out as a CSR matrix with G * m rows (segment g * m + i
// = row i of block g) whose column indices are offsets into the block's
// window, and planned like any other matrix with its tiles cut into the G blocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "plan_impl.h"

namespace gbk {
namespace {

// Largest e in [lo, hi] with pptr[e] <= v: the segment holding nonzero v.
__device__ __forceinline__ int seg_of(const int32_t *pptr, int lo, int hi, int64_t v) {
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (pptr[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// First nonzero of block g when nt tiles of T nonzeros are cut into G blocks by the Sec. II rule.
__host__ __device__ __forceinline__ int64_t block_begin(int g, int nt, int G, int T, int64_t nnz) {
    const int q = nt / G, r = nt % G;
    const int64_t t = (int64_t)g * q + (g < r ? g : r);
    return t * T < nnz ? t * T : nnz;
}

// Block holding nonzero k (inverse of block_begin; G <= nt, so every block has a tile).
__device__ __forceinline__ int block_of(int64_t k, int nt, int G, int T) {
    const int q = nt / G, r = nt % G;
    const int64_t t = k / T;
    const int64_t big = (int64_t)r * (q + 1);
    return t < big ? (int)(t / (q + 1)) : (int)(r + (t - big) / q);
}

// For the candidate block counts G_c = (c + 1) * sms: the widest window of any block (the segments
// it spans, from its first one rounded down to a multiple of xa).  One thread per (candidate, block).
__global__ void block_span_kernel(const int32_t *__restrict__ pptr, int n_major, int64_t nnz, int nt, int T, int sms,
                                  int ncand, int xa, int32_t *__restrict__ maxspan) {
    const int64_t total = (int64_t)sms * ncand * (ncand + 1) / 2;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        int64_t rem = x;
        while (rem >= (int64_t)(c + 1) * sms) {
            rem -= (int64_t)(c + 1) * sms;
            ++c;
        }
        const int G = (c + 1) * sms, g = (int)rem;
        if (G > nt) continue;
        const int64_t a = block_begin(g, nt, G, T, nnz), b = block_begin(g + 1, nt, G, T, nnz);
        if (b <= a) continue;
        const int jf = seg_of(pptr, 0, n_major, a) / xa * xa, jl = seg_of(pptr, 0, n_major, b - 1);
        atomicMax(&maxspan[c], jl - jf + 1);
    }
}

// Window (first segment, rounded down to a multiple of xa so that it starts on a 16-byte
// boundary of the vector; number of segments) of every block for the chosen G.
__global__ void block_window_kernel(const int32_t *__restrict__ pptr, int n_major, int64_t nnz, int nt, int T, int G,
                                    int xa, int2 *__restrict__ win) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int64_t a = block_begin(g, nt, G, T, nnz), b = block_begin(g + 1, nt, G, T, nnz);
    if (b <= a) {
        win[g] = make_int2(0, 0);
        return;
    }
    const int jf = seg_of(pptr, 0, n_major, a) / xa * xa, jl = seg_of(pptr, 0, n_major, b - 1);
    win[g] = make_int2(jf, jl - jf + 1);
}

// One warp per major segment j: for each of its nonzeros k, the segment of the copy
// (block * n_minor + minor index) and the column within the block's window.
__global__ void block_keys_kernel(const int32_t *__restrict__ pptr, const int32_t *__restrict__ idx, int n_major,
                                  int n_minor, int nt, int T, int G, const int2 *__restrict__ win,
                                  int32_t *__restrict__ bmaj, int32_t *__restrict__ bmin) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_major; j += nwarps) {
        const int e = pptr[j + 1];
        for (int64_t k = pptr[j] + lane; k < e; k += 32) {
            const int g = block_of(k, nt, G, T);
            bmaj[k] = g * n_minor + idx[k];
            bmin[k] = (int)j - win[g].x;
        }
    }
}

}  // namespace

// Candidate block counts: multiples of the SM count up to this many per SM.
constexpr int BLOCK_CANDIDATES = 16;
// Fewest nonzeros per (block, short-vector entry) for the copy to pay (its segments
// must be long enough for the segmented pass, and the per-block short vectors few).
constexpr int BLOCK_MIN_DENSITY = 8;

spmv_status build_row_blocks(spmv_plan_s *p, int sms, cudaStream_t s) {
    if (p->nnz == 0) return SPMV_OK;
    const int n_minor = p->n_minor;
    const int xa = 16 / p->sx;
    // The copy is tiled like the plan (half tiles, which leave room for wider windows, measured
    // much slower per nonzero).  The widest window of every candidate block count comes from one
    // pass over the block boundaries; the smallest count whose windows fit is taken.
    int G = 0, wmax = 0, T = 0;
    for (int pass = 0; pass < 1; ++pass) {
        const int Tc = p->T;
        if (Tc < 64 || (Tc % 8) != 0) break;
        const int nt = (int)((p->nnz + Tc - 1) / Tc);
        if (nt < sms) continue;
        const int mwp = (int)(((size_t)Tc + 8 + 31) / 32 + 3) / 4 * 4;
        // the window budget: what the segmented pass leaves beside 16 warps of staging slots
        const size_t slot = (size_t)p->S * (((size_t)Tc * 4 + 127) / 128 * 128 +
                                            ((size_t)Tc * p->sv + 127) / 128 * 128 + (size_t)mwp * 4 +
                                            ((size_t)p->mwq * 2 + 15) / 16 * 16 + 160);
        const size_t budget =
            (size_t)p->smem_max > BAR_BYTES + 16 * slot ? (size_t)p->smem_max - BAR_BYTES - 16 * slot : 0;
        const int64_t max_elems = (int64_t)(budget / p->sx);
        if (max_elems < 64) continue;
        int32_t *d_max = nullptr;
        if (cudaMalloc(&d_max, BLOCK_CANDIDATES * 4) != cudaSuccess) return set_error(SPMV_ERR_OOM, "row blocks");
        std::vector<int32_t> mx(BLOCK_CANDIDATES, 0);
        cudaMemsetAsync(d_max, 0, BLOCK_CANDIDATES * 4, s);
        block_span_kernel<<<std::max(1, sms * 4), 256, 0, s>>>(p->pptr, p->n_major, p->nnz, nt, Tc, sms,
                                                               BLOCK_CANDIDATES, xa, d_max);
        cudaError_t ce = cudaMemcpyAsync(mx.data(), d_max, BLOCK_CANDIDATES * 4, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        cudaFree(d_max);
        if (ce != cudaSuccess) return set_error(SPMV_ERR_CUDA, std::string("row blocks: ") + cudaGetErrorString(ce));
        for (int c = 0; c < BLOCK_CANDIDATES; ++c) {
            const int Gc = (c + 1) * sms;
            if (Gc > nt) break;
            if (mx[c] > 0 && mx[c] <= max_elems) {
                if (G == 0 || Gc < G) {
                    G = Gc;
                    wmax = mx[c];
                    T = Tc;
                }
                break;
            }
        }
    }
    if (G == 0) return SPMV_OK;  // no block count gives windows that fit: keep the atomic pass
    const int nt = (int)((p->nnz + T - 1) / T);
    if ((int64_t)G * n_minor >= (1ll << 31) - 64 || p->nnz < (int64_t)BLOCK_MIN_DENSITY * G * n_minor) return SPMV_OK;

    // ---- windows, per-nonzero segment and window column, stable sort into the copy
    const size_t nseg = (size_t)G * n_minor;
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_win = 0, o_bptr = up((size_t)G * 8), o_ypart = o_bptr + up((nseg + 1) * 4);
    const size_t bws_bytes = o_ypart + up(nseg * p->sx);
    if (cudaMalloc(&p->bws, bws_bytes) != cudaSuccess) return set_error(SPMV_ERR_OOM, "row blocks");
    p->bws_bytes = bws_bytes;
    int2 *win = reinterpret_cast<int2 *>(static_cast<char *>(p->bws) + o_win);
    int32_t *bptr = reinterpret_cast<int32_t *>(static_cast<char *>(p->bws) + o_bptr);
    p->ypart = static_cast<char *>(p->bws) + o_ypart;
    int32_t *keys = nullptr;  // bmaj then bmin, nnz each
    if (cudaMalloc(&keys, (size_t)p->nnz * 8) != cudaSuccess) return set_error(SPMV_ERR_OOM, "row blocks");
    int32_t *bmaj = keys, *bmin = keys + p->nnz;
    block_window_kernel<<<(G + 255) / 256, 256, 0, s>>>(p->pptr, p->n_major, p->nnz, nt, T, G, xa, win);
    block_keys_kernel<<<std::max(1, sms * 16), 256, 0, s>>>(p->pptr, p->idx, p->n_major, n_minor, nt, T, G, win, bmaj,
                                                            bmin);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
        cudaFree(keys);
        return set_error(SPMV_ERR_CUDA, std::string("row blocks: ") + cudaGetErrorString(ce));
    }
    CooSort cs;
    const int32_t *smaj = nullptr;
    int32_t *sidx = nullptr;
    void *svals = nullptr;
    spmv_status st = coo_sort(cs, bmaj, bmin, p->vals, p->sv, p->nnz, (int)nseg, wmax, sms * 8, p->err, s, &smaj,
                              &sidx, &svals);
    if (st == SPMV_OK) {
        ce = launch_coo_ptr(smaj, p->nnz, (int)nseg, bptr, sms * 8, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) st = set_error(SPMV_ERR_CUDA, std::string("row blocks: ") + cudaGetErrorString(ce));
    }
    cudaFree(keys);
    if (st != SPMV_OK) return st;
    int32_t e = 0;
    cudaMemcpy(&e, p->err, 4, cudaMemcpyDeviceToHost);
    if (e) return set_error(SPMV_ERR_DEVICE, "row blocks: index out of range while sorting");

    // ---- the copy as a CSR matrix of G * m rows over windows of wmax columns; one CTA per SM runs
    // G / sms blocks in turn, restaging the window between them
    PlanInternal pi;
    pi.ctas = sms;
    pi.blocks_per_cta = G / sms;
    pi.segdot_only = true;
    spmv_plan_opts o{};
    o.tile_items = T;
    o.stages = p->S;
    o.warps_per_cta = p->W;
    o.chunk_tiles = p->chunk_tiles;
    spmv_plan_s *q = nullptr;
    st = plan_create(&q, (int64_t)nseg, wmax, p->nnz, SPMV_CSR_TALL, bptr, sidx, svals, p->val_t, p->vec_t, s,
                     p->flags & SPMV_PLAN_BANK_ORDER, &o, &pi);
    if (st != SPMV_OK) return st;
    if (!q->onchip || q->ctas * q->bpc != G) {  // the windows must sit in shared memory, block by block
        plan_free(q);
        return SPMV_OK;
    }
    q->win = win;
    if (!q->owned_nz) {  // the sub-plan multiplies the sorted copy itself: keep it
        p->bown = cs.own;
        p->bown_bytes = cs.own_bytes;
        cs.own = nullptr;
    }
    p->tplan = q;
    p->blocks = G;
    p->block_window = wmax;
    return SPMV_OK;
}

}  // namespace gbk
