// Plan kernels: structural checks, the nonzero partition of Sec. II, the
// overlap-zone set-up of Sec. IV-B (needLeft, needRight, leftGroupEnd,
// rightGroup, leftGroup, procsOnLeft, procsOnRight), and the merge-order tiles
// each chunk streams through shared memory.
#include <algorithm>

#include "internal.h"

namespace gbk {

// Error bits of the structural check (plan-time; the host maps them to messages).
// 1: ptr[0] != 0, 2: ptr decreasing or outside [0, nnz], 4: ptr[last] != nnz, 8: index out of range.
__global__ void validate_kernel(const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, int n_major,
                                int nnz, int n_minor, int32_t *err) {
    int bits = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j <= n_major; j += stride) {
        const int pj = ptr[j];
        if (j == 0 && pj != 0) bits |= 1;
        if (pj < 0 || pj > nnz) bits |= 2;
        if (j < n_major && ptr[j + 1] < pj) bits |= 2;
        if (j == n_major && pj != nnz) bits |= 4;
    }
    for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int r = idx[k];
        if (r < 0 || r >= n_minor) bits |= 8;
    }
    if (bits) atomicOr(err, bits);
}

cudaError_t launch_validate(const int32_t *ptr, const int32_t *idx, int n_major, int nnz, int n_minor, int32_t *err,
                            cudaStream_t s) {
    validate_kernel<<<1024, 256, 0, s>>>(ptr, idx, n_major, nnz, n_minor, err);
    return cudaGetLastError();
}

// Plan-owned copy of the pointer array, padded with nnz to `padded` entries
// (so 16-byte staged windows never read past its end).
__global__ void pad_ptr_kernel(const int32_t *__restrict__ ptr, int32_t *__restrict__ pptr, int n_major, int nnz,
                               int padded) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < padded; j += stride)
        pptr[j] = j <= n_major ? ptr[j] : nnz;
}

cudaError_t launch_pad_ptr(const int32_t *ptr, int32_t *pptr, int n_major, int nnz, int padded, cudaStream_t s) {
    pad_ptr_kernel<<<1024, 256, 0, s>>>(ptr, pptr, n_major, nnz, padded);
    return cudaGetLastError();
}

// Number of segments j in [lo, hi) with pptr[j+1] <= v, searched in [lo, hi]:
// the largest e in [lo, hi] with pptr[e] <= v (given pptr[lo] <= v).
__device__ __forceinline__ int ends_upto(const int32_t *pptr, int lo, int hi, long v) {
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (pptr[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One thread per chunk c: its nonzeros (by the Sec. II rule, or from an explicit
// boundary array), its first and last segment (j^f, j^l), the segment end
// events it owns, and how many execution tiles of at most tmax nonzeros it is
// cut into.
__global__ void chunks_kernel(const int32_t *__restrict__ pptr, int n_major, int nnz, int P,
                              const int32_t *__restrict__ nzb_arr, int tmax, ChunkAux *__restrict__ aux) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P) return;
    int nzb, nze;
    if (nzb_arr) {
        nzb = nzb_arr[c];
        nze = nzb_arr[c + 1];
    } else {
        const int q = nnz / P, r = nnz % P;
        nzb = c * q + min(c, r);
        nze = nzb + q + (c < r ? 1 : 0);
    }
    ChunkAux a;
    a.nz_begin = nzb;
    a.nz_end = nze;
    // end events owned: segments whose end is ordered no later than the chunk's last nonzero
    a.e_end = ends_upto(pptr, 0, n_major, nze);
    a.e_begin = (c == 0) ? 0 : ends_upto(pptr, 0, n_major, nzb);
    if (nze > nzb) {
        a.jf = ends_upto(pptr, 0, n_major, nzb);      // segment holding nonzero nzb
        a.jl = ends_upto(pptr, 0, n_major, nze - 1);  // segment holding nonzero nze-1
    } else {
        a.jf = -1;
        a.jl = -1;
    }
    a.ntiles = (nze - nzb + tmax - 1) / tmax;
    a.needLeft = a.needRight = a.leftGroupEnd = a.rightGroup = a.leftGroup = a.procsOnLeft = a.procsOnRight = 0;
    aux[c] = a;
}

cudaError_t launch_chunks(const int32_t *pptr, int n_major, int nnz, int P, const int32_t *nzb, int tmax, ChunkAux *aux,
                          cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    chunks_kernel<<<(P + 255) / 256, 256, 0, s>>>(pptr, n_major, nnz, P, nzb, tmax, aux);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sec. IV-B over P chunks on the whole GPU.  Chunk c's flags depend only on its
// neighbours; the three scans (the additive scan of leftGroupEnd, the forward
// segmented scan of (needLeft, leftGroup) and the backward one of (needRight,
// rightGroup)) each run in three steps: every block of SU_ITEMS chunks scans its
// own chunks and leaves an aggregate, one block scans the aggregates, and every
// block rescans its chunks from its prefix.

struct SegPair {  // (s, k) of the segmented operator o; `has` = false is the empty prefix
    int s, k, has;
};

__device__ __forceinline__ SegPair seg_op(SegPair a, SegPair b) {
    // (s,k) o (t,l) = (s+t, l) if k == l else (t, l)  (Sec. IV-B)
    if (!a.has) return b;
    if (!b.has) return a;
    SegPair r;
    r.s = (a.k == b.k) ? a.s + b.s : b.s;
    r.k = b.k;
    r.has = 1;
    return r;
}

constexpr int SU_THREADS = 256, SU_IPT = 8, SU_ITEMS = SU_THREADS * SU_IPT;

struct AddOp {
    __device__ __forceinline__ int operator()(int a, int b) const { return a + b; }
};
struct SegOp {
    __device__ __forceinline__ SegPair operator()(SegPair a, SegPair b) const { return seg_op(a, b); }
};

// Exclusive scan over the threads of a block (thread order), `id` the empty prefix; returns the
// block total through *total.
template <typename T, typename Op>
__device__ T block_exclusive(T v, T id, Op op, T *total) {
    __shared__ T sh[SU_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o;
        if constexpr (sizeof(T) == sizeof(int)) {
            o = __shfl_up_sync(0xffffffffu, inc, d);
        } else {
            o.s = __shfl_up_sync(0xffffffffu, inc.s, d);
            o.k = __shfl_up_sync(0xffffffffu, inc.k, d);
            o.has = __shfl_up_sync(0xffffffffu, inc.has, d);
        }
        if (lane >= d) inc = op(o, inc);
    }
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    T wpre = id;
    for (int q = 0; q < w; ++q) wpre = op(wpre, sh[q]);
    T all = id;
    for (int q = 0; q < SU_THREADS / 32; ++q) all = op(all, sh[q]);
    T ex;
    if constexpr (sizeof(T) == sizeof(int)) {
        ex = __shfl_up_sync(0xffffffffu, inc, 1);
    } else {
        ex.s = __shfl_up_sync(0xffffffffu, inc.s, 1);
        ex.k = __shfl_up_sync(0xffffffffu, inc.k, 1);
        ex.has = __shfl_up_sync(0xffffffffu, inc.has, 1);
    }
    if (lane == 0) ex = id;
    __syncthreads();
    *total = all;
    return op(wpre, ex);
}

// 1. "Determine overlap zones" and "determine ranks of overlap groups" (the flags), and every
// block's sum of leftGroupEnd.
__global__ void __launch_bounds__(SU_THREADS) setup_flags_kernel(ChunkAux *__restrict__ aux, int P,
                                                                 int *__restrict__ blk_sum) {
    const int c0 = blockIdx.x * SU_ITEMS + threadIdx.x * SU_IPT;
    int sum = 0;
    for (int i = 0; i < SU_IPT; ++i) {
        const int c = c0 + i;
        if (c >= P) break;
        const ChunkAux a = aux[c];
        const bool ne = a.nz_end > a.nz_begin;
        const int nl = (c > 0 && ne && aux[c - 1].nz_end > aux[c - 1].nz_begin && a.jf == aux[c - 1].jl) ? 1 : 0;
        const int nr = (c < P - 1 && ne && aux[c + 1].nz_end > aux[c + 1].nz_begin && a.jl == aux[c + 1].jf) ? 1 : 0;
        const int lge = (nl == 1 && (nr == 0 || a.jf != a.jl)) ? 1 : 0;
        aux[c].needLeft = nl;
        aux[c].needRight = nr;
        aux[c].leftGroupEnd = lge;
        sum += lge;
    }
    int total;
    block_exclusive(sum, 0, AddOp(), &total);
    if (threadIdx.x == 0) blk_sum[blockIdx.x] = total;
}

// 2, 4. One block: exclusive scans of the block aggregates (additive; or segmented forward
// and backward), in place.
__global__ void __launch_bounds__(SU_THREADS) setup_scan_add_kernel(int *__restrict__ blk, int nb, int32_t *counts) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += SU_THREADS) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? blk[i] : 0;
        int total;
        const int ex = block_exclusive(v, 0, AddOp(), &total);
        if (i < nb) blk[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[0] = carry;  // z = number of overlap zones
}

__global__ void __launch_bounds__(SU_THREADS) setup_scan_seg_kernel(SegPair *__restrict__ fwd, SegPair *__restrict__ bwd,
                                                                    int nb) {
    __shared__ SegPair carry;
    const SegPair id{0, 0, 0};
    // forward, in block order
    if (threadIdx.x == 0) carry = id;
    __syncthreads();
    for (int base = 0; base < nb; base += SU_THREADS) {
        const int i = base + threadIdx.x;
        const SegPair v = i < nb ? fwd[i] : id;
        SegPair total;
        const SegPair ex = block_exclusive(v, id, SegOp(), &total);
        if (i < nb) fwd[i] = seg_op(carry, ex);
        __syncthreads();
        if (threadIdx.x == 0) carry = seg_op(carry, total);
        __syncthreads();
    }
    // backward: element i of the reversed order is block nb - 1 - i
    if (threadIdx.x == 0) carry = id;
    __syncthreads();
    for (int base = 0; base < nb; base += SU_THREADS) {
        const int i = base + threadIdx.x;
        const SegPair v = i < nb ? bwd[nb - 1 - i] : id;
        SegPair total;
        const SegPair ex = block_exclusive(v, id, SegOp(), &total);
        if (i < nb) bwd[nb - 1 - i] = seg_op(carry, ex);
        __syncthreads();
        if (threadIdx.x == 0) carry = seg_op(carry, total);
        __syncthreads();
    }
}

// 3. rightGroup (inclusive scan of leftGroupEnd from the block's prefix) and leftGroup; every
// block's aggregates of (needLeft, leftGroup) in order and of (needRight, rightGroup) in reverse order.
__global__ void __launch_bounds__(SU_THREADS) setup_groups_kernel(ChunkAux *__restrict__ aux, int P,
                                                                  const int *__restrict__ blk_pre,
                                                                  SegPair *__restrict__ fwd, SegPair *__restrict__ bwd) {
    const int c0 = blockIdx.x * SU_ITEMS + threadIdx.x * SU_IPT;
    int sum = 0;
    for (int i = 0; i < SU_IPT && c0 + i < P; ++i) sum += aux[c0 + i].leftGroupEnd;
    int total;
    int run = blk_pre[blockIdx.x] + block_exclusive(sum, 0, AddOp(), &total);
    const SegPair id{0, 0, 0};
    SegPair f = id;
    for (int i = 0; i < SU_IPT && c0 + i < P; ++i) {
        const int c = c0 + i;
        const int lge = aux[c].leftGroupEnd;
        run += lge;
        aux[c].rightGroup = run;
        aux[c].leftGroup = run - lge;
        f = seg_op(f, SegPair{aux[c].needLeft, run - lge, 1});
    }
    SegPair ft;
    block_exclusive(f, id, SegOp(), &ft);
    // backward aggregate: this block's chunks from the last to the first, thread t taking the
    // chunks thread SU_THREADS - 1 - t wrote above
    __syncthreads();
    SegPair b = id;
    const int c1 = blockIdx.x * SU_ITEMS + (SU_THREADS - 1 - threadIdx.x) * SU_IPT;
    for (int i = SU_IPT - 1; i >= 0; --i) {
        const int c = c1 + i;
        if (c < P) b = seg_op(b, SegPair{aux[c].needRight, aux[c].rightGroup, 1});
    }
    SegPair bt;
    block_exclusive(b, id, SegOp(), &bt);
    if (threadIdx.x == 0) {
        fwd[blockIdx.x] = ft;
        bwd[blockIdx.x] = bt;
    }
}

// 5. procsOnLeft / procsOnRight from the blocks' prefixes, the descriptors, the zone list
// (the chunk closing a left group names zone leftGroup) and V = max |S_k|.
__global__ void __launch_bounds__(SU_THREADS) setup_extents_kernel(ChunkAux *__restrict__ aux, int P,
                                                                   const SegPair *__restrict__ fwd,
                                                                   const SegPair *__restrict__ bwd,
                                                                   ChunkDev *__restrict__ chunks,
                                                                   ZoneDev *__restrict__ zones, int32_t *counts) {
    const SegPair id{0, 0, 0};
    const int c0 = blockIdx.x * SU_ITEMS + threadIdx.x * SU_IPT;
    // forward: procsOnLeft
    SegPair f = id;
    for (int i = 0; i < SU_IPT && c0 + i < P; ++i) f = seg_op(f, SegPair{aux[c0 + i].needLeft, aux[c0 + i].leftGroup, 1});
    SegPair tot;
    SegPair run = seg_op(fwd[blockIdx.x], block_exclusive(f, id, SegOp(), &tot));
    for (int i = 0; i < SU_IPT && c0 + i < P; ++i) {
        const int c = c0 + i;
        run = seg_op(run, SegPair{aux[c].needLeft, aux[c].leftGroup, 1});
        aux[c].procsOnLeft = run.s;
    }
    // backward: procsOnRight (threads and chunks in reverse order)
    const int c1 = blockIdx.x * SU_ITEMS + (SU_THREADS - 1 - threadIdx.x) * SU_IPT;
    SegPair b = id;
    for (int i = SU_IPT - 1; i >= 0; --i)
        if (c1 + i < P) b = seg_op(b, SegPair{aux[c1 + i].needRight, aux[c1 + i].rightGroup, 1});
    run = seg_op(bwd[blockIdx.x], block_exclusive(b, id, SegOp(), &tot));
    for (int i = SU_IPT - 1; i >= 0; --i) {
        const int c = c1 + i;
        if (c >= P) continue;
        run = seg_op(run, SegPair{aux[c].needRight, aux[c].rightGroup, 1});
        aux[c].procsOnRight = run.s;
    }
    __syncthreads();
    int vmax = 0;
    for (int i = 0; i < SU_IPT && c0 + i < P; ++i) {
        const int c = c0 + i;
        const ChunkAux a = aux[c];
        ChunkDev d;
        d.nz_begin = a.nz_begin;
        d.nz_end = a.nz_end;
        d.e_begin = a.e_begin;
        d.e_end = a.e_end;
        d.jf = a.jf;
        d.flags = (a.needLeft ? 1 : 0) | (a.needRight ? 2 : 0);
        chunks[c] = d;
        if (a.leftGroupEnd) {
            ZoneDev zd;
            zd.first = c - a.procsOnLeft;
            zd.last = c;
            zd.col = a.jf;
            zd.pad = 0;
            zones[a.leftGroup] = zd;
            vmax = max(vmax, a.procsOnLeft + 1);
        }
    }
    if (vmax) atomicMax(&counts[2], vmax);  // V = max |S_k|
}

cudaError_t launch_setup(ChunkAux *aux, int P, ChunkDev *chunks, ZoneDev *zones, int32_t *counts, void *scratch,
                         cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    const int nb = (P + SU_ITEMS - 1) / SU_ITEMS;
    int *blk = static_cast<int *>(scratch);
    SegPair *fwd = reinterpret_cast<SegPair *>(blk + ((nb + 3) & ~3));
    SegPair *bwd = fwd + nb;
    setup_flags_kernel<<<nb, SU_THREADS, 0, s>>>(aux, P, blk);
    setup_scan_add_kernel<<<1, SU_THREADS, 0, s>>>(blk, nb, counts);
    setup_groups_kernel<<<nb, SU_THREADS, 0, s>>>(aux, P, blk, fwd, bwd);
    setup_scan_seg_kernel<<<1, SU_THREADS, 0, s>>>(fwd, bwd, nb);
    setup_extents_kernel<<<nb, SU_THREADS, 0, s>>>(aux, P, fwd, bwd, chunks, zones, counts);
    return cudaGetLastError();
}

size_t setup_scratch_bytes(int P) {
    const int nb = (P + SU_ITEMS - 1) / SU_ITEMS;
    return (size_t)((nb + 3) & ~3) * sizeof(int) + 2 * (size_t)nb * sizeof(SegPair) + 64;
}

// Execution tile boundaries: tile t covers nonzeros [t*T, min((t+1)*T, nnz)), so
// every tile starts on a multiple of 8 and fills whole steps of the kernels.
__global__ void tile_bounds_kernel(int ntiles, int T, int nnz, int32_t *__restrict__ tile_nzb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= ntiles) tile_nzb[t] = (int)min((long)t * T, (long)nnz);
}

cudaError_t launch_tile_bounds(int ntiles, int T, int nnz, int32_t *tile_nzb, cudaStream_t s) {
    tile_bounds_kernel<<<(ntiles + 1 + 255) / 256, 256, 0, s>>>(ntiles, T, nnz, tile_nzb);
    return cudaGetLastError();
}

// One warp per tile: the segment-start bits of the tile (bit pos set when a
// segment j in (i0, i1] starts at nonzero kb0 + pos, pos < nze - kb0, kb0 =
// nzb rounded down to 8) and the tile descriptor read by the streaming kernel.
// Flags: needLeft / needRight of the tile, from its neighbours' last and first
// segments (the "determine overlap zones" step of Sec. IV-B; tiles are never
// empty); bit 2 marks a tile in which an empty segment ends (then several
// segments can start at one position and the kernels take their general path).
__global__ void masks_kernel(const int32_t *__restrict__ pptr, const ChunkAux *__restrict__ tiles, int ntiles, int nnz,
                             int n_major, int mwp, uint32_t *__restrict__ masks, int mwq, uint16_t *__restrict__ pfx,
                             TileMeta *__restrict__ meta) {
    __shared__ uint32_t sm[8][32];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int t = blockIdx.x * 8 + wib;
    if (t >= ntiles) return;
    const ChunkAux d = tiles[t];
    const int kb0 = d.nz_begin & ~7;
    const int rel_hi = d.nz_end - kb0;
    sm[wib][lane] = 0u;
    __syncwarp();
    bool dup = false;
    for (int j = d.e_begin + 1 + lane; j <= d.e_end; j += 32) {
        const int pj = pptr[j];
        const int pos = pj - kb0;
        if (pos >= 0 && pos < rel_hi && pos < 32 * mwp) atomicOr(&sm[wib][pos >> 5], 1u << (pos & 31));
        if (j < d.e_end && pptr[j + 1] == pj) dup = true;
    }
    dup = __any_sync(0xffffffffu, dup);
    __syncwarp();
    if (lane < mwp) masks[(size_t)t * mwp + lane] = sm[wib][lane];
    // segment starts before each word (exclusive prefix over the tile's words; from word mwp on,
    // all of the tile's), for the segmented passes
    {
        const int c = lane < mwp ? __popc(sm[wib][lane]) : 0;
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int j = lane; j < mwq; j += 32)  // (entry j < 32 is lane j's own)
            pfx[(size_t)t * mwq + j] = static_cast<uint16_t>(j < 32 ? incl - c : total);
    }
    if (lane == 0) {
        TileMeta m;
        m.nzb = d.nz_begin;
        m.e_begin = d.e_begin;
        const bool need_left = t > 0 && tiles[t - 1].jl == d.jf;
        const bool need_right = t + 1 < ntiles && tiles[t + 1].jf == d.jl;
        m.flags = (need_left ? 1 : 0) | (need_right ? 2 : 0) | (dup ? 4 : 0);
        m.pad = 0;
        meta[t] = m;
        if (t == ntiles - 1) {
            TileMeta e;
            e.nzb = nnz;
            e.e_begin = n_major;
            e.flags = 0;
            e.pad = 0;
            meta[ntiles] = e;
        }
    }
}

cudaError_t launch_masks(const int32_t *pptr, const ChunkAux *tiles, int ntiles, int nnz, int n_major, int mwp,
                         uint32_t *masks, int mwq, uint16_t *pfx, TileMeta *meta, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    masks_kernel<<<(ntiles + 7) / 8, 256, 0, s>>>(pptr, tiles, ntiles, nnz, n_major, mwp, masks, mwq, pfx, meta);
    return cudaGetLastError();
}

// The processors of the streaming launches, in the kernel's order (the same for every warp
// count): CTA g takes tiles [ta, ta + nct) by the Sec. II rule over the grid and cuts them
// into nb chunks of C tiles followed by nct - nb C single-tile chunks, where the single
// tiles number at least MAX_WARPS (C + 1) (or all nct).
// nzb[q] = first nonzero of chunk q; nzb[nproc] = nnz.
int stream_processors(int ntiles, int T, int nnz, int ctas, int C, int32_t *nzb) {
    if (ctas < 1 || C < 1) return 0;
    const int tq = ntiles / ctas, tr = ntiles % ctas;
    int np = 0;
    auto put = [&](int tile) {
        if (nzb) nzb[np] = (int)((int64_t)tile * T < nnz ? (int64_t)tile * T : nnz);
        ++np;
    };
    for (int g = 0; g < ctas; ++g) {
        const int ta = g * tq + (g < tr ? g : tr);
        const int nct = tq + (g < tr ? 1 : 0);
        const int tail_min = MAX_WARPS * C + MAX_WARPS;
        const int nb = (nct - (nct < tail_min ? nct : tail_min)) / C;
        for (int j = 0; j < nb; ++j) put(ta + j * C);
        for (int t = ta + nb * C; t < ta + nct; ++t) put(t);
    }
    if (nzb) nzb[np] = nnz;
    return np;
}

// Plan-owned copy of the nonzeros, permuted within every major segment (a column of a
// CSC matrix, a row of a CSR one), so that the minor indices one warp instruction of the
// streaming kernels reads or updates in shared memory fall into distinct banks.  The
// streaming kernels touch tile positions r (r = nonzero position mod T) in these patterns:
// the scatter pass 32 consecutive ones (r = 32a + b, b = 0..31); the segmented pass one of
// 8 positions per lane, 8l + (e ^ 4((l >> 2) & 1)); the multi-vector segmented pass, whose
// lane groups read the VL consecutive words of one index each (VL = 8: 4 groups at positions
// 32a + 8c + e, c = 0..3, so that the index mod 4 picks the group's banks; VL = 4: 8 groups
// at 64a + 8c + e, c = 0..7, index mod 8).  With 4-byte words (32 banks) position
// r = 256 t + 32a + 8c + e asks for bank (4a + c + 4e) mod 32, one-to-one over the lanes
// of the first two patterns and over the groups of the third; with 8-byte words (16 banks)
// for ((r & 31) + ((r >> 5) & 7)) mod 16, one-to-one over each half of the lanes of the
// first two.
//
// One warp per segment: a position asking bank b is served by a nonzero of bank b when it is
// among the first cnt[b] positions of the segment asking b (cnt[b]: the segment's nonzeros of
// bank b), which serves as many positions as the pools allow; the positions left over take, in
// order, the nonzeros left over, dealt round the banks (the first left-over nonzero of every
// bank that has one, in bank order, then the second, ...), so that neighbouring left-over
// positions differ in bank.  Within a bank the stored order is kept.  The warp passes over the
// segment in chunks of 32 (lane = position or nonzero): the counts; the served positions'
// lists (per bank, in order) and the overflow list, in slots[s ..); then every nonzero to its
// position.  Every access stays in the segment's clamped range [s, e), so a malformed ptr (an
// unvalidated plan) stays in bounds.
__device__ __forceinline__ int bank_asked(int r, int nbm) {
    return nbm == 31 ? (4 * ((r >> 5) & 7) + ((r >> 3) & 3) + 4 * (r & 7)) & 31 : ((r & 31) + ((r >> 5) & 7)) & nbm;
}

constexpr int BO_WARPS = 8;
constexpr unsigned FULL = 0xffffffffu;

// Segment [s, e) (at least 2 nonzeros) by the whole warp; run: this warp's 32 shared counters.
template <typename W>
__device__ void bank_order_segment(int s, int e, const int32_t *__restrict__ idx, const W *__restrict__ vals,
                                int32_t *__restrict__ oidx, W *__restrict__ ovals, int32_t *__restrict__ slots, int T,
                                int nbm, int *run) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int len = e - s;
    const int r0 = s % T;
    // ---- per-bank counts: nonzeros (cnt) and positions asking (ask); lane b holds bank b's
    run[lane] = 0;
    __syncwarp();
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        const int b = q < len ? (idx[s + q] & nbm) : 32 + lane;  // past the end: a bank of its own
        const unsigned peers = __match_any_sync(FULL, b);
        if (q < len && (peers & lt) == 0u) run[b] += __popc(peers);
        __syncwarp();
    }
    const int cnt = run[lane];
    __syncwarp();
    run[lane] = 0;
    __syncwarp();
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        const int b = q < len ? bank_asked((r0 + q) % T, nbm) : 32 + lane;
        const unsigned peers = __match_any_sync(FULL, b);
        if (q < len && (peers & lt) == 0u) run[b] += __popc(peers);
        __syncwarp();
    }
    const int ask = run[lane];
    // served per bank and where its served positions start
    const int served = min(cnt, ask), left = cnt - served;
    int off = served;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, off, d);
        if (lane >= d) off += o;
    }
    const int total_served = __shfl_sync(FULL, off, 31);
    off -= served;  // exclusive
    // ---- positions: served ones into their bank's list, the others into the overflow list
    __syncwarp();
    run[lane] = 0;
    __syncwarp();
    int ovf = 0;
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        const bool in = q < len;
        const int b = in ? bank_asked((r0 + q) % T, nbm) : 32 + lane;
        const unsigned peers = __match_any_sync(FULL, b);
        const int bb = in ? b : 0;
        const int rank = run[bb] + __popc(peers & lt);
        const int cb = __shfl_sync(FULL, cnt, bb);  // (every lane takes part in the shuffles)
        const int ob = __shfl_sync(FULL, off, bb);
        const bool srv = in && rank < cb;
        const unsigned om = __ballot_sync(FULL, in && !srv);
        if (srv) {
            slots[s + ob + rank] = s + q;
        } else if (in) {
            const int t = total_served + ovf + __popc(om & lt);
            if (t < len) slots[s + t] = s + q;
        }
        __syncwarp();
        if (in && (peers & lt) == 0u) run[b] += __popc(peers);
        ovf += __popc(om);
        __syncwarp();
    }
    // ---- every nonzero to its position
    run[lane] = 0;
    __syncwarp();
    for (int base = 0; base < len; base += 32) {
        const int q = base + lane;
        const bool in = q < len;
        const int32_t ix = in ? idx[s + q] : 0;
        const int b = in ? (ix & nbm) : 32 + lane;
        const unsigned peers = __match_any_sync(FULL, b);
        const int bb = in ? b : 0;
        const int rank = run[bb] + __popc(peers & lt);
        const int sv = __shfl_sync(FULL, served, bb);
        const int o = __shfl_sync(FULL, off, bb);
        const bool lo = in && rank >= sv;  // a left-over nonzero, number jj of its bank
        const int jj = rank - sv;
        int k = o + rank;
        if (__any_sync(FULL, lo)) {
            // its place in the round of the banks: every bank's first min(left, jj) left-overs,
            // then those of the banks before it with more than jj (at most one left-over per
            // bank: the banks before it that have one)
            int before;
            if (__ballot_sync(FULL, left > 1) == 0u) {
                before = __popc(__ballot_sync(FULL, left > 0) & ((1u << bb) - 1u));
            } else {
                before = 0;
                for (int b2 = 0; b2 <= nbm; ++b2) {
                    const int l2 = __shfl_sync(FULL, left, b2);
                    before += min(l2, max(jj, 0)) + ((b2 < bb && l2 > jj) ? 1 : 0);
                }
            }
            if (lo) k = total_served + before;
        }
        if (in) {
            const int dst = (k >= 0 && k < len) ? slots[s + k] : -1;
            if (dst >= s && dst < e) {
                oidx[dst] = ix;
                ovals[dst] = vals[s + q];
            }
        }
        __syncwarp();
        if (in && (peers & lt) == 0u) run[b] += __popc(peers);
        __syncwarp();
    }
    __syncwarp();
}

template <typename W>
__global__ void __launch_bounds__(BO_WARPS * 32) bank_order_kernel(const int32_t *__restrict__ ptr, int n_major,
                                                                   int nnz, const int32_t *__restrict__ idx,
                                                                   const W *__restrict__ vals,
                                                                   int32_t *__restrict__ oidx, W *__restrict__ ovals,
                                                                   int32_t *__restrict__ slots, int T, int nbm) {
    __shared__ int sh_run[BO_WARPS][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long nw = (long)gridDim.x * BO_WARPS;
    for (long c = (long)blockIdx.x * BO_WARPS + wib; c < n_major; c += nw) {
        const int s = min(max(ptr[c], 0), nnz);
        const int e = min(max(ptr[c + 1], s), nnz);
        if (e - s == 1) {
            if (lane == 0) {
                oidx[s] = idx[s];
                ovals[s] = vals[s];
            }
        } else if (e - s > 1) {
            bank_order_segment(s, e, idx, vals, oidx, ovals, slots, T, nbm, sh_run[wib]);
        }
    }
}

cudaError_t launch_bank_order(const int32_t *ptr, int n_major, int nnz, const int32_t *idx, const void *vals,
                              int val_bytes, int32_t *oidx, void *ovals, int32_t *slots, int T, int banks,
                              cudaStream_t s) {
    if (n_major <= 0 || nnz <= 0) return cudaSuccess;
    if (banks != 16 && banks != 32) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long>(((long)n_major + BO_WARPS - 1) / BO_WARPS, 152L * 64);
    const int nbm = banks - 1;
    const int tb = BO_WARPS * 32;
    if (val_bytes == 8)
        bank_order_kernel<uint64_t><<<grid, tb, 0, s>>>(ptr, n_major, nnz, idx, static_cast<const uint64_t *>(vals),
                                                        oidx, static_cast<uint64_t *>(ovals), slots, T, nbm);
    else if (val_bytes == 4)
        bank_order_kernel<uint32_t><<<grid, tb, 0, s>>>(ptr, n_major, nnz, idx, static_cast<const uint32_t *>(vals),
                                                        oidx, static_cast<uint32_t *>(ovals), slots, T, nbm);
    else
        bank_order_kernel<uint16_t><<<grid, tb, 0, s>>>(ptr, n_major, nnz, idx, static_cast<const uint16_t *>(vals),
                                                        oidx, static_cast<uint16_t *>(ovals), slots, T, nbm);
    return cudaGetLastError();
}

}  // namespace gbk
