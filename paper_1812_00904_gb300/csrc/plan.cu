// Plan kernels: structural checks, the nonzero partition of Sec. II, the
// overlap-zone set-up of Sec. IV-B (needLeft, needRight, leftGroupEnd,
// rightGroup, leftGroup, procsOnLeft, procsOnRight), and the merge-order tiles
// each chunk streams through shared memory.
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

// One thread per chunk c: its nonzeros by the Sec. II rule, its first and
// last segment (j^f, j^l), the segment end events it owns and its tile count.
__global__ void chunks_kernel(const int32_t *__restrict__ pptr, int n_major, int nnz, int P, int D,
                              ChunkAux *__restrict__ aux) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P) return;
    const int q = nnz / P, r = nnz % P;
    const int nzb = c * q + min(c, r);
    const int nze = nzb + q + (c < r ? 1 : 0);
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
    const long items = (long)(a.e_end - a.e_begin) + (nze - nzb);
    a.ntiles = (int)((items + D - 1) / D);
    a.needLeft = a.needRight = a.leftGroupEnd = a.rightGroup = a.leftGroup = a.procsOnLeft = a.procsOnRight = 0;
    aux[c] = a;
}

cudaError_t launch_chunks(const int32_t *pptr, int n_major, int nnz, int P, int D, ChunkAux *aux, cudaStream_t s) {
    chunks_kernel<<<(P + 255) / 256, 256, 0, s>>>(pptr, n_major, nnz, P, D, aux);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Sec. IV-B on one CTA.  Thread t owns the chunk range [t*per, (t+1)*per); each
// scan is: local pass, sequential scan of the per-thread aggregates by thread
// 0, local re-scan from the thread's prefix.

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

constexpr int SETUP_THREADS = 1024;

__global__ void __launch_bounds__(SETUP_THREADS) setup_kernel(ChunkAux *__restrict__ aux, int P,
                                                              ChunkDev *__restrict__ chunks,
                                                              ZoneDev *__restrict__ zones, int32_t *counts) {
    __shared__ int sh_a[SETUP_THREADS];
    __shared__ int sh_b[SETUP_THREADS];
    __shared__ SegPair sh_p[SETUP_THREADS];
    const int t = threadIdx.x;
    const int per = (P + SETUP_THREADS - 1) / SETUP_THREADS;
    const int lo = min(P, t * per), hi = min(P, lo + per);

    // "Determine overlap zones": needLeft / needRight from the neighbours' first and last segments
    for (int c = lo; c < hi; ++c) {
        ChunkAux a = aux[c];
        const bool ne = a.nz_end > a.nz_begin;
        a.needLeft = (c > 0 && ne && aux[c - 1].nz_end > aux[c - 1].nz_begin && a.jf == aux[c - 1].jl) ? 1 : 0;
        a.needRight = (c < P - 1 && ne && aux[c + 1].nz_end > aux[c + 1].nz_begin && a.jl == aux[c + 1].jf) ? 1 : 0;
        // "Determine ranks of overlap groups"
        a.leftGroupEnd = (a.needLeft == 1 && (a.needRight == 0 || a.jf != a.jl)) ? 1 : 0;
        aux[c].needLeft = a.needLeft;
        aux[c].needRight = a.needRight;
        aux[c].leftGroupEnd = a.leftGroupEnd;
    }
    __syncthreads();
    // additive scans: rightGroup = inclusive scan of leftGroupEnd; tile offsets = exclusive scan of ntiles
    int s_lge = 0, s_tiles = 0;
    for (int c = lo; c < hi; ++c) {
        s_lge += aux[c].leftGroupEnd;
        s_tiles += aux[c].ntiles;
    }
    sh_a[t] = s_lge;
    sh_b[t] = s_tiles;
    __syncthreads();
    if (t == 0) {
        int ra = 0, rb = 0;
        for (int i = 0; i < SETUP_THREADS; ++i) {
            const int va = sh_a[i], vb = sh_b[i];
            sh_a[i] = ra;
            sh_b[i] = rb;
            ra += va;
            rb += vb;
        }
        counts[0] = ra;  // z = number of overlap zones
        counts[1] = rb;  // total tiles
    }
    __syncthreads();
    {
        int ra = sh_a[t], rb = sh_b[t];
        for (int c = lo; c < hi; ++c) {
            ra += aux[c].leftGroupEnd;
            aux[c].rightGroup = ra;
            aux[c].leftGroup = ra - aux[c].leftGroupEnd;
            chunks[c].tile_begin = rb;
            rb += aux[c].ntiles;
            chunks[c].tile_end = rb;
        }
    }
    __syncthreads();
    // "Determine group extents": forward o-scan of (needLeft, leftGroup) -> procsOnLeft
    {
        SegPair agg{0, 0, 0};
        for (int c = lo; c < hi; ++c) agg = seg_op(agg, SegPair{aux[c].needLeft, aux[c].leftGroup, 1});
        sh_p[t] = agg;
        __syncthreads();
        if (t == 0) {
            SegPair run{0, 0, 0};
            for (int i = 0; i < SETUP_THREADS; ++i) {
                const SegPair v = sh_p[i];
                sh_p[i] = run;
                run = seg_op(run, v);
            }
        }
        __syncthreads();
        SegPair run = sh_p[t];
        for (int c = lo; c < hi; ++c) {
            run = seg_op(run, SegPair{aux[c].needLeft, aux[c].leftGroup, 1});
            aux[c].procsOnLeft = run.s;
        }
    }
    __syncthreads();
    // backward o-scan of (needRight, rightGroup) -> procsOnRight
    {
        SegPair agg{0, 0, 0};
        for (int c = hi - 1; c >= lo; --c) agg = seg_op(agg, SegPair{aux[c].needRight, aux[c].rightGroup, 1});
        sh_p[t] = agg;
        __syncthreads();
        if (t == 0) {
            SegPair run{0, 0, 0};
            for (int i = SETUP_THREADS - 1; i >= 0; --i) {
                const SegPair v = sh_p[i];
                sh_p[i] = run;
                run = seg_op(run, v);
            }
        }
        __syncthreads();
        SegPair run = sh_p[t];
        for (int c = hi - 1; c >= lo; --c) {
            run = seg_op(run, SegPair{aux[c].needRight, aux[c].rightGroup, 1});
            aux[c].procsOnRight = run.s;
        }
    }
    __syncthreads();
    // descriptors and the zone list: the chunk closing a left group names zone leftGroup
    int vmax = 0;
    for (int c = lo; c < hi; ++c) {
        const ChunkAux a = aux[c];
        ChunkDev d = chunks[c];
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
    sh_a[t] = vmax;
    __syncthreads();
    if (t == 0) {
        int v = 0;
        for (int i = 0; i < SETUP_THREADS; ++i) v = max(v, sh_a[i]);
        counts[2] = v;  // V = max |S_k|
    }
}

cudaError_t launch_setup(ChunkAux *aux, int P, ChunkDev *chunks, ZoneDev *zones, int32_t *counts, cudaStream_t s) {
    setup_kernel<<<1, SETUP_THREADS, 0, s>>>(aux, P, chunks, zones, counts);
    return cudaGetLastError();
}

// One thread per tile: the tile starts where the merge order of segment ends
// and nonzeros reaches the diagonal e_begin + nz_begin + q*D (the classic merge
// path split), moved back to right before a nonzero at a multiple of 8 so that
// every staged copy starts on a 16-byte boundary.
__global__ void tiles_kernel(const int32_t *__restrict__ pptr, int n_major, const ChunkAux *__restrict__ aux,
                             const ChunkDev *__restrict__ chunks, int P, int D, int ntiles, int4 *__restrict__ tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    // chunk owning tile t: the last chunk with tile_begin <= t
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (chunks[mid].tile_begin <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ChunkAux a = aux[lo];
    const int q = t - chunks[lo].tile_begin;
    int4 out;
    out.z = 0;
    out.w = 0;
    if (q == 0) {
        out.x = a.nz_begin;
        out.y = a.e_begin;
    } else {
        const long d = (long)a.e_begin + a.nz_begin + (long)q * D;
        // largest i in [ilo, ihi] with pptr[i] + i <= d
        int ilo = (int)max((long)a.e_begin, d - a.nz_end);
        int ihi = (int)min((long)a.e_end, d - a.nz_begin);
        while (ilo < ihi) {
            const int mid = ilo + (ihi - ilo + 1) / 2;
            if ((long)pptr[mid] + mid <= d)
                ilo = mid;
            else
                ihi = mid - 1;
        }
        const int k = (int)(d - ilo);
        const int kk = max(a.nz_begin, k & ~7);
        int e = ends_upto(pptr, a.e_begin, a.e_end, kk);
        out.x = kk;
        out.y = e;
    }
    tiles[t] = out;
}

cudaError_t launch_tiles(const int32_t *pptr, int n_major, const ChunkAux *aux, const ChunkDev *chunks, int P, int D,
                         int ntiles, int4 *tiles, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    tiles_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(pptr, n_major, aux, chunks, P, D, ntiles, tiles);
    return cudaGetLastError();
}

// One warp per tile: the segment-start bits of the tile (bit pos set when a
// segment j in (i0, i1] starts at nonzero kb0 + pos, pos < k1 - kb0), and flag
// bit 0 when an empty segment ends inside the tile (then several segments can
// start at one position and the kernels take their general path).
__global__ void masks_kernel(const int32_t *__restrict__ pptr, const ChunkDev *__restrict__ chunks, int P, int ntiles,
                             int mwp, int4 *__restrict__ tiles, uint32_t *__restrict__ masks) {
    __shared__ uint32_t sm[8][32];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int t = blockIdx.x * 8 + wib;
    if (t >= ntiles) return;
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (chunks[mid].tile_begin <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    const ChunkDev cd = chunks[lo];
    const int4 a = tiles[t];
    int k1, i1;
    if (t + 1 < cd.tile_end) {
        const int4 b = tiles[t + 1];
        k1 = b.x;
        i1 = b.y;
    } else {
        k1 = cd.nz_end;
        i1 = cd.e_end;
    }
    const int kb0 = a.x & ~7;
    const int rel_hi = k1 - kb0;
    sm[wib][lane] = 0u;
    __syncwarp();
    bool dup = false;
    for (int j = a.y + 1 + lane; j <= i1; j += 32) {
        const int pj = pptr[j];
        const int pos = pj - kb0;
        if (pos >= 0 && pos < rel_hi && pos < 1024) atomicOr(&sm[wib][pos >> 5], 1u << (pos & 31));
        if (j < i1 && pptr[j + 1] == pj) dup = true;
    }
    dup = __any_sync(0xffffffffu, dup);
    __syncwarp();
    if (lane < mwp) masks[(size_t)t * mwp + lane] = sm[wib][lane];
    if (lane == 0) tiles[t].z = dup ? 1 : 0;
}

cudaError_t launch_masks(const int32_t *pptr, const ChunkDev *chunks, int P, int ntiles, int mwp, int4 *tiles,
                         uint32_t *masks, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    masks_kernel<<<(ntiles + 7) / 8, 256, 0, s>>>(pptr, chunks, P, ntiles, mwp, tiles, masks);
    return cudaGetLastError();
}

}  // namespace gbk
