// Plans from coordinate triples (row, column, value) stored in the matrix's storage
// order -- column-major for a wide CSC matrix, row-major for a tall CSR one -- the
// triple stream the paper's implementation reads (Sec. V).  The compressed
// pointer array is derived on the device (the plan owns it); the minor indices and
// the values are borrowed as they are.  Triples in any order (SPMV_PLAN_COO_UNSORTED)
// are first sorted on the device by (major, minor) index into a plan-owned copy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <utility>

#include "plan_impl.h"

namespace gbk {
namespace {

// err bit 1: a major index outside [0, n_major); bit 2: major indices decreasing
__global__ void coo_check_kernel(const int32_t *__restrict__ major, int64_t nnz, int n_major, int32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int32_t j = major[k];
        if (static_cast<uint32_t>(j) >= static_cast<uint32_t>(n_major)) atomicOr(err, 1);
        if (k > 0 && major[k - 1] > j) atomicOr(err, 2);
    }
}

// ptr[j] = number of triples whose major index is below j (binary search of the sorted stream)
__global__ void coo_ptr_kernel(const int32_t *__restrict__ major, int64_t nnz, int n_major, int32_t *__restrict__ ptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n_major; j += stride) {
        int64_t lo = 0, hi = nnz;  // first k with major[k] >= j
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (major[mid] < j)
                lo = mid + 1;
            else
                hi = mid;
        }
        ptr[j] = static_cast<int32_t>(lo);
    }
}

// ---- stable LSD radix sort of 64-bit keys (major * n_minor + minor) with a 32-bit payload (the
// triple's input position), 8 bits per pass.  A tile is 4096 keys: 256 threads x 16 rounds; in
// round j thread t holds tile element j * 256 + t, so tile order is round-major and every load is
// coalesced.  Deterministic: every key's destination follows from the keys alone.
constexpr int RS_THREADS = 256, RS_ROUNDS = 16, RS_TILE = RS_THREADS * RS_ROUNDS, RS_BINS = 256;

__device__ __forceinline__ int digit_of(uint64_t key, int shift) { return (int)((key >> shift) & 0xFFu); }

// err bit 1: major index outside [0, n_major); bit 4: minor index outside [0, n_minor)
__global__ void coo_keys_kernel(const int32_t *__restrict__ major, const int32_t *__restrict__ minor, int64_t nnz,
                                int n_major, int n_minor, uint64_t *__restrict__ keys, int32_t *__restrict__ pay,
                                int32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bits = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int32_t j = major[k], i = minor[k];
        const bool okj = static_cast<uint32_t>(j) < static_cast<uint32_t>(n_major);
        const bool oki = static_cast<uint32_t>(i) < static_cast<uint32_t>(n_minor);
        if (!okj) bits |= 1;
        if (!oki) bits |= 4;
        keys[k] = (okj && oki) ? (uint64_t)j * (uint64_t)n_minor + (uint64_t)i : 0;
        pay[k] = (int32_t)k;
    }
    if (bits) atomicOr(err, bits);
}

// hist[d * ntiles + tile] = number of keys of the tile whose digit is d
__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(const uint64_t *__restrict__ keys, int64_t nnz,
                                                             int shift, int ntiles, int32_t *__restrict__ hist) {
    __shared__ int h[RS_BINS];
    const int t = threadIdx.x;
    h[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        const int64_t k = base + (int64_t)j * RS_THREADS + t;
        if (k < nnz) atomicAdd(&h[digit_of(keys[k], shift)], 1);
    }
    __syncthreads();
    hist[(int64_t)t * ntiles + blockIdx.x] = h[t];
}

// exclusive scan of n int32 values in place: per-block sums, one-block scan of the sums, block scans
constexpr int SC_THREADS = 1024, SC_ITEMS = 4, SC_CHUNK = SC_THREADS * SC_ITEMS;

__device__ int block_exclusive_scan(int v, int *warp_tot, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int x = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += o;
        }
        if (lane < nw) warp_tot[lane] = x;  // inclusive over warps
    }
    __syncthreads();
    total = warp_tot[nw - 1];
    const int before = w > 0 ? warp_tot[w - 1] : 0;
    __syncthreads();  // warp_tot is reused by the next call
    return before + inc - v;
}

__global__ void __launch_bounds__(SC_THREADS) scan_sums_kernel(const int32_t *__restrict__ a, int64_t n,
                                                               int32_t *__restrict__ sums) {
    __shared__ int wt[32];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
    int v = 0;
    for (int e = 0; e < SC_ITEMS; ++e)
        if (base + e < n) v += a[base + e];
    int total;
    block_exclusive_scan(v, wt, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SC_THREADS) scan_top_kernel(int32_t *__restrict__ sums, int nb) {
    __shared__ int wt[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SC_THREADS) {
        const int b = b0 + (int)threadIdx.x;
        const int v = b < nb ? sums[b] : 0;
        int total;
        const int ex = block_exclusive_scan(v, wt, total);
        if (b < nb) sums[b] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SC_THREADS) scan_apply_kernel(int32_t *__restrict__ a, int64_t n,
                                                                const int32_t *__restrict__ sums) {
    __shared__ int wt[32];
    const int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_ITEMS;
    int v[SC_ITEMS], tot = 0;
    for (int e = 0; e < SC_ITEMS; ++e) {
        v[e] = base + e < n ? a[base + e] : 0;
        tot += v[e];
    }
    int total;
    int run = sums[blockIdx.x] + block_exclusive_scan(tot, wt, total);
    for (int e = 0; e < SC_ITEMS; ++e) {
        if (base + e < n) a[base + e] = run;
        run += v[e];
    }
}

// stable scatter: a key goes to offs[d * ntiles + tile] + (keys of digit d before it in the tile)
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(const uint64_t *__restrict__ kin,
                                                                const int32_t *__restrict__ pin, int64_t nnz, int shift,
                                                                int ntiles, const int32_t *__restrict__ offs,
                                                                uint64_t *__restrict__ kout, int32_t *__restrict__ pout,
                                                                int32_t *err) {
    constexpr int NW = RS_THREADS / 32;
    __shared__ int run[RS_BINS];        // keys of each digit placed so far in this tile
    __shared__ int wcnt[NW][RS_BINS];   // this round: keys of each digit in each warp
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    run[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    for (int q = 0; q < NW; ++q) wcnt[q][t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int j = 0; j < RS_ROUNDS; ++j) {
        const int64_t k = base + (int64_t)j * RS_THREADS + t;
        const bool live = k < nnz;
        uint64_t key = 0;
        int32_t pl = 0;
        int d = -1;
        if (live) {
            key = kin[k];
            pl = pin[k];
            d = digit_of(key, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int before_in_warp = __popc(peers & ((1u << lane) - 1u));
        if (live && before_in_warp == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (live) {
            int pos = run[d] + before_in_warp;
            for (int q = 0; q < w; ++q) pos += wcnt[q][d];
            if (pos >= 0 && pos < nnz) {
                kout[pos] = key;
                pout[pos] = pl;
            } else {
                atomicOr(err, 8);
            }
        }
        __syncthreads();
        int add = 0;
        for (int q = 0; q < NW; ++q) {
            add += wcnt[q][t];
            wcnt[q][t] = 0;
        }
        run[t] += add;
        __syncthreads();
    }
}

// sorted keys -> major (for the pointer array), minor indices and the values gathered by payload
template <typename W>
__global__ void coo_unpack_kernel(const uint64_t *__restrict__ keys, const int32_t *__restrict__ pay, int64_t nnz,
                                  int n_minor, const W *__restrict__ vals, int32_t *__restrict__ major,
                                  int32_t *__restrict__ minor, W *__restrict__ ovals, int32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const uint64_t key = keys[k];
        const uint64_t j = key / (uint64_t)n_minor;
        major[k] = (int32_t)j;
        minor[k] = (int32_t)(key - j * (uint64_t)n_minor);
        const int32_t src = pay[k];
        if (src >= 0 && src < nnz) {
            ovals[k] = vals[src];
        } else {
            ovals[k] = W(0);
            atomicOr(err, 8);
        }
    }
}

}  // namespace

CooSort::~CooSort() {
    if (tmp) cudaFree(tmp);
    if (own) cudaFree(own);
}

cudaError_t launch_coo_ptr(const int32_t *major_sorted, int64_t nnz, int n_major, int32_t *ptr, int grid,
                           cudaStream_t s) {
    coo_ptr_kernel<<<grid, 256, 0, s>>>(major_sorted, nnz, n_major, ptr);
    return cudaGetLastError();
}

// Sorts the triples by (major, minor), stably: the sorted minor indices and values go to the
// plan-owned block, the sorted major indices to the temporary one; all three come back through
// the out-parameters.  Range errors are reported through `err` (read by the caller after a sync).
spmv_status coo_sort(CooSort &cs, const int32_t *major, const int32_t *minor, const void *vals, int sv, int64_t nnz,
                     int n_major, int n_minor, int grid, int32_t *err, cudaStream_t s, const int32_t **major_sorted,
                     int32_t **minor_sorted, void **vals_sorted) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const int ntiles = (int)((nnz + RS_TILE - 1) / RS_TILE);
    const int64_t nh = (int64_t)RS_BINS * ntiles;
    const int nsc = (int)((nh + SC_CHUNK - 1) / SC_CHUNK);
    const size_t kb = up((size_t)nnz * 8), pb = up((size_t)nnz * 4), hb = up((size_t)nh * 4), sb = up((size_t)nsc * 4);
    if (cudaMalloc(&cs.tmp, 2 * kb + 2 * pb + hb + sb) != cudaSuccess) return set_error(SPMV_ERR_OOM, "sort scratch");
    char *t = static_cast<char *>(cs.tmp);
    uint64_t *ka = reinterpret_cast<uint64_t *>(t), *kb2 = reinterpret_cast<uint64_t *>(t + kb);
    int32_t *pa = reinterpret_cast<int32_t *>(t + 2 * kb), *pb2 = reinterpret_cast<int32_t *>(t + 2 * kb + pb);
    int32_t *hist = reinterpret_cast<int32_t *>(t + 2 * kb + 2 * pb);
    int32_t *sums = reinterpret_cast<int32_t *>(t + 2 * kb + 2 * pb + hb);
    const size_t ib = up((size_t)nnz * 4);
    cs.own_bytes = ib + up((size_t)nnz * sv);
    if (cudaMalloc(&cs.own, cs.own_bytes) != cudaSuccess) return set_error(SPMV_ERR_OOM, "sorted triples");

    coo_keys_kernel<<<grid, 256, 0, s>>>(major, minor, nnz, n_major, n_minor, ka, pa, err);
    const uint64_t span = (uint64_t)n_major * (uint64_t)n_minor;
    const int bits = span > 1 ? 64 - __builtin_clzll(span - 1) : 0;
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<ntiles, RS_THREADS, 0, s>>>(ka, nnz, shift, ntiles, hist);
        scan_sums_kernel<<<nsc, SC_THREADS, 0, s>>>(hist, nh, sums);
        scan_top_kernel<<<1, SC_THREADS, 0, s>>>(sums, nsc);
        scan_apply_kernel<<<nsc, SC_THREADS, 0, s>>>(hist, nh, sums);
        rs_scatter_kernel<<<ntiles, RS_THREADS, 0, s>>>(ka, pa, nnz, shift, ntiles, hist, kb2, pb2, err);
        std::swap(ka, kb2);
        std::swap(pa, pb2);
    }
    int32_t *omin = static_cast<int32_t *>(cs.own);
    void *ovals = static_cast<char *>(cs.own) + ib;
    int32_t *omaj = pb2;  // the free payload buffer
    if (sv == 8)
        coo_unpack_kernel<uint64_t><<<grid, 256, 0, s>>>(ka, pa, nnz, n_minor, static_cast<const uint64_t *>(vals), omaj,
                                                         omin, static_cast<uint64_t *>(ovals), err);
    else if (sv == 4)
        coo_unpack_kernel<uint32_t><<<grid, 256, 0, s>>>(ka, pa, nnz, n_minor, static_cast<const uint32_t *>(vals), omaj,
                                                         omin, static_cast<uint32_t *>(ovals), err);
    else
        coo_unpack_kernel<uint16_t><<<grid, 256, 0, s>>>(ka, pa, nnz, n_minor, static_cast<const uint16_t *>(vals), omaj,
                                                         omin, static_cast<uint16_t *>(ovals), err);
    if (cudaGetLastError() != cudaSuccess) return set_error(SPMV_ERR_CUDA, "sort launch failed");
    *major_sorted = omaj;
    *minor_sorted = omin;
    *vals_sorted = ovals;
    return SPMV_OK;
}

}  // namespace gbk

using namespace gbk;

namespace {

int dsize(int t) { return t == SPMV_F64 ? 8 : t == SPMV_F32 ? 4 : (t == SPMV_BF16 || t == SPMV_F16) ? 2 : 0; }

}  // namespace

extern "C" spmv_status spmv_plan_coo(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                                     const int32_t *rows, const int32_t *cols, const void *vals, int32_t val_dtype,
                                     int32_t vec_dtype, void *stream, uint32_t flags, const spmv_plan_opts *opts) {
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (layout != SPMV_CSC_WIDE && layout != SPMV_CSR_TALL) return set_error(SPMV_ERR_INVALID_ARG, "bad layout");
    if (m < 0 || n < 0 || nnz < 0 || m >= (1ll << 31) - 64 || n >= (1ll << 31) - 64 || nnz >= (1ll << 31) - 64)
        return set_error(SPMV_ERR_INVALID_ARG, "m, n and nnz must lie in [0, 2^31 - 64)");
    if (nnz > 0 && (!rows || !cols || !vals)) return set_error(SPMV_ERR_INVALID_ARG, "rows/cols/vals are NULL");
    const bool unsorted = (flags & SPMV_PLAN_COO_UNSORTED) != 0;
    if (unsorted && dsize(val_dtype) == 0) return set_error(SPMV_ERR_INVALID_ARG, "unknown dtype");
    const bool csc = layout == SPMV_CSC_WIDE;
    const int32_t *major = csc ? cols : rows;
    const int32_t *minor = csc ? rows : cols;
    const int n_major = (int)(csc ? n : m);
    const int n_minor = (int)(csc ? m : n);
    if (nnz > 0 && (n_major == 0 || n_minor == 0))
        return set_error(SPMV_ERR_BAD_MATRIX, "nonzeros need a nonempty matrix");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int32_t *ptr = nullptr, *err = nullptr;
    if (cudaMalloc(&ptr, ((size_t)n_major + 1) * 4 + 16) != cudaSuccess) return set_error(SPMV_ERR_OOM, "pointer array");
    err = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(ptr) + (((size_t)n_major + 1) * 4 + 3) / 4 * 4);
    auto fail = [&](spmv_status st, const char *msg) {
        cudaFree(ptr);
        return set_error(st, msg);
    };
    if (cudaMemsetAsync(err, 0, 4, s) != cudaSuccess) return fail(SPMV_ERR_CUDA, "memset");
    const int grid = std::max(1, sms * 8);
    CooSort cs;
    const int32_t *maj_use = major, *min_use = minor;
    const void *vals_use = vals;
    if (unsorted && nnz > 0) {
        int32_t *omin = nullptr;
        void *ovals = nullptr;
        const spmv_status st = coo_sort(cs, major, minor, vals, dsize(val_dtype), nnz, n_major, n_minor, grid, err, s,
                                        &maj_use, &omin, &ovals);
        if (st != SPMV_OK) {
            cudaFree(ptr);
            return st;
        }
        min_use = omin;
        vals_use = ovals;
    } else if (nnz > 0) {
        coo_check_kernel<<<grid, 256, 0, s>>>(major, nnz, n_major, err);
    }
    coo_ptr_kernel<<<grid, 256, 0, s>>>(maj_use, nnz, n_major, ptr);
    if (cudaGetLastError() != cudaSuccess) return fail(SPMV_ERR_CUDA, "launch failed");
    int32_t e = 0;
    if (cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SPMV_ERR_CUDA, "pointer construction failed");
    if (e & 1) return fail(SPMV_ERR_BAD_MATRIX, "a major index lies outside the matrix");
    if (e & 4) return fail(SPMV_ERR_BAD_MATRIX, "a minor index lies outside the matrix");
    if (e & 2) return fail(SPMV_ERR_BAD_MATRIX, "triples are not in storage order (major index decreases)");
    if (e & 8) return fail(SPMV_ERR_DEVICE, "inconsistent triple sort");
    spmv_status st = spmv_plan_ex(out, m, n, nnz, layout, ptr, min_use, vals_use, val_dtype, vec_dtype, stream,
                                  flags, opts);
    if (st != SPMV_OK) {
        cudaFree(ptr);
        return st;
    }
    (*out)->owned_ptr = ptr;  // freed with the plan
    if (cs.own && !(*out)->owned_nz) {
        // the plan multiplies the sorted copy (a bank-ordered plan made its own copy of it instead)
        (*out)->owned_nz = cs.own;
        (*out)->owned_bytes = cs.own_bytes;
        cs.own = nullptr;
    }
    return SPMV_OK;
}
