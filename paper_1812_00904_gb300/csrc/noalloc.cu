// Allocation-free SpMV: y = A x for a wide CSC matrix with FP32 values and
// vectors, for callers that may not allocate device memory at call time (for
// example code running inside a memory pool that forbids new allocations, or
// a host runtime that hands the library only pre-sized buffers).  The
// nonzeros are split over the CTAs by the same equal-count rule as the
// planned path; each CTA accumulates its share of y in shared memory and
// writes it as one partial vector into a fixed scratch array that lives in
// this library's static device memory; the existing fixed-order combine
// kernel then sums the partials in FP64 into y.
//
// Nothing is checked on the device: an index outside [0, m) is skipped, and
// the column walks never leave [0, n) even when ptr is malformed, but neither
// is reported (the call allocates nothing, not even an error word to read back).
//
// The scratch array is a file-scope __device__ array: every device that loads
// the library holds it (16 MiB) until the process exits, and every call shares
// it, so calls that overlap on the GPU race on it.  Each call overwrites the
// partial vectors it uses before reading them, so nothing needs clearing.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>
#include <mutex>

#include "plan_impl.h"

namespace gbk {

constexpr size_t NOALLOC_SCRATCH_FLOATS = size_t(1) << 22;  // 16 MiB of per-CTA partial sums
constexpr int NOALLOC_MAX_M = 49152;                          // rows accumulated in shared memory (192 KiB)
constexpr int NOALLOC_THREADS = 512;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

// One CTA per nonzero chunk; each warp walks an equal share of the chunk 32
// nonzeros at a time and finds every lane's column among the next 32 column
// ends with a shuffle binary search.
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_scatter_kernel(
    const int32_t *__restrict__ ptr, const int32_t *__restrict__ idx, const float *__restrict__ vals,
    const float *__restrict__ x, int m, int n, int nnz, float *__restrict__ part) {
    extern __shared__ float acc[];
    for (int i = threadIdx.x; i < m; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int P = gridDim.x, c = blockIdx.x;
    const int q = nnz / P, r = nnz % P;
    const int kb = c * q + min(c, r);
    const int ke = kb + q + (c < r ? 1 : 0);
    const int len = ke - kb, wq = len / W, wr = len % W;
    const int wb = kb + warp * wq + min(warp, wr);
    const int we = wb + wq + (warp < wr ? 1 : 0);
    if (wb < we) {
        // column holding nonzero wb: the last j with ptr[j] <= wb
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = lo + (hi - lo + 1) / 2;
            if (ptr[mid] <= wb)
                lo = mid;
            else
                hi = mid - 1;
        }
        int col = lo;  // in [0, n - 1] (n >= 1 here)
        for (int base = wb; base < we; base += 32) {
            const int k = base + lane;
            while (col + 1 < n && ptr[col + 1] <= base) ++col;  // warp-uniform: column holding position base
            const int ej = (col + 1 + lane <= n) ? ptr[col + 1 + lane] : INT_MAX;  // end of column col + lane
            int cnt = 0;  // number of those ends at or before k
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, ej, cnt + step - 1);
                if (v <= k) cnt += step;
            }
            const int e31 = __shfl_sync(0xffffffffu, ej, 31);
            if (cnt == 31 && e31 <= k) cnt = 32;
            int mycol = min(col + cnt, n - 1);
            if (k < we) {
                while (mycol + 1 < n && ptr[mycol + 1] <= k) ++mycol;  // only past runs of empty columns
                const int row = idx[k];
                if (static_cast<unsigned>(row) < static_cast<unsigned>(m)) atomicAdd(&acc[row], vals[k] * x[mycol]);
            }
        }
    }
    __syncthreads();
    float *dst = part + (size_t)c * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) dst[i] = acc[i];
}

struct NoallocDevice {
    float *scratch = nullptr;
    int sms = 0;
    bool ready = false;
};

static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];

}  // namespace gbk

using namespace gbk;

extern "C" spmv_status spmv_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *ptr, const int32_t *idx,
                                    const float *vals, const float *x, float *y, void *stream) {
    if (m < 0 || n < 0 || nnz < 0 || nnz >= (1ll << 31) - 64 || n >= (1ll << 31) - 64)
        return set_error(SPMV_ERR_INVALID_ARG, "spmv_noalloc: sizes out of range");
    if (m > NOALLOC_MAX_M)
        return set_error(SPMV_ERR_INVALID_ARG, "spmv_noalloc: m exceeds the allocation-free limit of 49152 rows");
    if (m == 0) return SPMV_OK;
    if (!ptr || !y || (nnz > 0 && (!idx || !vals || !x)))
        return set_error(SPMV_ERR_INVALID_ARG, "spmv_noalloc: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(SPMV_ERR_CUDA, "spmv_noalloc: no usable current device");
    NoallocDevice &D = g_noalloc_dev[dev];
    {
        // first call on this device: resolve the device address of the static scratch
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!D.ready) {
            void *a = nullptr;
            cudaError_t r1 = cudaGetSymbolAddress(&a, g_noalloc_scratch);
            int sms = 0;
            cudaError_t r3 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaError_t r4 = cudaFuncSetAttribute(noalloc_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  NOALLOC_MAX_M * (int)sizeof(float));
            if (r1 != cudaSuccess || r3 != cudaSuccess || r4 != cudaSuccess)
                return set_error(SPMV_ERR_CUDA, "spmv_noalloc: device set-up failed");
            D.scratch = static_cast<float *>(a);
            D.sms = sms;
            D.ready = true;
        }
    }
    if (nnz == 0 || n == 0) {
        if (cudaMemsetAsync(y, 0, (size_t)m * sizeof(float), s) != cudaSuccess)
            return set_error(SPMV_ERR_CUDA, "spmv_noalloc: memset failed");
        return SPMV_OK;
    }
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>(D.sms, (int64_t)(NOALLOC_SCRATCH_FLOATS / (size_t)m)));
    noalloc_scatter_kernel<<<P, NOALLOC_THREADS, (size_t)m * sizeof(float), s>>>(ptr, idx, vals, x, (int)m, (int)n,
                                                                                  (int)nnz, D.scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SPMV_ERR_CUDA, std::string("spmv_noalloc: ") + cudaGetErrorString(e));
    void *outs[1] = {y};
    e = launch_combine(false, false, D.scratch, P, (int)m, 1, outs, s);
    if (e != cudaSuccess) return set_error(SPMV_ERR_CUDA, std::string("spmv_noalloc: ") + cudaGetErrorString(e));
    return SPMV_OK;
}
