// Plans from coordinate triples (row, column, value) stored in the matrix's storage
// order -- column-major for a wide CSC matrix, row-major for a tall CSR one -- the
// triple stream the paper's implementation reads (Sec. V).  The compressed
// pointer array is derived on the device (the plan owns it); the minor indices and
// the values are borrowed as they are.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

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

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" spmv_status spmv_plan_coo(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout,
                                     const int32_t *rows, const int32_t *cols, const void *vals, int32_t val_dtype,
                                     int32_t vec_dtype, void *stream, uint32_t flags, const spmv_plan_opts *opts) {
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (layout != SPMV_CSC_WIDE && layout != SPMV_CSR_TALL) return set_error(SPMV_ERR_INVALID_ARG, "bad layout");
    if (m < 0 || n < 0 || nnz < 0 || m >= (1ll << 31) - 64 || n >= (1ll << 31) - 64 || nnz >= (1ll << 31) - 64)
        return set_error(SPMV_ERR_INVALID_ARG, "m, n and nnz must lie in [0, 2^31 - 64)");
    if (nnz > 0 && (!rows || !cols || !vals)) return set_error(SPMV_ERR_INVALID_ARG, "rows/cols/vals are NULL");
    const bool csc = layout == SPMV_CSC_WIDE;
    const int32_t *major = csc ? cols : rows;
    const int32_t *minor = csc ? rows : cols;
    const int n_major = (int)(csc ? n : m);
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
    if (nnz > 0) coo_check_kernel<<<grid, 256, 0, s>>>(major, nnz, n_major, err);
    coo_ptr_kernel<<<grid, 256, 0, s>>>(major, nnz, n_major, ptr);
    if (cudaGetLastError() != cudaSuccess) return fail(SPMV_ERR_CUDA, "launch failed");
    int32_t e = 0;
    if (cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(SPMV_ERR_CUDA, "pointer construction failed");
    if (e & 1) return fail(SPMV_ERR_BAD_MATRIX, "a major index lies outside the matrix");
    if (e & 2) return fail(SPMV_ERR_BAD_MATRIX, "triples are not in storage order (major index decreases)");
    spmv_status st = spmv_plan_ex(out, m, n, nnz, layout, ptr, minor, vals, val_dtype, vec_dtype, stream, flags, opts);
    if (st != SPMV_OK) {
        cudaFree(ptr);
        return st;
    }
    (*out)->owned_ptr = ptr;  // freed with the plan
    return SPMV_OK;
}
