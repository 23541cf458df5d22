// Cross-chunk combines: the sum of the per-CTA partial short vectors (the
// Allreduce of Sec. III) and the overlap-zone fixup (the per-zone reductions of
// Sec. IV-A).  Both add in FP64 in a fixed order, so results do not depend on
// which CTA finished first.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace gbk {

struct OutPtrs {
    void *p[KB_MAX];
};

// out_b[i] = sum_{q < nparts} part[(q * kb + b) * n_minor + i]
template <typename XT, typename PT>
__global__ void __launch_bounds__(256) combine_kernel(const PT *__restrict__ part, int nparts, int n_minor, int kb,
                                                      OutPtrs out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= n_minor) return;
    const PT *src = part + (size_t)b * n_minor + i;
    const size_t stride = (size_t)kb * n_minor;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int q = 0;
    // four independent loads in flight; the final order (s0+s1)+(s2+s3) is fixed
    for (; q + 4 <= nparts; q += 4) {
        s0 += static_cast<double>(__ldg(src + (size_t)(q + 0) * stride));
        s1 += static_cast<double>(__ldg(src + (size_t)(q + 1) * stride));
        s2 += static_cast<double>(__ldg(src + (size_t)(q + 2) * stride));
        s3 += static_cast<double>(__ldg(src + (size_t)(q + 3) * stride));
    }
    for (; q < nparts; ++q) s0 += static_cast<double>(__ldg(src + (size_t)q * stride));
    static_cast<XT *>(out.p[b])[i] = static_cast<XT>((s0 + s1) + (s2 + s3));
}

// Zone k spans chunks S_k = [first, last]: u_{j_k} = right record of the first
// chunk + whole-chunk records of the middle chunks + left record of the last.
template <typename XT>
__global__ void __launch_bounds__(256) fixup_kernel(const ZoneDev *__restrict__ zones, int z,
                                                    const double *__restrict__ rec_left,
                                                    const double *__restrict__ rec_right, int P, int kb, OutPtrs out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z) return;
    const ZoneDev zd = zones[k];
    for (int b = 0; b < kb; ++b) {
        double s = rec_right[(size_t)b * P + zd.first];
        for (int c = zd.first + 1; c < zd.last; ++c) s += rec_right[(size_t)b * P + c];
        s += rec_left[(size_t)b * P + zd.last];
        static_cast<XT *>(out.p[b])[zd.col] = static_cast<XT>(s);
    }
}

cudaError_t launch_combine(bool vec_f64, bool part_f64, const void *part, int nparts, int n_minor, int kb,
                           void *const *out, cudaStream_t s) {
    if (n_minor <= 0) return cudaSuccess;
    OutPtrs o;
    for (int b = 0; b < KB_MAX; ++b) o.p[b] = b < kb ? out[b] : nullptr;
    dim3 grid((n_minor + 255) / 256, kb);
    if (vec_f64) {
        combine_kernel<double, double><<<grid, 256, 0, s>>>(static_cast<const double *>(part), nparts, n_minor, kb, o);
    } else if (part_f64) {
        combine_kernel<float, double><<<grid, 256, 0, s>>>(static_cast<const double *>(part), nparts, n_minor, kb, o);
    } else {
        combine_kernel<float, float><<<grid, 256, 0, s>>>(static_cast<const float *>(part), nparts, n_minor, kb, o);
    }
    return cudaGetLastError();
}

cudaError_t launch_fixup(bool vec_f64, const ZoneDev *zones, int z, const double *rec_left, const double *rec_right,
                         int P, int kb, void *const *out, cudaStream_t s) {
    if (z <= 0) return cudaSuccess;
    OutPtrs o;
    for (int b = 0; b < KB_MAX; ++b) o.p[b] = b < kb ? out[b] : nullptr;
    const int grid = (z + 255) / 256;
    if (vec_f64)
        fixup_kernel<double><<<grid, 256, 0, s>>>(zones, z, rec_left, rec_right, P, kb, o);
    else
        fixup_kernel<float><<<grid, 256, 0, s>>>(zones, z, rec_left, rec_right, P, kb, o);
    return cudaGetLastError();
}

}  // namespace gbk
