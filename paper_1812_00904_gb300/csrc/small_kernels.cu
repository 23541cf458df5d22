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

// Zone k spans tiles S_k = [first, last]: u_{j_k} = right record of the first
// tile + whole-tile records of the middle tiles + left record of the last.
// Records are (hi, lo) pairs of the accumulation type, added with
// compensated (TwoSum) arithmetic in that type in a fixed order.
template <typename T> __device__ __forceinline__ void two_sum_add(T &s, T &c, T v) {
    const T t = s + v;
    const T bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

template <typename XT, typename T, typename RT>
__global__ void __launch_bounds__(256) fixup_kernel(const ZoneDev *__restrict__ zones, int z,
                                                    const RT *__restrict__ rec_left, const RT *__restrict__ rec_right,
                                                    int P, int kb, OutPtrs out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z) return;
    const ZoneDev zd = zones[k];
    for (int b = 0; b < kb; ++b) {
        const RT *rr = rec_right + (size_t)b * P;
        const RT f = rr[zd.first];
        T s = f.x, c = f.y;
        for (int q = zd.first + 1; q < zd.last; ++q) {
            const RT m = rr[q];
            two_sum_add(s, c, m.x);
            c += m.y;
        }
        const RT l = rec_left[(size_t)b * P + zd.last];
        two_sum_add(s, c, l.x);
        c += l.y;
        static_cast<XT *>(out.p[b])[zd.col] = static_cast<XT>(s + c);
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

cudaError_t launch_fixup(bool vec_f64, const ZoneDev *zones, int z, const void *rec_left, const void *rec_right,
                         int P, int kb, void *const *out, cudaStream_t s) {
    if (z <= 0) return cudaSuccess;
    OutPtrs o;
    for (int b = 0; b < KB_MAX; ++b) o.p[b] = b < kb ? out[b] : nullptr;
    const int grid = (z + 255) / 256;
    if (vec_f64)
        fixup_kernel<double, double, double2><<<grid, 256, 0, s>>>(zones, z, static_cast<const double2 *>(rec_left),
                                                           static_cast<const double2 *>(rec_right), P, kb, o);
    else
        fixup_kernel<float, float, float2><<<grid, 256, 0, s>>>(zones, z, static_cast<const float2 *>(rec_left),
                                                         static_cast<const float2 *>(rec_right), P, kb, o);
    return cudaGetLastError();
}

}  // namespace gbk
