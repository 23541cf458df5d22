// Cross-chunk combines: the sum of the per-CTA partial short vectors (the
// Allreduce of Sec. III) and the overlap-zone fixup (the per-zone reductions of
// Sec. IV-A).  Both add in a fixed order, so results do not depend on which CTA
// finished first: FP32 data in compensated FP32 pairs, FP64 data in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace gbk {

struct OutPtrs {
    void *p[KB_MAX];
};

// Compensated addition (TwoSum): s + c accumulates v with the rounding error of
// every addition kept in c.  The error term is exact whatever the operand order.
template <typename T> __device__ __forceinline__ void two_sum_add(T &s, T &c, T v) {
    const T t = s + v;
    const T bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

// out_b[i] = sum_{q < nparts} part[(q * kb + b) * n_minor + i].  A block takes 32
// consecutive elements; its 8 thread rows sum the partials q = row, row + 8, ... and
// the 8 row sums are added in row order: a fixed order, independent of timing.
// FP32 partials are added with TwoSum in FP32 pairs (about twice the FP32 precision,
// without the FP64 pipe); FP64 partials in FP64.
constexpr int COMB_X = 32, COMB_Y = 8;
template <typename XT, typename PT>
__global__ void __launch_bounds__(COMB_X * COMB_Y) combine_kernel(const PT *__restrict__ part, int nparts, int n_minor,
                                                                  int kb, OutPtrs out) {
    using T = PT;
    __shared__ T sh_s[COMB_Y][COMB_X], sh_c[COMB_Y][COMB_X];
    const int i = blockIdx.x * COMB_X + threadIdx.x;
    const int b = blockIdx.y;
    const int row = threadIdx.y;
    T s = T(0), c = T(0);
    if (i < n_minor) {
        const PT *src = part + (size_t)b * n_minor + i;
        const size_t stride = (size_t)kb * n_minor;
#pragma unroll 4
        for (int q = row; q < nparts; q += COMB_Y) two_sum_add(s, c, __ldg(src + (size_t)q * stride));
    }
    sh_s[row][threadIdx.x] = s;
    sh_c[row][threadIdx.x] = c;
    __syncthreads();
    if (row == 0 && i < n_minor) {
        T ts = sh_s[0][threadIdx.x], tc = sh_c[0][threadIdx.x];
#pragma unroll
        for (int r = 1; r < COMB_Y; ++r) {
            two_sum_add(ts, tc, sh_s[r][threadIdx.x]);
            tc += sh_c[r][threadIdx.x];
        }
        static_cast<XT *>(out.p[b])[i] = static_cast<XT>(ts + tc);
    }
}

// Zone k spans tiles S_k = [first, last]: u_{j_k} = right record of the first
// tile + the records of the middle tiles (whole-tile sums, kept as right records)
// + left record of the last, added in this order with TwoSum in the accumulation
// type.  One thread per zone (most zones span two tiles); the loads of a long zone
// are issued eight at a time.  Every zone's column is written once.
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
        const RT l = rec_left[(size_t)b * P + zd.last];
        T s = f.x, c = f.y;
        int q = zd.first + 1;
        for (; q + 8 <= zd.last; q += 8) {
            RT m[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) m[e] = rr[q + e];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                two_sum_add(s, c, m[e].x);
                c += m[e].y;
            }
        }
        for (; q < zd.last; ++q) {
            const RT m = rr[q];
            two_sum_add(s, c, m.x);
            c += m.y;
        }
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
    const dim3 grid((n_minor + COMB_X - 1) / COMB_X, kb), block(COMB_X, COMB_Y);
    if (vec_f64) {
        combine_kernel<double, double><<<grid, block, 0, s>>>(static_cast<const double *>(part), nparts, n_minor, kb, o);
    } else if (part_f64) {
        combine_kernel<float, double><<<grid, block, 0, s>>>(static_cast<const double *>(part), nparts, n_minor, kb, o);
    } else {
        combine_kernel<float, float><<<grid, block, 0, s>>>(static_cast<const float *>(part), nparts, n_minor, kb, o);
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
