// Cross-chunk combines: the sum of the per-CTA partial short vectors (the
// Allreduce of Sec. III) and the overlap-zone fixup (the per-zone reductions of
// Sec. IV-A).  Both add in FP64 and in a fixed order, so results do not depend
// on which CTA finished first; FP32 partials and (hi, lo) FP32 carry pairs are
// widened to FP64 on read.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"

namespace gbk {

struct OutPtrs {
    void *p[VL_MAX];
};
struct InPtrs {
    const void *p[VL_MAX];
};

// An FP32 value widened to FP64 exactly, by integer operations on its bits only: the FP64
// pipe (slow on this part) is left to the additions.  Normal numbers move the sign, the
// exponent (rebiased from 127 to 1023) and the mantissa; a subnormal m 2^-149 is normalised
// at its leading one bit h (exponent h - 149); zeros keep their sign; infinities and NaNs
// take the all-ones exponent with the mantissa bits (a NaN stays a NaN).
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t mant = u & 0x7FFFFFu;
    const uint64_t sign = static_cast<uint64_t>(u & 0x80000000u) << 32;
    uint64_t d;
    if (e == 0u) {
        const int h = 31 - __clz(mant | 1u);
        d = mant == 0u ? sign
                       : sign | (static_cast<uint64_t>(h + 874) << 52) |
                             (static_cast<uint64_t>(mant ^ (1u << h)) << (52 - h));
    } else {
        const uint64_t ed = e == 0xFFu ? 0x7FFull : static_cast<uint64_t>(e + 896u);
        d = sign | (ed << 52) | (static_cast<uint64_t>(mant) << 29);
    }
    return __longlong_as_double(static_cast<long long>(d));
}
__device__ __forceinline__ double widen(double f) { return f; }

// out_b[i] = sum_{q < nparts} part[q * qstride + b * bstride + i].  A block takes 32
// consecutive elements; its 8 thread rows sum the partials q = row, row + 8, ... in
// FP64 and the 8 row sums are added in row order: a fixed order, independent of
// timing.  Partials of any type are widened to FP64 before they are added.
constexpr int COMB_X = 32, COMB_Y = 8;
template <typename XT, typename PT>
__global__ void __launch_bounds__(COMB_X * COMB_Y) combine_kernel(const PT *__restrict__ part, int nparts, int n_minor,
                                                                  size_t qstride, size_t bstride, OutPtrs out) {
    __shared__ double sh_s[COMB_Y][COMB_X];
    const int i = blockIdx.x * COMB_X + threadIdx.x;
    const int b = blockIdx.y;
    const int row = threadIdx.y;
    double s = 0.0;
    if (i < n_minor) {
        const PT *src = part + (size_t)b * bstride + i;
#pragma unroll 4
        for (int q = row; q < nparts; q += COMB_Y) s += widen(__ldg(src + (size_t)q * qstride));
    }
    sh_s[row][threadIdx.x] = s;
    __syncthreads();
    if (row == 0 && i < n_minor) {
        double t = sh_s[0][threadIdx.x];
#pragma unroll
        for (int r = 1; r < COMB_Y; ++r) t += sh_s[r][threadIdx.x];
        static_cast<XT *>(out.p[b])[i] = static_cast<XT>(t);
    }
}

// Zone k spans tiles S_k = [first, last]: u_{j_k} = right record of the first
// tile + the records of the middle tiles (whole-tile sums, kept as right records)
// + left record of the last, added in this order in FP64 (the hi and the lo
// parts of the (hi, lo) records in two FP64 sums, added at the end).  One thread
// per zone (most zones span two tiles); the loads of a long zone are issued
// eight at a time.  Every zone's column is written once.
template <typename XT, typename RT>
__global__ void __launch_bounds__(256) fixup_kernel(const ZoneDev *__restrict__ zones, int z,
                                                    const RT *__restrict__ rec_left, const RT *__restrict__ rec_right,
                                                    int P, int kb, OutPtrs out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= z) return;
    const ZoneDev zd = zones[k];
    for (int b = 0; b < kb; ++b) {
        const RT *rr = rec_right + (size_t)b * P;
        const RT l = rec_left[(size_t)b * P + zd.last];
        // hi and lo parts summed apart in FP64 (for FP32 records both widen exactly)
        double sh = widen(rr[zd.first].x), sl = widen(rr[zd.first].y);
        int q = zd.first + 1;
        for (; q + 8 <= zd.last; q += 8) {
            RT m[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) m[e] = rr[q + e];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                sh += widen(m[e].x);
                sl += widen(m[e].y);
            }
        }
        for (; q < zd.last; ++q) {
            sh += widen(rr[q].x);
            sl += widen(rr[q].y);
        }
        sh += widen(l.x);
        sl += widen(l.y);
        const double s = sh + sl;
        static_cast<XT *>(out.p[b])[zd.col] = static_cast<XT>(s);
    }
}

cudaError_t launch_combine(bool vec_f64, bool part_f64, const void *part, int nparts, int n_minor, int kb,
                           void *const *out, cudaStream_t s, size_t qstride, size_t bstride) {
    if (n_minor <= 0) return cudaSuccess;
    if (kb < 1 || kb > VL_MAX) return cudaErrorInvalidValue;
    OutPtrs o;
    for (int b = 0; b < VL_MAX; ++b) o.p[b] = b < kb ? out[b] : nullptr;
    if (qstride == 0) {  // [part][vector][element]
        qstride = (size_t)kb * n_minor;
        bstride = (size_t)n_minor;
    }
    const dim3 grid((n_minor + COMB_X - 1) / COMB_X, kb), block(COMB_X, COMB_Y);
    if (vec_f64) {
        combine_kernel<double, double><<<grid, block, 0, s>>>(static_cast<const double *>(part), nparts, n_minor,
                                                               qstride, bstride, o);
    } else if (part_f64) {
        combine_kernel<float, double><<<grid, block, 0, s>>>(static_cast<const double *>(part), nparts, n_minor,
                                                              qstride, bstride, o);
    } else {
        combine_kernel<float, float><<<grid, block, 0, s>>>(static_cast<const float *>(part), nparts, n_minor,
                                                             qstride, bstride, o);
    }
    return cudaGetLastError();
}

// out[i * KB + b] = in_b[i] for b < kb, 0 for kb <= b < KB: k vectors interleaved for the
// multi-vector segmented passes over vectors kept in global memory.  A block moves IT
// consecutive entries of every vector: coalesced reads of each vector into shared memory,
// then coalesced writes of the interleaved rows.
template <typename XT, int KB>
__global__ void __launch_bounds__(256) interleave_kernel(InPtrs in, int kb, int64_t len, XT *__restrict__ out) {
    constexpr int IT = 256;
    constexpr int RS = KB + 1;  // padded row: no bank conflicts in either phase
    __shared__ XT sh[IT * RS];
    for (int64_t i0 = (int64_t)blockIdx.x * IT; i0 < len; i0 += (int64_t)gridDim.x * IT) {
        const int cnt = (int)(len - i0 < IT ? len - i0 : (int64_t)IT);
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const XT *src = b < kb ? static_cast<const XT *>(in.p[b]) : nullptr;
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) sh[t * RS + b] = src ? src[i0 + t] : XT(0);
        }
        __syncthreads();
        XT *dst = out + i0 * KB;
        for (int t = threadIdx.x; t < cnt * KB; t += blockDim.x) dst[t] = sh[(t / KB) * RS + t % KB];
        __syncthreads();
    }
}

cudaError_t launch_interleave(bool f64, int kbt, int kb, const void *const *in, int64_t len, void *out,
                              cudaStream_t s) {
    if (len <= 0) return cudaSuccess;
    if (kb < 1 || kb > kbt || kbt > VL_MAX || (f64 && kbt > KB_MAX)) return cudaErrorInvalidValue;
    InPtrs ip;
    for (int b = 0; b < VL_MAX; ++b) ip.p[b] = b < kb ? in[b] : nullptr;
    const int grid = (int)std::min<int64_t>((len + 255) / 256, 152 * 8);
    if (f64) {
        double *o = static_cast<double *>(out);
        if (kbt == 2) interleave_kernel<double, 2><<<grid, 256, 0, s>>>(ip, kb, len, o);
        else if (kbt == 4) interleave_kernel<double, 4><<<grid, 256, 0, s>>>(ip, kb, len, o);
        else interleave_kernel<double, 8><<<grid, 256, 0, s>>>(ip, kb, len, o);
    } else {
        float *o = static_cast<float *>(out);
        if (kbt == 2) interleave_kernel<float, 2><<<grid, 256, 0, s>>>(ip, kb, len, o);
        else if (kbt == 4) interleave_kernel<float, 4><<<grid, 256, 0, s>>>(ip, kb, len, o);
        else interleave_kernel<float, 8><<<grid, 256, 0, s>>>(ip, kb, len, o);
    }
    return cudaGetLastError();
}

cudaError_t launch_fixup(bool vec_f64, const ZoneDev *zones, int z, const void *rec_left, const void *rec_right,
                         int P, int kb, void *const *out, cudaStream_t s) {
    if (z <= 0) return cudaSuccess;
    if (kb < 1 || kb > VL_MAX) return cudaErrorInvalidValue;
    OutPtrs o;
    for (int b = 0; b < VL_MAX; ++b) o.p[b] = b < kb ? out[b] : nullptr;
    const int grid = (z + 255) / 256;
    if (vec_f64)
        fixup_kernel<double, double2><<<grid, 256, 0, s>>>(zones, z, static_cast<const double2 *>(rec_left),
                                                           static_cast<const double2 *>(rec_right), P, kb, o);
    else
        fixup_kernel<float, float2><<<grid, 256, 0, s>>>(zones, z, static_cast<const float2 *>(rec_left),
                                                         static_cast<const float2 *>(rec_right), P, kb, o);
    return cudaGetLastError();
}

}  // namespace gbk
