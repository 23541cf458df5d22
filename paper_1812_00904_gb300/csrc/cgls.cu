// Least squares on the device: the normal-equation operator u = A^T (A x) and CGLS
// (conjugate gradients on A^T A x = A^T b).  The paper measures SpMV-SpVTM pairs
// because first-order methods for wide or tall problems are built from them
// (Sec. V); here the SpVTM consumes the SpMV's result.  Every vector operation runs
// in the kernels below; the scalars of the iteration stay in device memory, and the
// host reads them only every few iterations to test convergence.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "plan_impl.h"

namespace gbk {
namespace {

#define CG_TRY(expr)                                                              \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) return set_error(SPMV_ERR_CUDA, cudaGetErrorString(_e)); \
    } while (0)

size_t cg_align(size_t v, size_t a) { return (v + a - 1) / a * a; }
bool cg_aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS = 608;  // fixed: the summation order must not depend on the device

struct CgScalars {
    double gamma, gamma0, delta, alpha, beta;
};

template <typename T> __device__ __forceinline__ void two_sum(T &s, T &c, T v) {
    const T t = s + v;
    const T bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

// Block partial sums of a . b: block g takes elements g, g + G, g + 2G, ... in thread
// order; compensated sums; the block reduces its threads in a fixed tree order.
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) dot_partial_kernel(const T *__restrict__ a, const T *__restrict__ b,
                                                                  int64_t len, double *__restrict__ part) {
    __shared__ T sh_s[DOT_THREADS], sh_c[DOT_THREADS];
    T s = T(0), c = T(0);
    const int64_t stride = (int64_t)gridDim.x * DOT_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < len; i += stride) two_sum(s, c, a[i] * b[i]);
    sh_s[threadIdx.x] = s;
    sh_c[threadIdx.x] = c;
    __syncthreads();
    for (int w = DOT_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            T ss = sh_s[threadIdx.x], cc = sh_c[threadIdx.x];
            two_sum(ss, cc, sh_s[threadIdx.x + w]);
            cc += sh_c[threadIdx.x + w];
            sh_s[threadIdx.x] = ss;
            sh_c[threadIdx.x] = cc;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = (double)sh_s[0] + (double)sh_c[0];
}

// Sum of the block partials (fixed order) and the scalar update of the iteration:
// what = 0: gamma0 = gamma = sum (start); 1: delta = sum, alpha = gamma / delta;
// 2: beta = sum / gamma, gamma = sum.
__global__ void __launch_bounds__(32) dot_final_kernel(const double *__restrict__ part, int nparts, int what,
                                                       CgScalars *sc) {
    double s = 0.0;
    for (int q = threadIdx.x; q < nparts; q += 32) s += part[q];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (threadIdx.x == 0) {
        if (what == 0) {
            sc->gamma = sc->gamma0 = s;
        } else if (what == 1) {
            sc->delta = s;
            sc->alpha = s > 0.0 ? sc->gamma / s : 0.0;
        } else {
            sc->beta = sc->gamma > 0.0 ? s / sc->gamma : 0.0;
            sc->gamma = s;
        }
    }
}

// x += alpha p (n entries), r -= alpha q (m entries)
template <typename T>
__global__ void xr_update_kernel(T *__restrict__ x, const T *__restrict__ p, int64_t n, T *__restrict__ r,
                                 const T *__restrict__ q, int64_t m, const CgScalars *sc) {
    const T alpha = (T)sc->alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t len = n > m ? n : m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        if (i < n) x[i] += alpha * p[i];
        if (i < m) r[i] -= alpha * q[i];
    }
}

// p = s + beta p (beta = 0 copies)
template <typename T>
__global__ void p_update_kernel(T *__restrict__ p, const T *__restrict__ s, int64_t n, const CgScalars *sc,
                                int first) {
    const T beta = first ? T(0) : (T)sc->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = first ? s[i] : s[i] + beta * p[i];
}

// r = b - r
template <typename T>
__global__ void residual_kernel(const T *__restrict__ b, T *__restrict__ r, int64_t m) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) r[i] = b[i] - r[i];
}

template <typename T> struct Cgls {
    spmv_plan_s *p;
    cudaStream_t s;
    int grid;
    T *r = nullptr, *sv = nullptr, *pv = nullptr, *q = nullptr;
    double *part = nullptr;
    CgScalars *sc = nullptr;

    cudaError_t dot(const T *a, const T *b, int64_t len, int what) {
        dot_partial_kernel<T><<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(a, b, len, part);
        dot_final_kernel<<<1, 32, 0, s>>>(part, DOT_BLOCKS, what, sc);
        return cudaGetLastError();
    }

    spmv_status run(const T *bvec, T *x, int max_iters, double tol, int32_t *iters_done, double *rel) {
        const int64_t m = p->m, n = p->n;
        const T *cin = x;
        void *cout = r;
        spmv_status st = run_op(p, SPMV_OP_AX, 1, reinterpret_cast<const void *const *>(&cin), &cout, s);
        if (st != SPMV_OK) return st;
        residual_kernel<T><<<grid, 256, 0, s>>>(bvec, r, m);
        const T *rin = r;
        void *sout = sv;
        if ((st = run_op(p, SPMV_OP_VTA, 1, reinterpret_cast<const void *const *>(&rin), &sout, s)) != SPMV_OK)
            return st;
        CG_TRY(dot(sv, sv, n, 0));
        p_update_kernel<T><<<grid, 256, 0, s>>>(pv, sv, n, sc, 1);
        CgScalars h{};
        int it = 0;
        while (it < max_iters) {
            const T *pin = pv;
            void *qout = q;
            if ((st = run_op(p, SPMV_OP_AX, 1, reinterpret_cast<const void *const *>(&pin), &qout, s)) != SPMV_OK)
                return st;
            CG_TRY(dot(q, q, m, 1));
            xr_update_kernel<T><<<grid, 256, 0, s>>>(x, pv, n, r, q, m, sc);
            if ((st = run_op(p, SPMV_OP_VTA, 1, reinterpret_cast<const void *const *>(&rin), &sout, s)) != SPMV_OK)
                return st;
            CG_TRY(dot(sv, sv, n, 2));
            p_update_kernel<T><<<grid, 256, 0, s>>>(pv, sv, n, sc, 0);
            CG_TRY(cudaGetLastError());
            ++it;
            if (it % 8 == 0 || it == max_iters) {  // convergence test on the host
                CG_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
                CG_TRY(cudaStreamSynchronize(s));
                if (!(h.gamma0 > 0.0) || std::sqrt(h.gamma / h.gamma0) <= tol) break;
            }
        }
        CG_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
        CG_TRY(cudaStreamSynchronize(s));
        if (iters_done) *iters_done = it;
        if (rel) *rel = h.gamma0 > 0.0 ? std::sqrt(h.gamma / h.gamma0) : 0.0;
        return SPMV_OK;
    }
};

template <typename T>
spmv_status cgls_typed(spmv_plan_s *p, const void *b, void *x, int max_iters, double tol, cudaStream_t s,
                       int32_t *iters_done, double *rel) {
    Cgls<T> c{p, s, 0};
    int sms = 0;
    CG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    c.grid = std::max(1, sms * 4);
    const size_t m = (size_t)std::max<int64_t>(p->m, 1), n = (size_t)std::max<int64_t>(p->n, 1);
    char *mem = nullptr;
    const size_t off_s = cg_align(m * sizeof(T), 256), off_p = off_s + cg_align(n * sizeof(T), 256);
    const size_t off_q = off_p + cg_align(n * sizeof(T), 256), off_part = off_q + cg_align(m * sizeof(T), 256);
    const size_t off_sc = off_part + cg_align(DOT_BLOCKS * sizeof(double), 256);
    const size_t total = off_sc + sizeof(CgScalars);
    CG_TRY(cudaMalloc(&mem, total));
    c.r = reinterpret_cast<T *>(mem);
    c.sv = reinterpret_cast<T *>(mem + off_s);
    c.pv = reinterpret_cast<T *>(mem + off_p);
    c.q = reinterpret_cast<T *>(mem + off_q);
    c.part = reinterpret_cast<double *>(mem + off_part);
    c.sc = reinterpret_cast<CgScalars *>(mem + off_sc);
    cudaError_t e = cudaMemsetAsync(c.sc, 0, sizeof(CgScalars), s);
    spmv_status st = e == cudaSuccess ? c.run(static_cast<const T *>(b), static_cast<T *>(x), max_iters, tol, iters_done,
                                               rel)
                                      : set_error(SPMV_ERR_CUDA, cudaGetErrorString(e));
    cudaStreamSynchronize(s);
    cudaFree(mem);
    return st;
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" {

spmv_status spmv_normal(spmv_plan_t p, const void *x, void *u, void *y, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    if (!x || !u) return set_error(SPMV_ERR_INVALID_ARG, "null vector");
    if (!cg_aligned16(x) || !cg_aligned16(u) || !cg_aligned16(y))
        return set_error(SPMV_ERR_INVALID_ARG, "vectors must be 16-byte aligned device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *yb = y;
    if (!yb) {
        std::lock_guard<std::mutex> lk(p->host_mu);
        if (!p->ynorm) CG_TRY(cudaMalloc(&p->ynorm, (size_t)std::max<int64_t>(p->m, 1) * p->sx + 16));
        yb = p->ynorm;
    }
    const void *xin = x;
    spmv_status st = run_op(p, SPMV_OP_AX, 1, &xin, &yb, s);
    if (st != SPMV_OK) return st;
    const void *yin = yb;
    return run_op(p, SPMV_OP_VTA, 1, &yin, &u, s);
}

spmv_status spmv_cgls(spmv_plan_t p, const void *b, void *x, int32_t max_iters, double tol, void *stream,
                      int32_t *iters_done, double *rel_grad) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    if (!b || !x) return set_error(SPMV_ERR_INVALID_ARG, "null vector");
    if (!cg_aligned16(b) || !cg_aligned16(x))
        return set_error(SPMV_ERR_INVALID_ARG, "vectors must be 16-byte aligned device memory");
    if (max_iters < 0 || !(tol >= 0.0)) return set_error(SPMV_ERR_INVALID_ARG, "max_iters >= 0 and tol >= 0 required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->vec_t == SPMV_F64) return cgls_typed<double>(p, b, x, max_iters, tol, s, iters_done, rel_grad);
    return cgls_typed<float>(p, b, x, max_iters, tol, s, iters_done, rel_grad);
}

}  // extern "C"
