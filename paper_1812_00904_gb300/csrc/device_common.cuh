// Device helpers for sm_103a: mbarriers, bulk (TMA) copies, value loads.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gbk {

// Error bits written into the plan's device error word (never a trap).
constexpr int ERR_INDEX = 1;      // an index outside the short vector was met (entry skipped)
constexpr int ERR_WAIT = 2;       // a staging wait ran past its time limit
constexpr int ERR_STRUCT = 4;     // a tile descriptor was inconsistent with the chunk

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy (bulk copy) ones.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One bounded probe of the phase: the thread may be suspended for up to about a
// microsecond (the suspend-time hint) while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, giving up after
// `limit_ns` nanoseconds of global time.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// One-dimensional bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst and src 16-byte aligned, bytes a positive multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// element types

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename AT, typename T> __device__ __forceinline__ AT to_acc(T v) { return static_cast<AT>(to_f<T>(v)); }
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }

template <typename T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return static_cast<float>(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn(static_cast<float>(v));
}
template <> __device__ __forceinline__ __half from_d<__half>(double v) { return __float2half_rn(static_cast<float>(v)); }

// Load 4 consecutive values at element position p (a multiple of 4) of a
// 16-byte aligned shared-memory array into the accumulation type.
template <typename VT, typename AT> struct Load4;
template <> struct Load4<float, float> {
    __device__ __forceinline__ static void run(const void *base, int p, float (&v)[4]) {
        const float4 q = reinterpret_cast<const float4 *>(base)[p >> 2];
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Load4<double, double> {
    __device__ __forceinline__ static void run(const void *base, int p, double (&v)[4]) {
        const double2 a = reinterpret_cast<const double2 *>(base)[(p >> 1)];
        const double2 b = reinterpret_cast<const double2 *>(base)[(p >> 1) + 1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct Load4<__nv_bfloat16, float> {
    __device__ __forceinline__ static void run(const void *base, int p, float (&v)[4]) {
        const uint2 q = reinterpret_cast<const uint2 *>(base)[p >> 2];
        v[0] = __uint_as_float(q.x << 16); v[1] = __uint_as_float(q.x & 0xffff0000u);
        v[2] = __uint_as_float(q.y << 16); v[3] = __uint_as_float(q.y & 0xffff0000u);
    }
};
template <> struct Load4<__half, float> {
    __device__ __forceinline__ static void run(const void *base, int p, float (&v)[4]) {
        const uint2 q = reinterpret_cast<const uint2 *>(base)[p >> 2];
        const __half2 a = *reinterpret_cast<const __half2 *>(&q.x);
        const __half2 b = *reinterpret_cast<const __half2 *>(&q.y);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
    }
};

// Load 8 consecutive values at element position p (a multiple of 8).
template <typename VT, typename AT> struct Load8 {
    __device__ __forceinline__ static void run(const void *base, int p, AT (&v)[8]) {
        AT a[4], b[4];
        Load4<VT, AT>::run(base, p, a);
        Load4<VT, AT>::run(base, p + 4, b);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] = a[e];
            v[e + 4] = b[e];
        }
    }
};
template <> struct Load8<__nv_bfloat16, float> {
    __device__ __forceinline__ static void run(const void *base, int p, float (&v)[8]) {
        const uint4 q = reinterpret_cast<const uint4 *>(base)[p >> 3];
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[2 * e] = __uint_as_float(w[e] << 16);
            v[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
        }
    }
};
template <> struct Load8<__half, float> {
    __device__ __forceinline__ static void run(const void *base, int p, float (&v)[8]) {
        const uint4 q = reinterpret_cast<const uint4 *>(base)[p >> 3];
        const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
            v[2 * e] = f.x;
            v[2 * e + 1] = f.y;
        }
    }
};

// Staggered 8-value loads.  A warp reads 8 consecutive values per lane (32 bytes
// of 4-byte values); lanes whose bit 2 is set read their two 16-byte halves in the
// opposite order, so that each 16-byte load instruction of the warp covers every
// shared-memory bank exactly four times (no two-way bank conflict).  Register e then
// holds position e ^ (4 * sw), sw = (lane >> 2) & 1.
__device__ __forceinline__ void stag8_idx(const int32_t *base, int p, int sw, int (&v)[8]) {
    const int4 *q = reinterpret_cast<const int4 *>(base) + (p >> 2);
    const int4 a = q[sw], b = q[1 - sw];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <typename VT, typename AT> struct Stag8;
template <> struct Stag8<float, float> {
    __device__ __forceinline__ static void run(const void *base, int p, int sw, float (&v)[8]) {
        const float4 *q = reinterpret_cast<const float4 *>(base) + (p >> 2);
        const float4 a = q[sw], b = q[1 - sw];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
};
template <> struct Stag8<double, double> {
    __device__ __forceinline__ static void run(const void *base, int p, int sw, double (&v)[8]) {
        const double2 *q = reinterpret_cast<const double2 *>(base) + (p >> 1);
        const double2 a = q[2 * sw], b = q[2 * sw + 1], c = q[2 - 2 * sw], d = q[3 - 2 * sw];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        v[4] = c.x; v[5] = c.y; v[6] = d.x; v[7] = d.y;
    }
};
template <> struct Stag8<__nv_bfloat16, float> {
    __device__ __forceinline__ static void run(const void *base, int p, int sw, float (&v)[8]) {
        const uint4 q = reinterpret_cast<const uint4 *>(base)[p >> 3];
        const unsigned w[4] = {sw ? q.z : q.x, sw ? q.w : q.y, sw ? q.x : q.z, sw ? q.y : q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[2 * e] = __uint_as_float(w[e] << 16);
            v[2 * e + 1] = __uint_as_float(w[e] & 0xffff0000u);
        }
    }
};
template <> struct Stag8<__half, float> {
    __device__ __forceinline__ static void run(const void *base, int p, int sw, float (&v)[8]) {
        const uint4 q = reinterpret_cast<const uint4 *>(base)[p >> 3];
        const unsigned w[4] = {sw ? q.z : q.x, sw ? q.w : q.y, sw ? q.x : q.z, sw ? q.y : q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[e]));
            v[2 * e] = f.x;
            v[2 * e + 1] = f.y;
        }
    }
};

// Swap the two 4-bit halves of an 8-bit mask when sw is set (position <-> register order).
__device__ __forceinline__ uint32_t rot4(uint32_t m, int sw) {
    return sw ? (((m >> 4) | (m << 4)) & 0xFFu) : m;
}

}  // namespace gbk
