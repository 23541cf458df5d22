// C ABI of libspmv_gb300 (declared in include/spmv_gb300.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "plan_impl.h"

using namespace gbk;

namespace {

thread_local std::string g_last_error;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int dtype_size(int t) {
    switch (t) {
        case SPMV_F64: return 8;
        case SPMV_F32: return 4;
        case SPMV_BF16: return 2;
        case SPMV_F16: return 2;
        default: return 0;
    }
}

bool pair_supported(int vt, int xt) {
    return (vt == SPMV_F64 && xt == SPMV_F64) || (vt == SPMV_F32 && xt == SPMV_F32) ||
           (vt == SPMV_BF16 && xt == SPMV_F32) || (vt == SPMV_F16 && xt == SPMV_F32);
}

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return set_error(_e == cudaErrorMemoryAllocation ? SPMV_ERR_OOM : SPMV_ERR_CUDA,        \
                             std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
    } while (0)

cudaError_t launch_stream(const spmv_plan_s *p, int mode, int kb, const LaunchArgs &a) {
    switch (p->val_t) {
        case SPMV_F64: return launch_stream_f64(mode, kb, a);
        case SPMV_F32: return launch_stream_f32(mode, kb, a);
        case SPMV_BF16: return launch_stream_bf16(mode, kb, a);
        default: return launch_stream_f16(mode, kb, a);
    }
}

int kb_template(int kb) { return kb <= 1 ? 1 : kb <= 2 ? 2 : kb <= 4 ? 4 : 8; }

// Tiles per chunk of the streaming kernels (default): a warp carries a segment across the
// tiles of a chunk in registers, so overlap zones (and their FP64 fix-up) arise only at chunk
// boundaries, while the CTA's warps still stream a compact stretch of the arrays.
constexpr int CHUNK_TILES = 8;

// Kernel timers: bracket one launch with events when the plan profiles.
struct ProfScope {
    spmv_plan_s *p;
    int kernel;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(spmv_plan_s *p_, int k, cudaStream_t s_) : p(p_), kernel(k), s(s_) {
        if (p->prof_on.load(std::memory_order_relaxed)) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEventRecord(b, s);
            std::lock_guard<std::mutex> lk(p->prof_mu);
            p->prof.push_back({kernel, a, b});
        }
    }
};

StreamParams base_params(const spmv_plan_s *p) {
    StreamParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.idx = p->idx;
    sp.vals = p->vals;
    sp.pptr = p->pptr;
    sp.nnz = (int)p->nnz;
    sp.n_major = p->n_major;
    sp.n_minor = p->n_minor;
    sp.meta = p->meta;
    sp.masks = p->masks;
    sp.ntiles = p->ntiles;
    sp.mwp = p->mwp;
    sp.pfx = p->pfx;
    sp.mwq = p->mwq;
    sp.slots = p->S;
    sp.x_cap = p->x_cap;
    sp.tile_cap = p->T;
    sp.checked = (p->flags & SPMV_PLAN_NO_VALIDATE) ? 1 : 0;
    sp.rec_left = p->rec_left;
    sp.rec_right = p->rec_right;
    sp.chunk_tiles = p->chunk_tiles;
    sp.blocks_per_cta = p->bpc;
    sp.win = p->win;
    sp.err = p->err;
    return sp;
}

// Layout of one warp's staging slot: indices, values, segment-start masks and, for
// the scatter and gradient modes, the long-vector windows (16-byte aligned).
struct SlotGeom {
    int off_val, off_mask, off_x, off_hdr, bytes;
};
SlotGeom slot_geom(const spmv_plan_s *p, int mode, int kbt) {
    SlotGeom g;
    g.off_val = (int)align_up((size_t)p->T * 4, 128);
    g.off_mask = g.off_val + (int)align_up((size_t)p->T * p->sv, 128);
    g.off_x = g.off_mask + (int)align_up((size_t)p->mwp * 4, 16);
    const bool seg = mode == MODE_SEGDOT || mode == MODE_VSEG;
    const int nx = seg ? 0 : mode == MODE_DVALUES ? 1 : kbt;
    // the segmented modes stage the tile's head-count prefix table where the others stage windows
    const size_t xbytes = seg ? align_up((size_t)p->mwq * 2, 16) : (size_t)nx * p->x_cap * p->sx;
    g.off_hdr = (int)align_up((size_t)g.off_x + xbytes, 16);  // 32-byte tile header
    g.bytes = (int)align_up((size_t)g.off_hdr + 32, 128);
    return g;
}
// On-chip short-vector bytes of a pass (accumulator of the scatter mode, input otherwise).
size_t vec_bytes(const spmv_plan_s *p, int mode, int kbt, bool smemv) {
    if (mode == MODE_VSEG)  // 8 values of scratch per lane, then the interleaved vectors when on chip
        return (size_t)WARPS_VSEG * 32 * 8 * 4 + (smemv ? align_up((size_t)p->n_minor * kbt * p->sx, 128) : 0);
    if (!smemv) return 0;
    const size_t e = mode == MODE_SCATTER ? (size_t)p->sa : (size_t)p->sx;
    return align_up((size_t)p->n_minor * kbt * e, 128);
}
// Warps per CTA of a pass: the plan's warps, as many as the shared memory holds.
int warps_for(const spmv_plan_s *p, int mode, int kbt, bool smemv) {
    const size_t vec = vec_bytes(p, mode, kbt, smemv);
    const SlotGeom g = slot_geom(p, mode, kbt);
    const size_t room = (size_t)p->smem_max > vec + BAR_BYTES ? (size_t)p->smem_max - vec - BAR_BYTES : 0;
    const int fit = (int)std::min<size_t>(room / ((size_t)p->S * g.bytes), 64);
    const int w = std::min({p->W, mode == MODE_VSEG ? WARPS_VSEG : kbt > 1 ? MAX_WARPS_KB : MAX_WARPS, fit});
    // one warp beyond WARPS_REGS costs the others their larger register budget: not worth it
    return w == WARPS_REGS + 1 ? WARPS_REGS : w;
}

int warps_for(const spmv_plan_s *p, int mode, int kbt) { return warps_for(p, mode, kbt, p->onchip); }

// Launch geometry of one streaming pass (the short vector on chip when smemv).
void set_geometry(const spmv_plan_s *p, LaunchArgs &a, int mode, int kbt, bool smemv) {
    const SlotGeom g = slot_geom(p, mode, kbt);
    const int W = std::max(1, warps_for(p, mode, kbt, smemv));
    a.smemv = smemv;
    a.sp.vec_region_bytes = (int)vec_bytes(p, mode, kbt, smemv);
    a.sp.slot_bytes = g.bytes;
    a.sp.off_val = g.off_val;
    a.sp.off_mask = g.off_mask;
    a.sp.off_x = g.off_x;
    a.sp.off_pfx = g.off_x;
    a.sp.off_hdr = g.off_hdr;
    a.smem = a.sp.vec_region_bytes + BAR_BYTES + W * p->S * g.bytes;
    a.grid = p->ctas;
    a.block = W * 32;
}

enum PtrKind { PK_DEVICE, PK_HOST, PK_BAD };

PtrKind classify(const void *ptr) {
    if (!ptr) return PK_BAD;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PK_HOST;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return PK_DEVICE;
    return PK_HOST;
}

}  // namespace

namespace gbk {

spmv_status set_error(spmv_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

size_t plan_footprint(const spmv_plan_s *p) {
    size_t b = p->ws_bytes + p->owned_bytes + (size_t)p->nnz * (4 + p->sv) + (size_t)(p->n_major + 1) * 4;
    if (p->tplan) b += p->tplan->ws_bytes + p->tplan->owned_bytes + p->bws_bytes + p->bown_bytes;
    return b;
}

spmv_status run_scatter(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s) {
    const size_t out_bytes = (size_t)p->n_minor * p->sx;
    if (p->nnz == 0 || p->n_major == 0) {
        if (out_bytes)
            for (int b = 0; b < kb; ++b) CUDA_TRY(cudaMemsetAsync(out[b], 0, out_bytes, s));
        return SPMV_OK;
    }
    if (!p->onchip && kb > 1) {
        for (int b = 0; b < kb; ++b) {
            spmv_status st = run_scatter(p, 1, in + b, out + b, s);
            if (st != SPMV_OK) return st;
        }
        return SPMV_OK;
    }
    LaunchArgs a;
    a.sp = base_params(p);
    a.sp.kb = kb;
    for (int b = 0; b < kb; ++b) a.sp.vin[b] = in[b];
    set_geometry(p, a, MODE_SCATTER, kb_template(kb), p->onchip);
    a.sp.part = p->part;
    if (!p->onchip) CUDA_TRY(cudaMemsetAsync(p->part, 0, (size_t)p->n_minor * sizeof(double), s));
    a.stream = s;
    {
        ProfScope ps(p, 0, s);
        CUDA_TRY(launch_stream(p, MODE_SCATTER, kb, a));
    }
    {
        ProfScope ps(p, 1, s);
        const bool f64 = p->vec_t == SPMV_F64;
        CUDA_TRY(launch_combine(f64, f64 || !p->onchip, p->part, p->onchip ? p->ctas : 1, p->n_minor, kb, out, s));
    }
    return SPMV_OK;
}

// The plan's buffer vt holding kb input vectors interleaved with stride kbt (in_len entries
// each: the short vector, or the long vector of a row-sorted copy's windows).
static spmv_status interleave_inputs(spmv_plan_s *p, int kbt, int kb, const void *const *in, int64_t len,
                                     cudaStream_t s) {
    const size_t need = (size_t)std::max<int64_t>(len, 1) * std::max(KB_MAX, VL_MAX) * p->sx;
    if (p->vt_bytes < need) {
        if (p->vt) cudaFree(p->vt);
        p->vt = nullptr;
        p->vt_bytes = 0;
        CUDA_TRY(cudaMalloc(&p->vt, need));
        p->vt_bytes = need;
    }
    CUDA_TRY(launch_interleave(p->vec_t == SPMV_F64, kbt, kb, in, len, p->vt, s));
    return SPMV_OK;
}

// Several vectors of a segmented pass in one streaming of the nonzeros, read from the
// interleaved copy vt through L2: FP64 with MODE_SEGDOT (2..KB_MAX vectors), the other value
// types with MODE_VSEG (2..VL_MAX vectors, one per lane of a lane group).  Either way every
// vector's sums are formed exactly as in its single-vector pass.
static spmv_status run_segdot_global(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s,
                                     spmv_plan_s *prof, int id_dot, int id_fix, int64_t in_len) {
    const bool vseg = p->val_t != SPMV_F64;
    const int mode = vseg ? MODE_VSEG : MODE_SEGDOT;
    const int kbt = vseg ? (kb <= 4 ? 4 : 8) : kb_template(kb);
    // VSEG stages the interleaved vectors (or each block's window of them) when they leave room
    // for half of its warps
    const bool smemv = vseg && warps_for(p, MODE_VSEG, kbt, true) >= std::min(p->W, WARPS_VSEG) / 2;
    spmv_status st = interleave_inputs(p, kbt, kb, in, in_len >= 0 ? in_len : p->n_minor, s);
    if (st != SPMV_OK) return st;
    LaunchArgs a;
    a.sp = base_params(p);
    a.sp.kb = kb;
    a.sp.vin[0] = p->vt;
    for (int b = 0; b < kb; ++b) a.sp.vout[b] = out[b];
    set_geometry(p, a, mode, kbt, smemv);
    const spmv_plan_s::ProcZones &pz = p->pz;
    a.sp.nproc = pz.nproc;
    a.stream = s;
    {
        ProfScope ps(prof, id_dot, s);
        CUDA_TRY(launch_stream(p, mode, kb, a));
    }
    if (pz.z > 0) {
        ProfScope ps(prof, id_fix, s);
        CUDA_TRY(launch_fixup(p->vec_t == SPMV_F64, pz.zones, pz.z, p->rec_left, p->rec_right, pz.nproc, kb, out, s));
    }
    return SPMV_OK;
}

// Vectors per pass of a plan's multi-vector segmented passes.
static int seg_group(const spmv_plan_s *p) { return p->val_t == SPMV_F64 ? KB_MAX : VL_MAX; }

// The segmented pass (and its zone fix-up) of plan p; the launches are timed as kernels
// id_dot / id_fix of plan `prof`.  One vector runs with the short vector on chip when it fits;
// several run through run_segdot_global (FP64: on chip instead while batch_width holds them),
// seg_group(p) per pass.
static spmv_status run_segdot_impl(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s,
                                   spmv_plan_s *prof, int id_dot, int id_fix, int64_t in_len) {
    const size_t out_bytes = (size_t)p->n_major * p->sx;
    if (p->nnz == 0 || p->n_minor == 0) {
        if (out_bytes)
            for (int b = 0; b < kb; ++b) CUDA_TRY(cudaMemsetAsync(out[b], 0, out_bytes, s));
        return SPMV_OK;
    }
    const bool f64_onchip = p->val_t == SPMV_F64 && p->onchip && kb <= p->batch_width;
    if (kb > 1 && !f64_onchip) {
        const int grp = seg_group(p);
        for (int g0 = 0; g0 < kb; g0 += grp) {
            const int kg = std::min(grp, kb - g0);
            spmv_status st = kg == 1 ? run_segdot_impl(p, 1, in + g0, out + g0, s, prof, id_dot, id_fix, in_len)
                                     : run_segdot_global(p, kg, in + g0, out + g0, s, prof, id_dot, id_fix, in_len);
            if (st != SPMV_OK) return st;
        }
        return SPMV_OK;
    }
    LaunchArgs a;
    a.sp = base_params(p);
    a.sp.kb = kb;
    for (int b = 0; b < kb; ++b) {
        a.sp.vin[b] = in[b];
        a.sp.vout[b] = out[b];
    }
    set_geometry(p, a, MODE_SEGDOT, kb_template(kb), p->onchip);
    const spmv_plan_s::ProcZones &pz = p->pz;
    a.sp.nproc = pz.nproc;
    a.stream = s;
    {
        ProfScope ps(prof, id_dot, s);
        CUDA_TRY(launch_stream(p, MODE_SEGDOT, kb, a));
    }
    if (pz.z > 0) {
        ProfScope ps(prof, id_fix, s);
        CUDA_TRY(launch_fixup(p->vec_t == SPMV_F64, pz.zones, pz.z, p->rec_left, p->rec_right, pz.nproc, kb, out, s));
    }
    return SPMV_OK;
}

spmv_status run_segdot(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s) {
    const int grp = seg_group(p);
    for (int g0 = 0; g0 < kb; g0 += grp) {
        const int kg = std::min(grp, kb - g0);
        spmv_status st = run_segdot_impl(p, kg, in + g0, out + g0, s, p, 2, 3, -1);
        if (st != SPMV_OK) return st;
    }
    return SPMV_OK;
}

// The short-vector product over the row-sorted blocks (SPMV_PLAN_ROW_BLOCKS): the sub-plan's
// windowed segmented pass writes every block's short vector into ypart (its fix-up completes
// the entries split between chunks), then the blocks' vectors are added in FP64 in block
// order (Sec. III step 2).  One vector runs with its windows on chip; several (seg_group per
// pass) read their windows through L2 from an interleaved copy of the long vectors, into
// per-block vectors [vector][block][n_minor] (a plan-owned buffer made on first use).
static spmv_status run_row_blocks(spmv_plan_s *p, int kb, const void *const *in, void *const *out, cudaStream_t s) {
    spmv_plan_s *q = p->tplan;
    const bool f64 = p->vec_t == SPMV_F64;
    const size_t nseg = (size_t)p->blocks * p->n_minor;
    const int grp = seg_group(q);
    for (int g0 = 0; g0 < kb; g0 += grp) {
        const int kg = std::min(grp, kb - g0);
        void *yp[VL_MAX];
        void *base = p->ypart;
        if (kg > 1) {
            const size_t need = nseg * grp * p->sx;
            if (p->ypart_k_bytes < need) {
                if (p->ypart_k) cudaFree(p->ypart_k);
                p->ypart_k = nullptr;
                p->ypart_k_bytes = 0;
                CUDA_TRY(cudaMalloc(&p->ypart_k, need));
                p->ypart_k_bytes = need;
            }
            base = p->ypart_k;
        }
        for (int b = 0; b < kg; ++b) yp[b] = static_cast<char *>(base) + (size_t)b * nseg * p->sx;
        spmv_status st = run_segdot_impl(q, kg, in + g0, yp, s, p, 5, 6, p->n_major);
        if (st != SPMV_OK) return st;
        ProfScope ps(p, 1, s);
        CUDA_TRY(launch_combine(f64, f64, base, p->blocks, p->n_minor, kg, out + g0, s, (size_t)p->n_minor, nseg));
    }
    return SPMV_OK;
}

static spmv_status run_dvalues(spmv_plan_s *p, const void *r, const void *x, void *g, cudaStream_t s) {
    if (p->nnz == 0) return SPMV_OK;
    LaunchArgs a;
    a.sp = base_params(p);
    a.sp.kb = 1;
    // CSC: g = r[row] * x[col] -> minor r, major x;  CSR: g = r[row] * x[col] -> minor x, major r
    const bool csc = p->layout == SPMV_CSC_WIDE;
    a.sp.vin[0] = csc ? r : x;
    a.sp.vin[1] = csc ? x : r;
    a.sp.vout[0] = g;
    set_geometry(p, a, MODE_DVALUES, 1, p->onchip);
    a.stream = s;
    ProfScope ps(p, 4, s);
    CUDA_TRY(launch_stream(p, MODE_DVALUES, 1, a));
    return SPMV_OK;
}

spmv_status run_op(spmv_plan_s *p, int op, int k, const void *const *in, void *const *out, cudaStream_t s) {
    const bool scatter = (op == SPMV_OP_AX) == (p->layout == SPMV_CSC_WIDE);
    if (scatter && p->tplan && p->nnz > 0) return run_row_blocks(p, k, in, out, s);
    if (!scatter) return run_segdot(p, k, in, out, s);
    for (int g0 = 0; g0 < k; g0 += p->batch_width) {
        const int kb = std::min(p->batch_width, k - g0);
        spmv_status st = run_scatter(p, kb, in + g0, out + g0, s);
        if (st != SPMV_OK) return st;
    }
    return SPMV_OK;
}

}  // namespace gbk

namespace gbk {

void plan_free(spmv_plan_s *p) {
    if (!p) return;
    plan_free(p->tplan);
    if (p->vt) cudaFree(p->vt);
    if (p->ypart_k) cudaFree(p->ypart_k);
    if (p->bws) cudaFree(p->bws);
    if (p->bown) cudaFree(p->bown);
    for (auto &pr : p->prof) {
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    if (p->ws) cudaFree(p->ws);
    if (p->ws2) cudaFree(p->ws2);
    if (p->hin) cudaFree(p->hin);
    if (p->hout) cudaFree(p->hout);
    if (p->hv) cudaFree(p->hv);
    if (p->hu) cudaFree(p->hu);
    if (p->ev_x) cudaEventDestroy(p->ev_x);
    if (p->ev_u) cudaEventDestroy(p->ev_u);
    if (p->cstream) cudaStreamDestroy(p->cstream);
    if (p->hg) cudaFree(p->hg);
    if (p->ynorm) cudaFree(p->ynorm);
    if (p->owned_ptr) cudaFree(p->owned_ptr);
    if (p->owned_nz) cudaFree(p->owned_nz);
    delete p;
}

}  // namespace gbk

namespace {

struct PlanGuard {
    spmv_plan_s *p;
    ~PlanGuard() { plan_free(p); }
};

// Runs `fn` on device pointers, staging host pointers through plan buffers.
template <typename Fn>
spmv_status with_staging(spmv_plan_s *p, const void *in, size_t in_bytes, void *out, size_t out_bytes,
                         cudaStream_t s, Fn fn) {
    // an empty vector may be NULL (torch gives zero-size tensors a null address)
    const PtrKind ki = (in_bytes == 0 && !in) ? PK_DEVICE : classify(in);
    const PtrKind ko = (out_bytes == 0 && !out) ? PK_DEVICE : classify(out);
    if (ki == PK_BAD || ko == PK_BAD) return set_error(SPMV_ERR_INVALID_ARG, "null vector pointer");
    if (ki == PK_DEVICE && ko == PK_DEVICE) {
        if ((in && !aligned16(in)) || (out && !aligned16(out)))
            return set_error(SPMV_ERR_INVALID_ARG, "device vector pointers must be 16-byte aligned");
        return fn(in, out);
    }
    std::lock_guard<std::mutex> lk(p->host_mu);
    const size_t cap = (size_t)std::max(p->m, p->n) * p->sx + 16;
    if (!p->hin) CUDA_TRY(cudaMalloc(&p->hin, cap));
    if (!p->hout) CUDA_TRY(cudaMalloc(&p->hout, cap));
    const void *din = in;
    void *dout = out;
    if (ki == PK_HOST) {
        CUDA_TRY(cudaMemcpyAsync(p->hin, in, in_bytes, cudaMemcpyHostToDevice, s));
        din = p->hin;
    } else if (!aligned16(in)) {
        return set_error(SPMV_ERR_INVALID_ARG, "device vector pointers must be 16-byte aligned");
    }
    if (ko == PK_HOST) dout = p->hout;
    spmv_status st = fn(din, dout);
    if (st != SPMV_OK) return st;
    if (ko == PK_HOST) CUDA_TRY(cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace

extern "C" {

const char *spmv_last_error(void) { return g_last_error.c_str(); }

const char *spmv_version(void) { return "spmv_gb300 0.1 (sm_103a)"; }

spmv_status spmv_plan(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout, const int32_t *ptr,
                      const int32_t *idx, const void *vals, int32_t val_dtype, int32_t vec_dtype, void *stream,
                      uint32_t flags) {
    return spmv_plan_ex(out, m, n, nnz, layout, ptr, idx, vals, val_dtype, vec_dtype, stream, flags, nullptr);
}

spmv_status spmv_plan_ex(spmv_plan_t *out, int64_t m, int64_t n, int64_t nnz, int32_t layout, const int32_t *ptr,
                         const int32_t *idx, const void *vals, int32_t val_dtype, int32_t vec_dtype, void *stream,
                         uint32_t flags, const spmv_plan_opts *opts) {
    g_last_error.clear();
    return plan_create(out, m, n, nnz, layout, ptr, idx, vals, val_dtype, vec_dtype, static_cast<cudaStream_t>(stream),
                       flags, opts, nullptr);
}

}  // extern "C"

spmv_status gbk::plan_create(spmv_plan_s **out, int64_t m, int64_t n, int64_t nnz, int32_t layout, const int32_t *ptr,
                             const int32_t *idx, const void *vals, int32_t val_dtype, int32_t vec_dtype,
                             cudaStream_t s, uint32_t flags, const spmv_plan_opts *opts, const PlanInternal *pi) {
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (layout != SPMV_CSC_WIDE && layout != SPMV_CSR_TALL) return set_error(SPMV_ERR_INVALID_ARG, "bad layout");
    if (m < 0 || n < 0 || nnz < 0 || m >= (1ll << 31) - 64 || n >= (1ll << 31) - 64 || nnz >= (1ll << 31) - 64)
        return set_error(SPMV_ERR_INVALID_ARG, "m, n and nnz must lie in [0, 2^31 - 64)");
    if (dtype_size(val_dtype) == 0 || dtype_size(vec_dtype) == 0)
        return set_error(SPMV_ERR_INVALID_ARG, "unknown dtype");
    if (!pair_supported(val_dtype, vec_dtype))
        return set_error(SPMV_ERR_UNSUPPORTED, "supported (values, vectors): (f64,f64) (f32,f32) (bf16,f32) (f16,f32)");
    if (!ptr) return set_error(SPMV_ERR_INVALID_ARG, "ptr is NULL");
    if (nnz > 0 && (!idx || !vals)) return set_error(SPMV_ERR_INVALID_ARG, "idx/vals are NULL");
    if (nnz > 0 && (layout == SPMV_CSC_WIDE ? m : n) == 0)
        return set_error(SPMV_ERR_BAD_MATRIX, "nonzeros need a nonempty indexed dimension");
    if (!aligned16(ptr) || (nnz > 0 && (!aligned16(idx) || !aligned16(vals))))
        return set_error(SPMV_ERR_INVALID_ARG, "ptr, idx and vals must be 16-byte aligned device pointers");
    for (const void *q : {(const void *)ptr, (const void *)idx, vals}) {
        if (q && classify(q) != PK_DEVICE)
            return set_error(SPMV_ERR_INVALID_ARG, "ptr, idx and vals must be device pointers");
    }
    spmv_plan_s *p = new (std::nothrow) spmv_plan_s();
    if (!p) return set_error(SPMV_ERR_OOM, "host allocation failed");
    PlanGuard guard{p};
    CUDA_TRY(cudaGetDevice(&p->device));
    p->m = m;
    p->n = n;
    p->nnz = nnz;
    p->layout = layout;
    p->val_t = val_dtype;
    p->vec_t = vec_dtype;
    p->flags = flags;
    p->prof_on = (flags & SPMV_PLAN_PROFILE) != 0;
    p->n_major = (int)(layout == SPMV_CSC_WIDE ? n : m);
    p->n_minor = (int)(layout == SPMV_CSC_WIDE ? m : n);
    p->ptr = ptr;
    p->idx = idx;
    p->vals = vals;
    p->sv = dtype_size(val_dtype);
    p->sx = dtype_size(vec_dtype);
    p->sa = (val_dtype == SPMV_F64) ? 8 : 4;

    int sms = 0, smem_max = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    smem_max -= 1024;  // static shared memory and slack

    // ---- launch configuration: tiles of T nonzeros, up to W warps per CTA, S staging slots per warp
    // default tile: 512 nonzeros (two whole 256-position steps); smaller when the matrix has
    // too few nonzeros to give every warp of a full wave about two tiles
    p->T = 512;
    if (opts && opts->tile_items) {
        p->T = opts->tile_items;
    } else {
        const int64_t fill = (int64_t)sms * 16 * 2;
        if (nnz < fill * 512) p->T = (int)std::max<int64_t>(64, std::min<int64_t>(512, (nnz / fill) & ~int64_t(7)));
    }
    p->S = (opts && opts->stages) ? opts->stages : 2;
    int W = (opts && opts->warps_per_cta) ? opts->warps_per_cta : MAX_WARPS;
    if (p->T < 8 || p->T > 992 || (p->T % 8) != 0)
        return set_error(SPMV_ERR_INVALID_ARG, "tile_items must be a multiple of 8 in [8, 992]");
    if (p->S < 2 || p->S > MAX_STAGES) return set_error(SPMV_ERR_INVALID_ARG, "stages must lie in [2, 4]");
    if (W < 1 || W > MAX_WARPS) return set_error(SPMV_ERR_INVALID_ARG, "warps_per_cta must lie in [1, 24]");
    if (opts && (opts->chunk_tiles < 0 || opts->chunk_tiles > 64))
        return set_error(SPMV_ERR_INVALID_ARG, "chunk_tiles must lie in [0, 64]");
    p->mwp = (int)align_up((size_t)(p->T + 8 + 31) / 32, 4);
    // prefix entries: one per mask word and the total, and at least one per word a step reads
    p->mwq = (int)align_up((size_t)std::max(p->mwp + 1, 8 * ((p->T + 255) / 256)), 8);
    p->x_cap = (int)align_up((size_t)p->T / 4 + 16, 8);  // columns of a tile's window (fall back to global beyond)
    p->smem_max = smem_max;
    p->W = W;
    // the short vector on chip when it leaves room for at least 4 warps of the scatter pass
    p->onchip = !(flags & SPMV_PLAN_SHORT_IN_GLOBAL);
    if (p->onchip && warps_for(p, MODE_SCATTER, 1) < std::min(W, 4)) p->onchip = false;
    for (int mode : {MODE_SCATTER, MODE_SEGDOT, MODE_DVALUES})
        if (warps_for(p, mode, 1) < 1) return set_error(SPMV_ERR_INVALID_ARG, "tile_items/stages leave no room for one warp");
    // vectors per pass of spmv_batch: as many as still leave most of the warps
    p->batch_width = 1;
    if (p->onchip && !(pi && pi->segdot_only)) {
        const int want = std::min(warps_for(p, MODE_SCATTER, 1), 12);
        for (int kb : {8, 4, 2}) {
            if (warps_for(p, MODE_SCATTER, kb) >= want && warps_for(p, MODE_SEGDOT, kb) >= want) {
                p->batch_width = kb;
                break;
            }
        }
    }
    p->W_info = warps_for(p, MODE_SCATTER, 1);
    // reporting chunks: the paper's P (default: one per warp of a full GPU wave); execution
    // tiles: T consecutive nonzeros each, every tile a processor of the kernels
    const int64_t nt64 = (nnz + p->T - 1) / p->T;
    if (nt64 > (1 << 26)) return set_error(SPMV_ERR_INVALID_ARG, "too many tiles");
    p->P = (opts && opts->chunks > 0) ? opts->chunks : (int)std::max<int64_t>(1, std::min<int64_t>(nt64, (int64_t)sms * 16));
    if (p->P > (1 << 24)) return set_error(SPMV_ERR_INVALID_ARG, "too many chunks");
    {
        const int64_t q = nnz / p->P;
        p->max_chunk = q + (nnz % p->P ? 1 : 0);
        p->min_chunk = q;
    }

    // ---- workspace, part 1: pointer copy, reporting chunks, counters
    p->pptr_len = (int)align_up((size_t)p->n_major + 1 + 8, 4);
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    const size_t o_pptr = carve((size_t)p->pptr_len * 4);
    const size_t o_aux = carve((size_t)p->P * sizeof(ChunkAux));
    const size_t o_chunks = carve((size_t)p->P * sizeof(ChunkDev));
    const size_t o_zones = carve((size_t)p->P * sizeof(ZoneDev));
    const size_t o_counts = carve(128);
    const size_t o_sscr = carve(setup_scratch_bytes(p->P));
    const size_t o_err = carve(16);
    const size_t ws1 = off;
    CUDA_TRY(cudaMalloc(&p->ws, ws1));
    char *w1 = static_cast<char *>(p->ws);
    p->pptr = reinterpret_cast<int32_t *>(w1 + o_pptr);
    p->aux = reinterpret_cast<ChunkAux *>(w1 + o_aux);
    p->chunks = reinterpret_cast<ChunkDev *>(w1 + o_chunks);
    p->zones = reinterpret_cast<ZoneDev *>(w1 + o_zones);
    p->counts = reinterpret_cast<int32_t *>(w1 + o_counts);
    p->err = reinterpret_cast<int32_t *>(w1 + o_err);
    CUDA_TRY(cudaMemsetAsync(p->counts, 0, 128, s));
    CUDA_TRY(cudaMemsetAsync(p->err, 0, 16, s));

    // ---- structural checks
    if (!(flags & SPMV_PLAN_NO_VALIDATE)) {
        CUDA_TRY(launch_validate(ptr, idx, p->n_major, (int)nnz, p->n_minor, p->err, s));
        int32_t e = 0;
        CUDA_TRY(cudaMemcpyAsync(&e, p->err, 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (e) {
            std::string msg = "malformed matrix:";
            if (e & 1) msg += " ptr[0] != 0;";
            if (e & 2) msg += " ptr decreasing or outside [0, nnz];";
            if (e & 4) msg += " ptr[last] != nnz;";
            if (e & 8) msg += " index out of range;";
            return set_error(SPMV_ERR_BAD_MATRIX, msg);
        }
    }

    // ---- the plan's own copy of the nonzeros in bank order (same nonzeros, permuted within
    // each segment); the caller's idx/vals are not read after this point
    if ((flags & SPMV_PLAN_BANK_ORDER) && nnz > 0) {
        const size_t ib = align_up((size_t)nnz * 4, 256);
        const size_t vb = align_up((size_t)nnz * p->sv, 256);
        CUDA_TRY(cudaMalloc(&p->owned_nz, ib + vb));
        p->owned_bytes = ib + vb;
        int32_t *slots = nullptr;
        CUDA_TRY(cudaMalloc(&slots, (size_t)nnz * 4));
        int32_t *oidx = static_cast<int32_t *>(p->owned_nz);
        void *ovals = static_cast<char *>(p->owned_nz) + ib;
        cudaError_t ce = launch_bank_order(ptr, p->n_major, (int)nnz, idx, vals, p->sv, oidx, ovals, slots, p->T,
                                           p->sx == 8 ? 16 : 32, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        cudaFree(slots);
        if (ce != cudaSuccess) return set_error(SPMV_ERR_CUDA, std::string("bank order: ") + cudaGetErrorString(ce));
        p->idx = oidx;
        p->vals = ovals;
    }

    // ---- Sec. II partition and Sec. IV-B set-up on the device: reporting chunks
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, s));
    CUDA_TRY(launch_pad_ptr(ptr, p->pptr, p->n_major, (int)nnz, p->pptr_len, s));
    CUDA_TRY(launch_chunks(p->pptr, p->n_major, (int)nnz, p->P, nullptr, p->T, p->aux, s));
    CUDA_TRY(launch_setup(p->aux, p->P, p->chunks, p->zones, p->counts, static_cast<char *>(p->ws) + o_sscr, s));
    p->ntiles = (int)nt64;

    // ---- workspace, part 2: tiles (descriptors, masks), processor zones, records and partial sums
    const int nt = p->ntiles;
    p->ctas = (pi && pi->ctas > 0) ? std::min(pi->ctas, std::max(nt, 1)) : std::max(1, std::min(sms, nt));
    p->bpc = (pi && pi->blocks_per_cta > 1 && (int64_t)p->ctas * pi->blocks_per_cta <= nt) ? pi->blocks_per_cta : 1;
    p->chunk_tiles = (opts && opts->chunk_tiles > 0) ? opts->chunk_tiles : CHUNK_TILES;
    // processors (chunks of tiles) of the streaming passes and their nonzero boundaries
    std::vector<int32_t> pnzb;
    {
        spmv_plan_s::ProcZones &pz = p->pz;
        pz.nproc = stream_processors(nt, p->T, (int)nnz, p->ctas * p->bpc, p->chunk_tiles, nullptr);
        pnzb.resize((size_t)pz.nproc + 1);
        stream_processors(nt, p->T, (int)nnz, p->ctas * p->bpc, p->chunk_tiles, pnzb.data());
        p->max_nproc = std::max(1, pz.nproc);
    }
    const size_t part_bytes = (pi && pi->segdot_only) ? 16
                              : p->onchip ? (size_t)p->ctas * p->batch_width * p->n_minor * p->sa
                                          : (size_t)p->n_minor * sizeof(double);
    const size_t rec_bytes = (size_t)VL_MAX * p->max_nproc * 2 * p->sa;  // any segmented pass: up to VL_MAX vectors
    off = 0;
    const size_t o_meta = carve((size_t)(nt + 1) * sizeof(TileMeta));
    const size_t o_masks = carve((size_t)std::max(nt, 1) * p->mwp * 4);
    const size_t o_pfx = carve((size_t)std::max(nt, 1) * p->mwq * 2);
    const size_t o_pz = carve((size_t)p->max_nproc * sizeof(ZoneDev));
    const size_t o_recl = carve(rec_bytes);
    const size_t o_recr = carve(rec_bytes);
    const size_t o_part = carve(std::max(part_bytes, (size_t)16));
    // set-up only
    const size_t o_tnzb = carve((size_t)(nt + 1) * 4);
    const size_t o_taux = carve((size_t)std::max(nt, 1) * sizeof(ChunkAux));
    const size_t o_pnzb = carve((size_t)(p->max_nproc + 1) * 4);
    const size_t o_paux = carve((size_t)p->max_nproc * sizeof(ChunkAux));
    const size_t o_pdev = carve((size_t)p->max_nproc * sizeof(ChunkDev));
    const size_t o_pscr = carve(setup_scratch_bytes(p->max_nproc));
    const size_t ws2 = off;
    CUDA_TRY(cudaMalloc(&p->ws2, ws2));
    p->ws_bytes = ws1 + ws2;
    char *w2 = static_cast<char *>(p->ws2);
    p->meta = reinterpret_cast<TileMeta *>(w2 + o_meta);
    p->masks = reinterpret_cast<uint32_t *>(w2 + o_masks);
    p->pfx = reinterpret_cast<uint16_t *>(w2 + o_pfx);
    p->rec_left = w2 + o_recl;
    p->rec_right = w2 + o_recr;
    p->part = w2 + o_part;
    int32_t *tnzb = reinterpret_cast<int32_t *>(w2 + o_tnzb);
    ChunkAux *taux = reinterpret_cast<ChunkAux *>(w2 + o_taux);
    int32_t *dpnzb = reinterpret_cast<int32_t *>(w2 + o_pnzb);
    ChunkAux *paux = reinterpret_cast<ChunkAux *>(w2 + o_paux);
    ChunkDev *pdev = reinterpret_cast<ChunkDev *>(w2 + o_pdev);
    if (nt > 0) {
        // execution tiles: bounds, first/last segments, owned end events; masks and descriptors
        CUDA_TRY(launch_tile_bounds(nt, p->T, (int)nnz, tnzb, s));
        CUDA_TRY(launch_chunks(p->pptr, p->n_major, (int)nnz, nt, tnzb, p->T, taux, s));
        CUDA_TRY(launch_masks(p->pptr, taux, nt, (int)nnz, p->n_major, p->mwp, p->masks, p->mwq, p->pfx, p->meta, s));
        // the Sec. IV-B set-up over the processors (chunks) gives their overlap zones
        spmv_plan_s::ProcZones &pz = p->pz;
        pz.zones = reinterpret_cast<ZoneDev *>(w2 + o_pz);
        CUDA_TRY(cudaMemcpyAsync(dpnzb, pnzb.data(), ((size_t)pz.nproc + 1) * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(launch_chunks(p->pptr, p->n_major, (int)nnz, pz.nproc, dpnzb, p->T, paux, s));
        CUDA_TRY(launch_setup(paux, pz.nproc, pdev, pz.zones, p->counts + 8, w2 + o_pscr, s));
    }
    CUDA_TRY(cudaMemsetAsync(p->rec_left, 0, rec_bytes, s));
    CUDA_TRY(cudaMemsetAsync(p->rec_right, 0, rec_bytes, s));
    CUDA_TRY(cudaEventRecord(e1, s));
    // zone counts of the reporting chunks ([0] z, [2] V) and of the processor tables ([8 + 4i])
    int32_t counts[32] = {0};
    CUDA_TRY(cudaMemcpyAsync(counts, p->counts, sizeof(counts), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // also keeps pnzb alive until its copies are done
    p->z = counts[0];
    p->vmax = counts[2];
    p->pz.z = nt > 0 ? counts[8] : 0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->setup_ms = ms;
    // the row-sorted copy for the short-vector accumulating product (validated plans only)
    if (!pi && (flags & SPMV_PLAN_ROW_BLOCKS) && !(flags & SPMV_PLAN_NO_VALIDATE) && nnz > 0) {
        spmv_status st = build_row_blocks(p, sms, s);
        if (st != SPMV_OK) return st;
    }
    guard.p = nullptr;
    *out = p;
    return SPMV_OK;
}

extern "C" {

spmv_status spmv_plan_destroy(spmv_plan_t plan) {
    if (!plan) return SPMV_OK;
    cudaDeviceSynchronize();
    plan_free(plan);
    return SPMV_OK;
}

spmv_status spmv_plan_info(spmv_plan_t p, spmv_plan_info_t *info) {
    if (!p || !info) return set_error(SPMV_ERR_INVALID_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->m = p->m;
    info->n = p->n;
    info->nnz = p->nnz;
    info->layout = p->layout;
    info->val_dtype = p->val_t;
    info->vec_dtype = p->vec_t;
    info->chunks = p->P;
    info->ctas = p->ctas;
    info->warps_per_cta = p->W_info;
    info->tile_items = p->T;
    info->stages = p->S;
    info->tiles = p->ntiles;
    info->zones = p->z;
    info->max_zone_size = p->vmax;
    info->short_on_chip = p->onchip ? 1 : 0;
    info->batch_width = p->batch_width;
    info->max_chunk_nnz = p->max_chunk;
    info->min_chunk_nnz = p->min_chunk;
    info->imbalance = p->nnz > 0 ? (double)p->P * (double)(p->max_chunk - p->min_chunk) / (double)p->nnz : 0.0;
    info->workspace_bytes = (int64_t)(p->ws_bytes + p->owned_bytes);
    info->setup_ms = p->setup_ms;
    info->row_blocks = p->tplan ? p->blocks : 0;
    info->row_block_window = p->tplan ? p->block_window : 0;
    if (p->tplan) info->workspace_bytes += (int64_t)(p->tplan->ws_bytes + p->tplan->owned_bytes + p->bws_bytes + p->bown_bytes);
    return SPMV_OK;
}

spmv_status spmv_plan_chunks(spmv_plan_t p, spmv_chunk_t *out, int32_t count) {
    if (!p || !out || count < 0 || count > p->P) return set_error(SPMV_ERR_INVALID_ARG, "bad arguments");
    std::vector<ChunkAux> aux((size_t)count);
    if (count > 0) CUDA_TRY(cudaMemcpy(aux.data(), p->aux, (size_t)count * sizeof(ChunkAux), cudaMemcpyDeviceToHost));
    for (int c = 0; c < count; ++c) {
        const ChunkAux &a = aux[c];
        spmv_chunk_t &h = out[c];
        h.nz_begin = a.nz_begin;
        h.nz_end = a.nz_end;
        h.jf = a.jf;
        h.jl = a.jl;
        h.needLeft = a.needLeft;
        h.needRight = a.needRight;
        h.leftGroupEnd = a.leftGroupEnd;
        h.rightGroup = a.rightGroup;
        h.leftGroup = a.leftGroup;
        h.procsOnLeft = a.procsOnLeft;
        h.procsOnRight = a.procsOnRight;
    }
    return SPMV_OK;
}

spmv_status spmv(spmv_plan_t p, const void *x, void *y, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return with_staging(p, x, (size_t)p->n * p->sx, y, (size_t)p->m * p->sx, s, [&](const void *dx, void *dy) {
        return run_op(p, SPMV_OP_AX, 1, &dx, &dy, s);
    });
}

spmv_status spvtm(spmv_plan_t p, const void *v, void *u, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return with_staging(p, v, (size_t)p->m * p->sx, u, (size_t)p->n * p->sx, s, [&](const void *dv, void *du) {
        return run_op(p, SPMV_OP_VTA, 1, &dv, &du, s);
    });
}

// The two products of a pair with host vectors: x's copy to the device runs on the plan's
// copy stream while the SpVTM kernels run on `s`, and u's copy to the host runs there while the
// SpMV kernels run.  Both streams are drained before returning, whatever happened.
static spmv_status pair_staged(spmv_plan_s *p, const void *x, void *y, const void *v, void *u, PtrKind kx,
                               PtrKind ky, PtrKind kv, PtrKind ku, cudaStream_t s) {
    const size_t cap = (size_t)std::max(p->m, p->n) * p->sx + 16;
    const size_t xb = (size_t)p->n * p->sx, yb = (size_t)p->m * p->sx;
    for (void **b : {&p->hin, &p->hout, &p->hv, &p->hu})
        if (!*b) CUDA_TRY(cudaMalloc(b, cap));
    if (!p->cstream) CUDA_TRY(cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking));
    if (!p->ev_x) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_x, cudaEventDisableTiming));
    if (!p->ev_u) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_u, cudaEventDisableTiming));
    cudaStream_t cs = p->cstream;
    spmv_status st = SPMV_OK;
    cudaError_t ce = cudaSuccess;
    auto step = [&](cudaError_t e) {
        if (ce == cudaSuccess && e != cudaSuccess) ce = e;
        return ce == cudaSuccess;
    };
    const void *dx = x, *dv = v;
    void *dy = ky == PK_HOST ? p->hout : y, *du = ku == PK_HOST ? p->hu : u;
    // the copy stream starts after the work already queued on s (which may use the buffers)
    step(cudaEventRecord(p->ev_u, s)) && step(cudaStreamWaitEvent(cs, p->ev_u, 0));
    // v's short copy is queued before x's long one: host-to-device copies share the copy
    // engines in the order they are issued, and the SpVTM waits for v only
    if (kv == PK_HOST && step(cudaMemcpyAsync(p->hv, v, yb, cudaMemcpyHostToDevice, s))) dv = p->hv;
    if (kx == PK_HOST && step(cudaMemcpyAsync(p->hin, x, xb, cudaMemcpyHostToDevice, cs)) &&
        step(cudaEventRecord(p->ev_x, cs)))
        dx = p->hin;
    if (ce == cudaSuccess) st = run_op(p, SPMV_OP_VTA, 1, &dv, &du, s);
    if (st == SPMV_OK && ku == PK_HOST && step(cudaEventRecord(p->ev_u, s)) && step(cudaStreamWaitEvent(cs, p->ev_u, 0)))
        step(cudaMemcpyAsync(u, p->hu, xb, cudaMemcpyDeviceToHost, cs));
    if (st == SPMV_OK && kx == PK_HOST) step(cudaStreamWaitEvent(s, p->ev_x, 0));
    if (st == SPMV_OK && ce == cudaSuccess) st = run_op(p, SPMV_OP_AX, 1, &dx, &dy, s);
    if (st == SPMV_OK && ky == PK_HOST) step(cudaMemcpyAsync(y, p->hout, yb, cudaMemcpyDeviceToHost, s));
    const cudaError_t e1 = cudaStreamSynchronize(cs), e2 = cudaStreamSynchronize(s);
    if (st != SPMV_OK) return st;
    step(e1);
    step(e2);
    if (ce != cudaSuccess)
        return set_error(ce == cudaErrorMemoryAllocation ? SPMV_ERR_OOM : SPMV_ERR_CUDA,
                         std::string("spmv_pair: ") + cudaGetErrorString(ce));
    return SPMV_OK;
}

// The two products of a pair with device vectors: the SpMV on `s`, the SpVTM on the plan's
// second stream, forked after the work queued on `s` and joined back into it.  They use
// disjoint parts of the workspace (per-CTA partials, carry records), and running side by side
// lets the short combine and fix-up kernels, and the tail of either pass, overlap the other.
// Asynchronous; whatever fails, the join is recorded so that `s` never runs ahead of the fork.
static spmv_status pair_device(spmv_plan_s *p, const void *x, void *y, const void *v, void *u, cudaStream_t s) {
    if (!p->cstream) CUDA_TRY(cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking));
    if (!p->ev_x) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_x, cudaEventDisableTiming));
    if (!p->ev_u) CUDA_TRY(cudaEventCreateWithFlags(&p->ev_u, cudaEventDisableTiming));
    cudaStream_t cs = p->cstream;
    CUDA_TRY(cudaEventRecord(p->ev_u, s));
    CUDA_TRY(cudaStreamWaitEvent(cs, p->ev_u, 0));
    spmv_status st_u = run_op(p, SPMV_OP_VTA, 1, &v, &u, cs);
    const std::string msg_u = st_u == SPMV_OK ? std::string() : std::string(spmv_last_error());
    spmv_status st_y = run_op(p, SPMV_OP_AX, 1, &x, &y, s);
    const cudaError_t e1 = cudaEventRecord(p->ev_x, cs);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(s, p->ev_x, 0) : e1;
    if (e2 != cudaSuccess) {  // the join could not be queued: wait for the second stream here
        cudaStreamSynchronize(cs);
        if (st_y == SPMV_OK && st_u == SPMV_OK)
            return set_error(SPMV_ERR_CUDA, std::string("spmv_pair: ") + cudaGetErrorString(e2));
    }
    if (st_y != SPMV_OK) return st_y;
    if (st_u != SPMV_OK) return set_error(st_u, msg_u);
    return SPMV_OK;
}

spmv_status spmv_pair(spmv_plan_t p, const void *x, void *y, const void *v, void *u, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto kind = [](const void *ptr, size_t bytes) { return (bytes == 0 && !ptr) ? PK_DEVICE : classify(ptr); };
    const size_t xb = (size_t)p->n * p->sx, yb = (size_t)p->m * p->sx;
    const PtrKind kx = kind(x, xb), ky = kind(y, yb), kv = kind(v, yb), ku = kind(u, xb);
    if (kx == PK_BAD || ky == PK_BAD || kv == PK_BAD || ku == PK_BAD)
        return set_error(SPMV_ERR_INVALID_ARG, "null vector pointer");
    const void *ptrs[4] = {x, y, v, u};
    const PtrKind kinds[4] = {kx, ky, kv, ku};
    for (int i = 0; i < 4; ++i)
        if (kinds[i] == PK_DEVICE && ptrs[i] && !aligned16(ptrs[i]))
            return set_error(SPMV_ERR_INVALID_ARG, "device vector pointers must be 16-byte aligned");
    std::lock_guard<std::mutex> lk(p->host_mu);
    if (kx == PK_DEVICE && ky == PK_DEVICE && kv == PK_DEVICE && ku == PK_DEVICE) return pair_device(p, x, y, v, u, s);
    return pair_staged(p, x, y, v, u, kx, ky, kv, ku, s);
}

spmv_status spmv_batch(spmv_plan_t p, int32_t op, int32_t k, const void *in, int64_t ld_in, void *out, int64_t ld_out,
                       void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    if (op != SPMV_OP_AX && op != SPMV_OP_VTA) return set_error(SPMV_ERR_INVALID_ARG, "bad op");
    if (k < 1 || k > 4096) return set_error(SPMV_ERR_INVALID_ARG, "k must lie in [1, 4096]");
    const int64_t len_in = op == SPMV_OP_AX ? p->n : p->m;
    const int64_t len_out = op == SPMV_OP_AX ? p->m : p->n;
    if (ld_in < len_in || ld_out < len_out) return set_error(SPMV_ERR_INVALID_ARG, "ld smaller than vector length");
    if ((ld_in * p->sx) % 16 || (ld_out * p->sx) % 16)
        return set_error(SPMV_ERR_INVALID_ARG, "ld * element size must be a multiple of 16 bytes");
    if (classify(in) != PK_DEVICE || classify(out) != PK_DEVICE || !aligned16(in) || !aligned16(out))
        return set_error(SPMV_ERR_INVALID_ARG, "spmv_batch takes 16-byte aligned device pointers");
    std::vector<const void *> vi(k);
    std::vector<void *> vo(k);
    for (int b = 0; b < k; ++b) {
        vi[b] = static_cast<const char *>(in) + (size_t)b * ld_in * p->sx;
        vo[b] = static_cast<char *>(out) + (size_t)b * ld_out * p->sx;
    }
    return run_op(p, op, k, vi.data(), vo.data(), static_cast<cudaStream_t>(stream));
}

spmv_status spmv_dvalues(spmv_plan_t p, const void *r, const void *x, void *g, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    if (!r || !x || (!g && p->nnz > 0)) return set_error(SPMV_ERR_INVALID_ARG, "null pointer");
    if (p->owned_nz)
        return set_error(SPMV_ERR_UNSUPPORTED, "spmv_dvalues on a bank-ordered plan (its values are permuted)");
    if (p->nnz == 0) return SPMV_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const PtrKind kr = classify(r), kx = classify(x), kg = classify(g);
    if (kr == PK_DEVICE && kx == PK_DEVICE && kg == PK_DEVICE) {
        if (!aligned16(r) || !aligned16(x) || !aligned16(g))
            return set_error(SPMV_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
        return run_dvalues(p, r, x, g, s);
    }
    std::lock_guard<std::mutex> lk(p->host_mu);
    const size_t cap = (size_t)std::max(p->m, p->n) * p->sx + 16;
    if (!p->hin) CUDA_TRY(cudaMalloc(&p->hin, cap));
    if (!p->hout) CUDA_TRY(cudaMalloc(&p->hout, cap));
    if (!p->hg) CUDA_TRY(cudaMalloc(&p->hg, (size_t)p->nnz * p->sv + 16));
    const void *dr = r, *dx = x;
    void *dg = g;
    if (kr == PK_HOST) {
        CUDA_TRY(cudaMemcpyAsync(p->hin, r, (size_t)p->m * p->sx, cudaMemcpyHostToDevice, s));
        dr = p->hin;
    }
    if (kx == PK_HOST) {
        CUDA_TRY(cudaMemcpyAsync(p->hout, x, (size_t)p->n * p->sx, cudaMemcpyHostToDevice, s));
        dx = p->hout;
    }
    if (kg == PK_HOST) dg = p->hg;
    spmv_status st = run_dvalues(p, dr, dx, dg, s);
    if (st != SPMV_OK) return st;
    if (kg == PK_HOST) CUDA_TRY(cudaMemcpyAsync(g, dg, (size_t)p->nnz * p->sv, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

spmv_status spmv_plan_export(spmv_plan_t p, int32_t *idx_out, void *vals_out, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    if (p->nnz == 0) return SPMV_OK;
    if (!idx_out || !vals_out) return set_error(SPMV_ERR_INVALID_ARG, "null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(idx_out, p->idx, (size_t)p->nnz * 4, cudaMemcpyDefault, s));
    CUDA_TRY(cudaMemcpyAsync(vals_out, p->vals, (size_t)p->nnz * p->sv, cudaMemcpyDefault, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SPMV_OK;
}

spmv_status spmv_check(spmv_plan_t p, void *stream) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    int32_t e = 0, et = 0;
    CUDA_TRY(cudaMemcpy(&e, p->err, 4, cudaMemcpyDeviceToHost));
    if (p->tplan) {
        CUDA_TRY(cudaMemcpy(&et, p->tplan->err, 4, cudaMemcpyDeviceToHost));
        if (et) CUDA_TRY(cudaMemset(p->tplan->err, 0, 4));
        e |= et;
    }
    if (e) {
        CUDA_TRY(cudaMemset(p->err, 0, 4));
        std::string msg = "device error:";
        if (e & 1) msg += " index outside the short vector (clamped into it);";
        if (e & 2) msg += " staging wait timed out;";
        if (e & 4) msg += " inconsistent tile descriptor;";
        return set_error(SPMV_ERR_DEVICE, msg);
    }
    return SPMV_OK;
}

spmv_status spmv_profile_read(spmv_plan_t p, int32_t kernel, double *ms, int64_t *launches) {
    if (!p || kernel < 0 || kernel > 6) return set_error(SPMV_ERR_INVALID_ARG, "bad arguments");
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(p->prof_mu);
    for (auto &pr : p->prof) {
        float t = 0.f;
        cudaEventElapsedTime(&t, pr.a, pr.b);
        p->prof_ms[pr.kernel] += t;
        p->prof_n[pr.kernel] += 1;
        cudaEventDestroy(pr.a);
        cudaEventDestroy(pr.b);
    }
    p->prof.clear();
    if (ms) *ms = p->prof_ms[kernel];
    if (launches) *launches = p->prof_n[kernel];
    return SPMV_OK;
}

spmv_status spmv_profile_enable(spmv_plan_t p, int32_t on) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    p->prof_on.store(on != 0);
    return SPMV_OK;
}

spmv_status spmv_profile_reset(spmv_plan_t p) {
    if (!p) return set_error(SPMV_ERR_INVALID_ARG, "null plan");
    double d;
    int64_t n;
    spmv_profile_read(p, 0, &d, &n);
    std::lock_guard<std::mutex> lk(p->prof_mu);
    for (int i = 0; i < 7; ++i) {
        p->prof_ms[i] = 0;
        p->prof_n[i] = 0;
    }
    return SPMV_OK;
}

}  // extern "C"
