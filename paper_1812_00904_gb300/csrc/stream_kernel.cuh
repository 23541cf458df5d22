// Streaming kernel: one warp per nonzero chunk (Sec. II), the chunk's tiles
// staged into shared memory by bulk (TMA) copies, one mbarrier per stage.
//
// Terms.  "major" is the compressed dimension (columns of a wide CSC matrix,
// rows of a tall CSR matrix), "minor" the indexed one.  A chunk owns the
// nonzeros [nz_begin, nz_end) and the END EVENTS of the major segments
// [e_begin, e_end): segment j ends after its last nonzero, and its end event
// is ordered before the nonzero at position ptr[j+1] (merge order of segment
// ends and nonzeros).  A tile is a run of that merge order of about
// `tile_items` items that starts right before a nonzero at a multiple of 8
// (or at the chunk start); tile t covers nonzeros [k0, k1) and the end events
// [i0, i1), so the nonzeros of the tile lie in segments i0..i1.
//
//   MODE_SCATTER: acc[idx[k]] += val[k] * w[seg(k)]  -- A_(i) x_(i) of Sec. III
//                 (wide CSC y = A x; tall CSR u = v^T A by role reversal).
//   MODE_SEGDOT:  out[j] = sum_k val[k] * w[idx[k]] over segment j -- v^T A_(i)
//                 of Sec. IV-A (wide CSC u^T = v^T A; tall CSR y = A x).  A
//                 segment split between chunks (an overlap zone) leaves its
//                 partial sums in carry records for the zone fixup.
//   MODE_DVALUES: g[k] = minor[idx[k]] * major[seg(k)].
//
// Pipeline.  Every lane of the warp computes the geometry of the tile to
// stage (tile descriptors are prefetched 32 at a time, one per lane); lane 0
// writes it into the stage's 64-byte header and issues the bulk copies; the
// consumer reads the header after the stage's mbarrier phase completes.
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace gbk {

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per staging wait
constexpr uint64_t DRAIN_LIMIT_NS = 200000000ull;   // 0.2 s per wait while draining after a failure
constexpr int WARP_HDR_BYTES = 256;                  // 8 mbarriers, 32 head-mask words (per warp)
constexpr int STAGE_HDR_BYTES = 64;                  // tile geometry at the start of every stage

struct Geo {              // 64 bytes, written by the producer into the stage header
    int k0, k1, i0, i1;   // nonzeros [k0, k1), end events [i0, i1)
    int kb0, ncov;        // staged nonzero cover [kb0, kb0 + ncov), kb0 = k0 rounded down to 8
    int flags;            // bit 0: an empty segment ends in the tile (general path)
    int off_val, off_mask, off_ptr, off_x;  // byte offsets after the header
    int pbase, npc;       // staged pointer cover [pbase, pbase + npc) (general path only)
    int xbase, nxc;       // staged major-vector cover
    int okwin;            // bit 0: descriptor consistent; bit 1: windows staged (else read from global memory)
};

template <typename VT, typename XT, int MODE>
__device__ __forceinline__ Geo make_geo(const StreamParams &p, int4 a, int2 b, int nvec) {
    Geo g;
    g.k0 = a.x;
    g.i0 = a.y;
    g.flags = a.z;
    g.k1 = b.x;
    g.i1 = b.y;
    g.kb0 = g.k0 & ~7;
    g.ncov = ((g.k1 + 7) & ~7) - g.kb0;
    g.off_val = g.ncov * 4;
    g.off_mask = g.off_val + g.ncov * (int)sizeof(VT);
    g.off_ptr = g.off_mask + p.mwp * 4;
    g.pbase = g.i0 & ~3;
    g.npc = (g.flags & 1) ? ((g.i1 + 1 + 3) & ~3) - g.pbase : 0;
    g.off_x = g.off_ptr + g.npc * 4;
    int bytes = g.off_x;
    g.xbase = 0;
    g.nxc = 0;
    if (MODE != MODE_SEGDOT) {
        constexpr int xa = 16 / (int)sizeof(XT);
        const int last = min(g.i1, p.n_major - 1);
        if (last >= g.i0) {
            g.xbase = g.i0 & ~(xa - 1);
            g.nxc = ((last + 1 + xa - 1) & ~(xa - 1)) - g.xbase;
        }
        bytes = g.off_x + nvec * g.nxc * (int)sizeof(XT);
    }
    const int cap = p.stage_bytes - STAGE_HDR_BYTES;
    // A descriptor that would overrun the stage or the 1024-position head mask
    // is refused; it cannot occur for a plan built by the set-up kernels.
    const bool ok = g.k1 >= g.k0 && g.i1 >= g.i0 && g.k0 >= 0 && g.k1 <= p.nnz && g.i1 <= p.n_major &&
                    g.ncov <= 1024 && g.off_ptr <= cap;
    g.okwin = (ok ? 1 : 0) | (bytes <= cap ? 2 : 0);
    return g;
}

__device__ __forceinline__ void copy_elem(unsigned char *d, const unsigned char *s, int es) {
    if (es == 8) {
        *reinterpret_cast<unsigned long long *>(d) = *reinterpret_cast<const unsigned long long *>(s);
    } else if (es == 4) {
        *reinterpret_cast<unsigned int *>(d) = *reinterpret_cast<const unsigned int *>(s);
    } else {
        *reinterpret_cast<unsigned short *>(d) = *reinterpret_cast<const unsigned short *>(s);
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Stage elements [e0, e0 + cnt) of an array of `len` elements of `es` bytes
// into dst (e0 a multiple of 16/es): the part below the array's last 16-byte
// boundary by bulk copy (its bytes announced on `bar` first), the rest -- at
// most 15 bytes at the very end of the array -- by plain loads.  Lane 0 only.
__device__ __forceinline__ void stage_part(unsigned char *dst, const void *src, int e0, int cnt, int len, int es,
                                           uint64_t *bar) {
    const int al = 16 / es;
    const int lim = len & ~(al - 1);
    const int end = e0 + cnt;
    const int bend = end < lim ? end : lim;
    if (bend > e0) {
        const uint32_t bytes = static_cast<uint32_t>(bend - e0) * es;
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, static_cast<const unsigned char *>(src) + (size_t)e0 * es, bytes, bar);
    }
    if (end > lim) {
        const int t1 = end < len ? end : len;
        for (int e = (e0 > lim ? e0 : lim); e < t1; ++e)
            copy_elem(dst + (size_t)(e - e0) * es, static_cast<const unsigned char *>(src) + (size_t)e * es, es);
    }
}

template <typename XT> __device__ __forceinline__ XT zero_of() { return XT(0); }

template <bool B> struct BoolC {
    static constexpr bool value = B;
};

template <typename VT, typename XT, int MODE, int KB, bool SMEMV>
__global__ void __launch_bounds__(MAX_WARPS * 32, 1) stream_kernel(const __grid_constant__ StreamParams p) {
    using AT = typename Acc<VT>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int kb = (MODE == MODE_DVALUES) ? 1 : p.kb;
    const int nvec = (MODE == MODE_DVALUES) ? 1 : p.kb;
    const unsigned n_minor = static_cast<unsigned>(p.n_minor);

    // ---- the short (minor) vector on chip: accumulator (SCATTER) or input (SEGDOT / DVALUES)
    if constexpr (SMEMV) {
        if constexpr (MODE == MODE_SCATTER) {
            AT *acc = reinterpret_cast<AT *>(smem);
            for (int i = threadIdx.x; i < p.n_minor * KB; i += blockDim.x) acc[i] = AT(0);
        } else {
            XT *vs = reinterpret_cast<XT *>(smem);
            for (int i = threadIdx.x; i < p.n_minor; i += blockDim.x) {
#pragma unroll
                for (int b = 0; b < KB; ++b)
                    vs[i * KB + b] = (b < kb) ? static_cast<const XT *>(p.vin[b])[i] : zero_of<XT>();
            }
        }
    }
    __syncthreads();

    const int c = blockIdx.x * W + warp;
    if (c < p.P) {
        const ChunkDev cd = p.chunks[c];
        const bool needLeft = (cd.flags & 1) != 0;
        const bool needRight = (cd.flags & 2) != 0;
        unsigned char *wbase = smem + p.vec_region_bytes + warp * p.warp_bytes;
        uint64_t *bars = reinterpret_cast<uint64_t *>(wbase);
        unsigned char *stages = wbase + WARP_HDR_BYTES;
        const int S = p.stages;
        const int tb = cd.tile_begin;
        const int nt = cd.tile_end - cd.tile_begin;
        // running sum of the open segment: compensated (hi + lo) in the accumulation type
        AT chi[KB], clo[KB];
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            chi[b] = AT(0);
            clo[b] = AT(0);
        }

        // Emit the finished dot product of segment `col` for vector b (SEGDOT):
        // the first segment of a chunk that shares it with its left neighbour
        // goes to the chunk's left carry record (Sec. IV-A), the rest to out.
        auto emit = [&](int col, int b, AT value) {
            if (needLeft && col == cd.jf)
                p.rec_left[b * p.P + c] = static_cast<double>(value);
            else
                static_cast<XT *>(p.vout[b])[col] = static_cast<XT>(value);
        };

        // tile descriptors, one per lane, a block of 32 at a time (next block prefetched)
        int bcur = 0;
        int4 dcur = make_int4(0, 0, 0, 0), dnext = make_int4(0, 0, 0, 0);
        auto load_block = [&](int blk) -> int4 {
            const int q = blk * 32 + lane;
            return q < nt ? p.tiles[tb + q] : make_int4(cd.nz_end, cd.e_end, 0, 0);
        };
        // descriptor of chunk-local tile q (q == nt gives the chunk end); q's block is bcur or bcur + 1
        auto tile_at = [&](int q) -> int4 {
            const int4 src = ((q >> 5) == bcur) ? dcur : dnext;
            int4 r;
            r.x = __shfl_sync(FULL, src.x, q & 31);
            r.y = __shfl_sync(FULL, src.y, q & 31);
            r.z = __shfl_sync(FULL, src.z, q & 31);
            r.w = 0;
            return (q >= nt) ? make_int4(cd.nz_end, cd.e_end, 0, 0) : r;
        };
        // all lanes: geometry of tile q into stage s; lane 0 writes the header and issues the copies
        auto issue = [&](int q, int s) {
            while ((q >> 5) > bcur) {
                dcur = dnext;
                ++bcur;
                dnext = load_block(bcur + 1);
            }
            const int4 nx = tile_at(q + 1);
            const Geo g = make_geo<VT, XT, MODE>(p, tile_at(q), make_int2(nx.x, nx.y), nvec);
            unsigned char *st = stages + s * p.stage_bytes;
            uint64_t *bar = &bars[s];
            unsigned char *d = st + STAGE_HDR_BYTES;
            if (lane == 0) *reinterpret_cast<Geo *>(st) = g;
            // One staged array per lane, in the same instruction stream: 0 indices, 1 values,
            // 2 head mask, 3 pointer window, 4.. major-vector windows.  The part below an array's
            // last 16-byte boundary goes by bulk copy, the rest (at most 15 bytes at the very end
            // of an array) by plain loads before the arrive that releases them.
            const bool w = (g.okwin & 2) != 0;
            const void *src = p.idx;
            unsigned char *dst = d;
            int e0 = g.kb0, cnt = g.ncov, len = p.nnz, es = 4;
            if (lane == 1) {
                src = p.vals;
                dst = d + g.off_val;
                es = (int)sizeof(VT);
            } else if (lane == 2) {
                src = p.masks + (size_t)(tb + q) * p.mwp;
                dst = d + g.off_mask;
                e0 = 0;
                cnt = p.mwp;
                len = p.mwp;
            } else if (lane == 3) {
                src = p.pptr;
                dst = d + g.off_ptr;
                e0 = g.pbase;
                cnt = w ? g.npc : 0;
                len = p.pptr_len;
            } else if (lane >= 4) {
                const int b = lane - 4;
                src = (MODE == MODE_DVALUES) ? p.vin[1] : p.vin[b < KB_MAX ? b : 0];
                dst = d + g.off_x + b * g.nxc * (int)sizeof(XT);
                e0 = g.xbase;
                cnt = (MODE != MODE_SEGDOT && w && b < nvec) ? g.nxc : 0;
                len = p.n_major;
                es = (int)sizeof(XT);
            }
            if (!(g.okwin & 1)) cnt = 0;
            const int al = 16 / es;
            const int lim = len & ~(al - 1);
            const int end = e0 + cnt;
            const int bend = min(end, lim);
            const uint32_t bytes = bend > e0 ? static_cast<uint32_t>(bend - e0) * es : 0u;
            if (cnt > 0 && end > lim) {
                const int t1 = min(end, len);
                for (int e = max(e0, lim); e < t1; ++e)
                    copy_elem(dst + (size_t)(e - e0) * es, static_cast<const unsigned char *>(src) + (size_t)e * es, es);
            }
            const uint32_t total = __reduce_add_sync(FULL, bytes);
            __syncwarp();
            // releases the header and the plain stores; the bulk bytes complete the phase
            if (lane == 0) mbar_arrive_expect_tx(bar, total);
            if (bytes) bulk_g2s(dst, static_cast<const unsigned char *>(src) + (size_t)e0 * es, bytes, bar);
        };

        if (nt > 0) {
            dcur = load_block(0);
            dnext = load_block(1);
            if (lane == 0) {
                for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
                fence_mbar_init();
            }
            __syncwarp();
            for (int q = 0; q < S && q < nt; ++q) issue(q, q);
            int s = 0;
            uint32_t phase = 0;
            for (int q = 0; q < nt; ++q) {
                unsigned char *st = stages + s * p.stage_bytes;
                bool ok = mbar_wait_bounded(&bars[s], phase, WAIT_LIMIT_NS);
                ok = __all_sync(FULL, ok);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(p.err, ERR_WAIT);
                        int ss = s;
                        uint32_t ph = phase;
                        for (int r = q; r < nt && r < q + S; ++r) {
                            mbar_wait_bounded(&bars[ss], ph, DRAIN_LIMIT_NS);
                            if (++ss == S) {
                                ss = 0;
                                ph ^= 1u;
                            }
                        }
                    }
                    __syncwarp();
                    break;
                }
                const Geo g = *reinterpret_cast<const Geo *>(st);
                if (g.okwin & 1) {
                    const unsigned char *dat = st + STAGE_HDR_BYTES;
                    const int rel_lo = g.k0 - g.kb0;
                    const int rel_hi = g.k1 - g.kb0;
                    const bool win = (g.okwin & 2) != 0;
                    const bool dup = (g.flags & 1) != 0;
                    const int32_t *idx_s = reinterpret_cast<const int32_t *>(dat);
                    const unsigned char *val_s = dat + g.off_val;
                    const int32_t *ptr_s = reinterpret_cast<const int32_t *>(dat + g.off_ptr);
                    const XT *x_s = reinterpret_cast<const XT *>(dat + g.off_x);
                    auto PW = [&](int j) -> int { return win ? ptr_s[j - g.pbase] : p.pptr[j]; };

                    // ---- A. segment-start bits of the tile (computed by the plan), one word per lane
                    const uint32_t mw = lane < p.mwp ? reinterpret_cast<const uint32_t *>(dat + g.off_mask)[lane] : 0u;
                    if constexpr (MODE == MODE_SEGDOT) {
                        if (dup) {  // empty segments ending in this tile get u_j = 0
                            for (int j = g.i0 + 1 + lane; j < g.i1; j += 32)
                                if (PW(j + 1) == PW(j)) {
#pragma unroll
                                    for (int b = 0; b < KB; ++b)
                                        if (b < kb) static_cast<XT *>(p.vout[b])[j] = zero_of<XT>();
                                }
                        }
                    }
                    int incl = __popc(mw);
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int v = __shfl_up_sync(FULL, incl, d);
                        if (lane >= d) incl += v;
                    }
                    const int cnt_ex = incl - __popc(mw);
                    const int htotal = __shfl_sync(FULL, incl, 31);

                    // Segment holding staged position pos (relative to kb0; pos may be -1): the last
                    // segment j in [i0, i1] starting at or before it.  Used when several segments
                    // start at one position (empty segments) or the window is not staged.
                    auto col_search = [&](int pos) -> int {
                        int lo = g.i0, hi = g.i1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (PW(mid) - g.kb0 <= pos)
                                lo = mid;
                            else
                                hi = mid - 1;
                        }
                        return lo;
                    };

                    // ---- B. 128 positions per step, 4 consecutive per lane
                    auto run_steps = [&](auto fast_tag) {
                        constexpr bool FAST = decltype(fast_tag)::value;  // one segment start per head bit, staged window
                        const int nsteps = (rel_hi + 127) >> 7;
#pragma unroll 2
                        for (int stp = 0; stp < nsteps; ++stp) {
                            const int p0 = (stp << 7) + (lane << 2);
                            const int sh = (lane & 7) << 2;
                            const uint32_t mwl = __shfl_sync(FULL, mw, p0 >> 5);
                            const int cwl = __shfl_sync(FULL, cnt_ex, p0 >> 5);
                            const uint32_t hb = (mwl >> sh) & 0xFu;
                            const int base = cwl + __popc(mwl & ((1u << sh) - 1u));  // heads before p0
                            // valid items of this lane: positions in [rel_lo, rel_hi)
                            const int lo_cut = min(max(rel_lo - p0, 0), 4);
                            const int hi_cut = min(max(rel_hi - p0, 0), 4);
                            uint32_t vm = ((1u << hi_cut) - 1u) & ~((1u << lo_cut) - 1u);
                            int ix[4] = {0, 0, 0, 0};
                            AT va[4] = {AT(0), AT(0), AT(0), AT(0)};
                            if (vm) {
                                const int4 qi = reinterpret_cast<const int4 *>(idx_s)[p0 >> 2];
                                ix[0] = qi.x;
                                ix[1] = qi.y;
                                ix[2] = qi.z;
                                ix[3] = qi.w;
                                Load4<VT, AT>::run(val_s, p0, va);
                                uint32_t bad = 0;
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    bad |= (static_cast<unsigned>(ix[e]) >= n_minor ? 1u : 0u) << e;
                                if (bad & vm) {
                                    atomicOr(p.err, ERR_INDEX);
                                    vm &= ~bad;
                                }
                            }
                            // segment of item e: heads at or before it
                            int col[4];
                            if constexpr (FAST) {
                                int cc = g.i0 + base;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    cc += (hb >> e) & 1u;
                                    col[e] = cc;
                                }
                            }

                            if constexpr (MODE == MODE_SCATTER) {
                                {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    if ((vm >> e) & 1u) {
                                        const int ce = FAST ? col[e] : col_search(p0 + e);
#pragma unroll
                                        for (int b = 0; b < KB; ++b) {
                                            if (b < kb) {
                                                                    const XT xv = (FAST || win) ? x_s[b * g.nxc + ce - g.xbase]
                                                                            : static_cast<const XT *>(p.vin[b])[ce];
                                                const AT contrib = va[e] * static_cast<AT>(xv);
                                                if constexpr (SMEMV) {
                                                    atomicAdd(reinterpret_cast<AT *>(smem) + ix[e] * KB + b, contrib);
                                                } else {
                                                    atomicAdd(static_cast<double *>(p.part) + (size_t)b * p.n_minor + ix[e],
                                                              static_cast<double>(contrib));
                                                }
                                            }
                                        }
                                    }
                                }
                                }
                            } else {  // MODE_DVALUES
                                VT *gout = static_cast<VT *>(p.vout[0]);
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    if ((vm >> e) & 1u) {
                                        const int ce = FAST ? col[e] : col_search(p0 + e);
                                        const XT xv = (FAST || win) ? x_s[ce - g.xbase]
                                                                      : static_cast<const XT *>(p.vin[1])[ce];
                                        AT mv;
                                        if constexpr (SMEMV) {
                                            mv = static_cast<AT>(reinterpret_cast<const XT *>(smem)[ix[e]]);
                                        } else {
                                            mv = static_cast<AT>(__ldg(static_cast<const XT *>(p.vin[0]) + ix[e]));
                                        }
                                        gout[g.kb0 + p0 + e] = from_d<VT>(static_cast<double>(mv * static_cast<AT>(xv)));
                                    }
                                }
                            }
                        }
                    };
                    // ---- B'. SEGDOT: 256 positions per step, 8 consecutive per lane
                    auto run_steps8 = [&](auto fast_tag) {
                        constexpr bool FAST = decltype(fast_tag)::value;
                        const int nsteps = (rel_hi + 255) >> 8;
                        for (int stp = 0; stp < nsteps; ++stp) {
                            const int p0 = (stp << 8) + (lane << 3);
                            const int sh = (lane & 3) << 3;
                            const uint32_t mwl = __shfl_sync(FULL, mw, p0 >> 5);
                            const int cwl = __shfl_sync(FULL, cnt_ex, p0 >> 5);
                            const uint32_t hb = (mwl >> sh) & 0xFFu;
                            const int base = cwl + __popc(mwl & ((1u << sh) - 1u));  // heads before p0
                            const int lo_cut = min(max(rel_lo - p0, 0), 8);
                            const int hi_cut = min(max(rel_hi - p0, 0), 8);
                            uint32_t vm = ((1u << hi_cut) - 1u) & ~((1u << lo_cut) - 1u);
                            int ix[8];
                            AT va[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                ix[e] = 0;
                                va[e] = AT(0);
                            }
                            if (vm) {
                                const int4 qa = reinterpret_cast<const int4 *>(idx_s)[p0 >> 2];
                                const int4 qb = reinterpret_cast<const int4 *>(idx_s)[(p0 >> 2) + 1];
                                ix[0] = qa.x;
                                ix[1] = qa.y;
                                ix[2] = qa.z;
                                ix[3] = qa.w;
                                ix[4] = qb.x;
                                ix[5] = qb.y;
                                ix[6] = qb.z;
                                ix[7] = qb.w;
                                Load8<VT, AT>::run(val_s, p0, va);
                                unsigned mx = 0;
#pragma unroll
                                for (int e = 0; e < 8; ++e) mx = max(mx, static_cast<unsigned>(ix[e]));
                                if (mx >= n_minor) {  // out-of-range entries are skipped and reported
                                    uint32_t bad = 0;
#pragma unroll
                                    for (int e = 0; e < 8; ++e)
                                        bad |= (static_cast<unsigned>(ix[e]) >= n_minor ? 1u : 0u) << e;
                                    if (bad & vm) atomicOr(p.err, ERR_INDEX);
                                    vm &= ~bad;
                                }
                            }
                            // lane-local inclusive prefix, restarted at every head
                            AT r[8][KB];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
#pragma unroll
                                for (int b = 0; b < KB; ++b) {
                                    AT w_ = AT(0);
                                    if ((vm >> e) & 1u) {
                                        if constexpr (SMEMV) {
                                            w_ = static_cast<AT>(reinterpret_cast<const XT *>(smem)[ix[e] * KB + b]);
                                        } else {
                                            w_ = static_cast<AT>(__ldg(static_cast<const XT *>(p.vin[b]) + ix[e]));
                                        }
                                    }
                                    const AT pr = va[e] * w_;
                                    r[e][b] = (e == 0 || ((hb >> e) & 1u)) ? pr : r[e > 0 ? e - 1 : 0][b] + pr;
                                }
                            }
                            // warp segmented scan of the lanes' open sums (the o operator of Sec. IV-B)
                            const unsigned bal = __ballot_sync(FULL, hb != 0u);
                            const unsigned le = bal & (FULL >> (31 - lane));
                            const int seg_start = le ? (31 - __clz(le)) : 0;
                            const bool before = (bal & ((1u << lane) - 1u)) != 0u;
                            const int nemit = bal ? static_cast<int>(__reduce_max_sync(FULL, static_cast<unsigned>(__popc(hb)))) : 0;
#pragma unroll
                            for (int b = 0; b < KB; ++b) {
                                AT T = r[7][b];
#pragma unroll
                                for (int d = 1; d < 32; d <<= 1) {
                                    const AT v = __shfl_up_sync(FULL, T, d);
                                    if (lane - d >= seg_start && lane >= d) T += v;
                                }
                                AT Tex = __shfl_up_sync(FULL, T, 1);
                                if (lane == 0) Tex = AT(0);
                                if (nemit > 0 && b < kb) {
                                    // value of the segment ending right before item h (h = 0..7):
                                    // h = 0 closes the segment open at the lane start; h >= 1 closes the
                                    // one ending at item h-1 (the leading one gets the incoming sum)
                                    const AT lead_add = Tex + (before ? AT(0) : chi[b] + clo[b]);
                                    uint32_t rem = hb;
                                    for (int it = 0; it < nemit; ++it) {
                                        const int h = rem ? __ffs(rem) - 1 : 0;
                                        // r[h-1] (h >= 1), selected without indexing the register array
                                        AT v = AT(0);
#pragma unroll
                                        for (int hh = 1; hh < 8; ++hh) v = (h == hh) ? r[hh - 1][b] : v;
                                        const uint32_t upto = hb & ((1u << h) - 1u);
                                        if (upto == 0u) v += lead_add;  // the segment started before this lane
                                        if (rem) {
                                            const int col = FAST ? g.i0 + base + __popc(upto) : col_search(p0 + h - 1);
                                            emit(col, b, v);
                                        }
                                        rem &= rem - 1u;
                                    }
                                }
                                const AT T31 = __shfl_sync(FULL, T, 31);
                                if (bal) {
                                    chi[b] = T31;
                                    clo[b] = AT(0);
                                } else {  // compensated addition (TwoSum) of the step total
                                    const AT s_ = chi[b] + T31;
                                    const AT bp = s_ - chi[b];
                                    clo[b] += (chi[b] - (s_ - bp)) + (T31 - bp);
                                    chi[b] = s_;
                                }
                            }
                        }
                    };
                    if constexpr (MODE == MODE_SEGDOT) {
                        if (!dup)
                            run_steps8(BoolC<true>{});
                        else
                            run_steps8(BoolC<false>{});
                    } else {
                        if (!dup && win)
                            run_steps(BoolC<true>{});
                        else
                            run_steps(BoolC<false>{});
                    }

                    // ---- C. tile end: a segment whose end event lies in this tile is complete
                    if constexpr (MODE == MODE_SEGDOT) {
                        int col_last = g.i0;
                        if (rel_hi > rel_lo) col_last = dup ? col_search(rel_hi - 1) : g.i0 + htotal;
                        if (col_last < g.i1) {
                            if (lane == 0)
                                for (int b = 0; b < kb; ++b) emit(col_last, b, chi[b] + clo[b]);
#pragma unroll
                            for (int b = 0; b < KB; ++b) {
                                chi[b] = AT(0);
                                clo[b] = AT(0);
                            }
                        }
                    }
                } else if (lane == 0) {
                    atomicOr(p.err, ERR_STRUCT);
                }
                // every lane's reads of this stage are done before its refill is issued
                __syncwarp();
                if (q + S < nt) issue(q + S, s);
                if (++s == S) {
                    s = 0;
                    phase ^= 1u;
                }
            }
        }
        if constexpr (MODE == MODE_SEGDOT) {
            // the chunk's last segment continues in the next chunk: right carry record
            if (needRight && lane == 0)
                for (int b = 0; b < kb; ++b) p.rec_right[b * p.P + c] = static_cast<double>(chi[b]) + static_cast<double>(clo[b]);
        }
    }

    if constexpr (MODE == MODE_SCATTER && SMEMV) {
        __syncthreads();
        const AT *acc = reinterpret_cast<const AT *>(smem);
        AT *part = static_cast<AT *>(p.part);
        for (int b = 0; b < kb; ++b)
            for (int i = threadIdx.x; i < p.n_minor; i += blockDim.x)
                part[((size_t)blockIdx.x * kb + b) * p.n_minor + i] = acc[i * KB + b];
    }
}

// Host-side launch of one instantiation; sets the shared-memory limit once.
template <typename VT, typename XT, int MODE, int KB, bool SMEMV>
cudaError_t launch_one(const LaunchArgs &a) {
    auto kern = stream_kernel<VT, XT, MODE, KB, SMEMV>;
    static int configured = 0;
    if (configured < a.smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem);
        if (e != cudaSuccess) return e;
        configured = a.smem;
    }
    kern<<<a.grid, a.block, a.smem, a.stream>>>(a.sp);
    return cudaGetLastError();
}

}  // namespace gbk
