// Streaming kernel: one warp per nonzero chunk (Sec. II), tiles of the chunk
// staged into shared memory by bulk (TMA) copies, one mbarrier per stage.
//
// Terms.  "major" is the compressed dimension (columns of a wide CSC matrix,
// rows of a tall CSR matrix), "minor" the indexed one.  A chunk owns the
// nonzeros [nz_begin, nz_end) and the END EVENTS of the major segments
// [e_begin, e_end): segment j ends after its last nonzero, and its end event
// is ordered before the nonzero at position ptr[j+1] (merge order of segment
// ends and nonzeros).  A tile is a run of that merge order of at most
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
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace gbk {

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per staging wait
constexpr uint64_t DRAIN_LIMIT_NS = 200000000ull;   // 0.2 s per wait while draining after a failure
constexpr int WARP_HDR_BYTES = 256;                  // 8 mbarriers + 32 mask words

struct TileGeom {
    int k0, k1, i0, i1;  // nonzeros [k0, k1), end events [i0, i1)
    int kb0, ncov;       // staged nonzero cover [kb0, kb0 + ncov), kb0 = k0 rounded down to 8
    int off_val, off_ptr, off_x;
    int pbase, npc;      // staged pointer cover [pbase, pbase + npc)
    int xbase, nxc;      // staged major-vector cover
    int bytes;
    bool win_smem;       // pointer/major windows staged (else read from global memory)
};

template <typename VT, typename XT, int MODE>
__device__ __forceinline__ TileGeom tile_geom(const StreamParams &p, const ChunkDev &cd, int t) {
    TileGeom g;
    const int2 a = p.tiles[t];
    g.k0 = a.x;
    g.i0 = a.y;
    if (t + 1 < cd.tile_end) {
        const int2 b = p.tiles[t + 1];
        g.k1 = b.x;
        g.i1 = b.y;
    } else {
        g.k1 = cd.nz_end;
        g.i1 = cd.e_end;
    }
    g.kb0 = g.k0 & ~7;
    g.ncov = ((g.k1 + 7) & ~7) - g.kb0;
    g.off_val = g.ncov * 4;
    g.off_ptr = g.off_val + g.ncov * (int)sizeof(VT);
    g.pbase = g.i0 & ~3;
    g.npc = ((g.i1 + 1 + 3) & ~3) - g.pbase;
    g.off_x = g.off_ptr + g.npc * 4;
    g.bytes = g.off_x;
    g.xbase = 0;
    g.nxc = 0;
    if (MODE != MODE_SEGDOT) {
        constexpr int xa = 16 / (int)sizeof(XT);
        const int last = min(g.i1, p.n_major - 1);
        if (last >= g.i0) {
            g.xbase = g.i0 & ~(xa - 1);
            g.nxc = ((last + 1 + xa - 1) & ~(xa - 1)) - g.xbase;
        }
        const int nvec = (MODE == MODE_DVALUES) ? 1 : p.kb;
        g.bytes = g.off_x + nvec * g.nxc * (int)sizeof(XT);
    }
    g.win_smem = g.bytes <= p.stage_bytes;
    return g;
}

// A descriptor that would overrun the stage or the 1024-position head mask is
// refused (error word) instead of staged; it cannot occur for a plan built by
// the set-up kernels.
__device__ __forceinline__ bool tile_ok(const TileGeom &g, const StreamParams &p) {
    return g.k1 >= g.k0 && g.i1 >= g.i0 && g.k0 >= 0 && g.k1 <= p.nnz && g.i1 <= p.n_major && g.ncov <= 1024 &&
           g.ncov < p.table_bytes / 4 && g.off_ptr <= p.stage_bytes;
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

struct CopyList {
    const void *src[2 + KB_MAX];
    void *dst[2 + KB_MAX];
    uint32_t bytes[2 + KB_MAX];
    int n;
    uint32_t tx;
};

// Plan the staging of elements [e0, e0 + cnt) of an array of `len` elements of
// `es` bytes into dst (e0 a multiple of 16/es): the part below the last
// 16-byte boundary of the array goes by bulk copy, the rest (at most 15 bytes
// at the very end of the array) is copied here with plain loads.
__device__ __forceinline__ void stage_range(CopyList &cl, unsigned char *dst, const void *src, long e0, int cnt,
                                            long len, int es) {
    const long al = 16 / es;
    const long lim = len & ~(al - 1);
    const long end = e0 + cnt;
    const long bend = end < lim ? end : lim;
    if (bend > e0) {
        cl.src[cl.n] = static_cast<const unsigned char *>(src) + e0 * es;
        cl.dst[cl.n] = dst;
        cl.bytes[cl.n] = static_cast<uint32_t>((bend - e0) * es);
        cl.tx += cl.bytes[cl.n];
        ++cl.n;
    }
    const long t0 = e0 > lim ? e0 : lim;
    const long t1 = end < len ? end : len;
    for (long e = t0; e < t1; ++e)
        copy_elem(dst + (e - e0) * es, static_cast<const unsigned char *>(src) + e * es, es);
}

// Issued by lane 0 of the owning warp.
template <typename VT, typename XT, int MODE>
__device__ __forceinline__ void issue_tile(const StreamParams &p, const ChunkDev &cd, int t, unsigned char *st,
                                        uint64_t *bar, int pptr_len) {
    const TileGeom g = tile_geom<VT, XT, MODE>(p, cd, t);
    CopyList cl;
    cl.n = 0;
    cl.tx = 0;
    if (!tile_ok(g, p)) {
        mbar_arrive_expect_tx(bar, 0);
        return;
    }
    stage_range(cl, st, p.idx, g.kb0, g.ncov, p.nnz, 4);
    stage_range(cl, st + g.off_val, p.vals, g.kb0, g.ncov, p.nnz, (int)sizeof(VT));
    if (g.win_smem) {
        stage_range(cl, st + g.off_ptr, p.pptr, g.pbase, g.npc, pptr_len, 4);
        if (MODE != MODE_SEGDOT && g.nxc > 0) {
            const int nvec = (MODE == MODE_DVALUES) ? 1 : p.kb;
            for (int b = 0; b < nvec; ++b) {
                const void *src = (MODE == MODE_DVALUES) ? p.vin[1] : p.vin[b];
                stage_range(cl, st + g.off_x + b * g.nxc * (int)sizeof(XT), src, g.xbase, g.nxc, p.n_major,
                            (int)sizeof(XT));
            }
        }
    }
    // The arrive releases the plain stores above; the bulk copies complete the transaction count.
    mbar_arrive_expect_tx(bar, cl.tx);
    for (int i = 0; i < cl.n; ++i) bulk_g2s(cl.dst[i], cl.src[i], cl.bytes[i], bar);
}

template <typename XT> __device__ __forceinline__ XT zero_of() { return XT(0); }

template <typename VT, typename XT, int MODE, int KB, bool SMEMV>
__global__ void __launch_bounds__(MAX_WARPS * 32, 1) stream_kernel(const __grid_constant__ StreamParams p) {
    const int pptr_len = p.pptr_len;
    const int table_bytes = p.table_bytes;
    using AT = typename Acc<VT>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int kb = (MODE == MODE_DVALUES) ? 1 : p.kb;

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
        uint32_t *mask = reinterpret_cast<uint32_t *>(wbase + 128);
        int32_t *table = reinterpret_cast<int32_t *>(wbase + WARP_HDR_BYTES);
        unsigned char *stages = wbase + WARP_HDR_BYTES + table_bytes;
        const int S = p.stages;
        const int nt = cd.tile_end - cd.tile_begin;
        double carry[KB];
#pragma unroll
        for (int b = 0; b < KB; ++b) carry[b] = 0.0;

        // Emit the finished dot product of segment `col` for vector b (SEGDOT):
        // the first segment of a chunk that shares it with its left neighbour
        // goes to the chunk's left carry record (Sec. IV-A), the rest to out.
        auto emit = [&](int col, int b, double value) {
            if (needLeft && col == cd.jf)
                p.rec_left[b * p.P + c] = value;
            else
                static_cast<XT *>(p.vout[b])[col] = from_d<XT>(value);
        };

        if (nt > 0) {
            if (lane == 0) {
                for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
                fence_mbar_init();
            }
            __syncwarp();
            if (lane == 0) {
                for (int q = 0; q < S && q < nt; ++q)
                    issue_tile<VT, XT, MODE>(p, cd, cd.tile_begin + q, stages + q * p.stage_bytes, &bars[q],
                                             pptr_len);
            }
            for (int q = 0; q < nt; ++q) {
                const int t = cd.tile_begin + q;
                const int s = q % S;
                unsigned char *st = stages + s * p.stage_bytes;
                bool ok = mbar_wait_bounded(&bars[s], (q / S) & 1, WAIT_LIMIT_NS);
                ok = __all_sync(FULL, ok);
                if (!ok) {
                    if (lane == 0) {
                        atomicOr(p.err, ERR_WAIT);
                        for (int r = q; r < nt && r < q + S; ++r)
                            mbar_wait_bounded(&bars[r % S], (r / S) & 1, DRAIN_LIMIT_NS);
                    }
                    __syncwarp();
                    break;
                }
                const TileGeom g = tile_geom<VT, XT, MODE>(p, cd, t);
                if (!tile_ok(g, p)) {
                    if (lane == 0) atomicOr(p.err, ERR_STRUCT);
                    __syncwarp();
                    if (lane == 0 && q + S < nt) {
                        fence_proxy_async_smem();
                        issue_tile<VT, XT, MODE>(p, cd, t + S, st, &bars[s], pptr_len);
                    }
                    continue;
                }
                const int rel_lo = g.k0 - g.kb0;
                const int rel_hi = g.k1 - g.kb0;
                const int32_t *idx_s = reinterpret_cast<const int32_t *>(st);
                const unsigned char *val_s = st + g.off_val;
                const int32_t *ptr_s = reinterpret_cast<const int32_t *>(st + g.off_ptr);
                const XT *x_s = reinterpret_cast<const XT *>(st + g.off_x);

                // ---- A. segment starts inside the tile -> head bits (positions relative to kb0)
                mask[lane] = 0u;
                __syncwarp();
                bool dup = false;
                for (int jb = g.i0 + 1; jb <= g.i1; jb += 32) {
                    const int j = jb + lane;
                    if (j <= g.i1) {
                        const int pj = g.win_smem ? ptr_s[j - g.pbase] : p.pptr[j];
                        const int pos = pj - g.kb0;
                        if (pos >= 0 && pos < rel_hi) atomicOr(&mask[pos >> 5], 1u << (pos & 31));
                        if (j < g.i1) {
                            const int pn = g.win_smem ? ptr_s[j + 1 - g.pbase] : p.pptr[j + 1];
                            if (pn == pj) {  // empty segment j (its end event is in this tile)
                                dup = true;
                                if constexpr (MODE == MODE_SEGDOT) {
                                    for (int b = 0; b < kb; ++b) static_cast<XT *>(p.vout[b])[j] = zero_of<XT>();
                                }
                            }
                        }
                    }
                }
                dup = __any_sync(FULL, dup);
                __syncwarp();
                const uint32_t mw = mask[lane];
                int incl = __popc(mw);
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, d);
                    if (lane >= d) incl += v;
                }
                const int cnt_ex = incl - __popc(mw);
                const int htotal = __shfl_sync(FULL, incl, 31);
                if (dup) {
                    // several segments start at one position: map head number -> segment id
                    for (int jb = g.i0 + 1; jb <= g.i1; jb += 32) {
                        const int j = jb + lane;
                        const bool in = j <= g.i1;
                        int pj = 0, pos = 0x7fffffff;
                        bool last_at = false;
                        if (in) {
                            pj = g.win_smem ? ptr_s[j - g.pbase] : p.pptr[j];
                            pos = pj - g.kb0;
                            const int pn =
                                (j == g.i1) ? -1 : (g.win_smem ? ptr_s[j + 1 - g.pbase] : p.pptr[j + 1]);
                            last_at = pos >= 0 && pos < rel_hi && pn != pj;
                        }
                        const int w = last_at ? (pos >> 5) : 0;
                        const uint32_t mww = __shfl_sync(FULL, mw, w);
                        const int cww = __shfl_sync(FULL, cnt_ex, w);
                        if (last_at) table[cww + __popc(mww & (FULL >> (31 - (pos & 31))))] = j;
                    }
                    __syncwarp();
                }
                // segment of the item preceded (inclusively) by h head bits in this tile
                auto colh = [&](int h) -> int { return h == 0 ? g.i0 : (dup ? table[h] : g.i0 + h); };

                // ---- B. 128 positions per step, 4 consecutive per lane
                const int nsteps = (rel_hi + 127) >> 7;
                for (int stp = 0; stp < nsteps; ++stp) {
                    const int p0 = (stp << 7) + (lane << 2);
                    const int w = p0 >> 5;
                    const uint32_t mwl = __shfl_sync(FULL, mw, w);
                    const int cwl = __shfl_sync(FULL, cnt_ex, w);
                    const uint32_t hb = (mwl >> (p0 & 31)) & 0xFu;
                    const int base = cwl + __popc(mwl & ((1u << (p0 & 31)) - 1u));
                    const bool any_valid = (p0 + 3 >= rel_lo) && (p0 < rel_hi);
                    int ix[4] = {0, 0, 0, 0};
                    AT va[4] = {AT(0), AT(0), AT(0), AT(0)};
                    if (any_valid) {
                        const int4 qi = reinterpret_cast<const int4 *>(idx_s)[p0 >> 2];
                        ix[0] = qi.x;
                        ix[1] = qi.y;
                        ix[2] = qi.z;
                        ix[3] = qi.w;
                        Load4<VT, AT>::run(val_s, p0, va);
                    }
                    bool valid[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        valid[e] = (p0 + e >= rel_lo) && (p0 + e < rel_hi);
                        if (valid[e] && static_cast<unsigned>(ix[e]) >= static_cast<unsigned>(p.n_minor)) {
                            atomicOr(p.err, ERR_INDEX);
                            valid[e] = false;
                        }
                    }

                    if constexpr (MODE == MODE_SEGDOT) {
                        AT prod[4][KB];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
#pragma unroll
                            for (int b = 0; b < KB; ++b) {
                                AT w_ = AT(0);
                                if (valid[e]) {
                                    if constexpr (SMEMV) {
                                        w_ = static_cast<AT>(reinterpret_cast<const XT *>(smem)[ix[e] * KB + b]);
                                    } else {
                                        w_ = (b < kb) ? static_cast<AT>(__ldg(static_cast<const XT *>(p.vin[b]) + ix[e]))
                                                      : AT(0);
                                    }
                                }
                                prod[e][b] = va[e] * w_;
                            }
                        }
                        AT lead[KB], run[KB];
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            lead[b] = AT(0);
                            run[b] = AT(0);
                        }
                        int nh = 0, h = base;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if ((hb >> e) & 1u) {
                                if (nh == 0) {
#pragma unroll
                                    for (int b = 0; b < KB; ++b) lead[b] = run[b];
                                } else {
                                    const int col = colh(h);
                                    for (int b = 0; b < kb; ++b) emit(col, b, static_cast<double>(run[b]));
                                }
                                ++h;
                                ++nh;
#pragma unroll
                                for (int b = 0; b < KB; ++b) run[b] = AT(0);
                            }
#pragma unroll
                            for (int b = 0; b < KB; ++b) run[b] += prod[e][b];
                        }
                        if (nh == 0) {
#pragma unroll
                            for (int b = 0; b < KB; ++b) lead[b] = run[b];
                        }
                        // warp segmented scan of the lanes' open sums (the o operator of Sec. IV-B)
                        const unsigned bal = __ballot_sync(FULL, nh > 0);
                        const unsigned le = bal & (FULL >> (31 - lane));
                        const int seg_start = le ? (31 - __clz(le)) : 0;
                        const bool before = (bal & ((1u << lane) - 1u)) != 0;
                        const int lead_col = colh(base);
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            AT T = nh ? run[b] : lead[b];
#pragma unroll
                            for (int d = 1; d < 32; d <<= 1) {
                                const AT v = __shfl_up_sync(FULL, T, d);
                                if (lane - d >= seg_start && lane >= d) T += v;
                            }
                            AT Tex = __shfl_up_sync(FULL, T, 1);
                            if (lane == 0) Tex = AT(0);
                            if (nh > 0 && b < kb) {
                                const double value = static_cast<double>(Tex + lead[b]) + (before ? 0.0 : carry[b]);
                                emit(lead_col, b, value);
                            }
                            const AT T31 = __shfl_sync(FULL, T, 31);
                            carry[b] = bal ? static_cast<double>(T31) : carry[b] + static_cast<double>(T31);
                        }
                    } else if constexpr (MODE == MODE_SCATTER) {
                        int h = base;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if ((hb >> e) & 1u) ++h;
                            if (valid[e]) {
                                const int col = colh(h);
                                for (int b = 0; b < kb; ++b) {
                                    const XT xv = g.win_smem ? x_s[b * g.nxc + col - g.xbase]
                                                             : static_cast<const XT *>(p.vin[b])[col];
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
                    } else {  // MODE_DVALUES
                        int h = base;
                        VT *gout = static_cast<VT *>(p.vout[0]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if ((hb >> e) & 1u) ++h;
                            if (valid[e]) {
                                const int col = colh(h);
                                const XT xv = g.win_smem ? x_s[col - g.xbase] : static_cast<const XT *>(p.vin[1])[col];
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

                // ---- C. tile end: a segment whose end event lies in this tile is complete
                if constexpr (MODE == MODE_SEGDOT) {
                    const int col_last = (rel_hi > rel_lo) ? colh(htotal) : g.i0;
                    if (col_last < g.i1) {
                        if (lane == 0)
                            for (int b = 0; b < kb; ++b) emit(col_last, b, carry[b]);
#pragma unroll
                        for (int b = 0; b < KB; ++b) carry[b] = 0.0;
                    }
                }
                __syncwarp();
                if (lane == 0 && q + S < nt) {
                    fence_proxy_async_smem();
                    issue_tile<VT, XT, MODE>(p, cd, t + S, st, &bars[s], pptr_len);
                }
            }
        }
        if constexpr (MODE == MODE_SEGDOT) {
            // the chunk's last segment continues in the next chunk: right carry record
            if (needRight && lane == 0)
                for (int b = 0; b < kb; ++b) p.rec_right[b * p.P + c] = carry[b];
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
