// Streaming kernel: the nonzeros are cut into equal-count tiles of T nonzeros;
// each CTA takes a contiguous range of tiles by the Sec. II rule and cuts it into
// chunks: nb chunks of C consecutive tiles, then a tail of single-tile chunks
// (at least MAX_WARPS (C + 1) tiles, when the CTA has that many).  The chunks are
// the "processors" of Sec. II: contiguous groups of nonzeros, each owning its own
// overlap-zone records; they do not depend on the number of warps of a pass, so a
// vector's sums come out the same in single- and multi-vector passes.  Warp w of
// W takes the C-tile chunks w, w + W, w + 2W, ... (the CTA's warps stream
// neighbouring parts of the arrays at any time), then a contiguous run of tail
// tiles that brings every warp to the same tile count, give or take one.
// Every warp streams its own tiles through S shared-memory slots of its own:
// when it has finished a tile it issues the bulk (TMA) copies of the tile S
// ahead into the freed slot (one copy per array: indices, values, segment-start
// masks and, for the scatter and gradient modes, the window of the long vector
// the tile needs), so no warp ever waits for another.
//
// Terms.  "major" is the compressed dimension (columns of a wide CSC matrix,
// rows of a tall CSR matrix), "minor" the indexed one.  Segment j ends after
// its last nonzero, and its end event is ordered before the nonzero at
// position ptr[j+1].  Tile t covers nonzeros [nzb, nze) and owns the end
// events [i0, i1) (TileMeta), so its nonzeros lie in segments i0..i1.
//
//   MODE_SCATTER: acc[idx[k]] += val[k] * w[seg(k)]  -- A_(i) x_(i) of Sec. III
//                 (wide CSC y = A x; tall CSR u = v^T A by role reversal), into
//                 an on-chip copy of the short vector per CTA.
//   MODE_SEGDOT:  out[j] = sum_k val[k] * w[idx[k]] over segment j -- v^T A_(i)
//                 of Sec. IV-A (wide CSC u^T = v^T A; tall CSR y = A x).  A
//                 segment that runs on from one tile of a chunk into the next is
//                 carried in registers; the first and last segments of a chunk
//                 that continue in the neighbouring chunks (overlap zones) leave
//                 their partial sums in the chunk's carry records for the zone
//                 fixup.
//   MODE_VSEG:    MODE_SEGDOT for several vectors in one pass: a lane group of VL lanes
//                 holds one vector per lane, and each lane forms its vector's sums with
//                 the same operations in the same order as the single-vector pass, so
//                 every vector's result equals its single-vector product bit for bit.
//   MODE_DVALUES: g[k] = minor[idx[k]] * major[seg(k)].
#pragma once

#include "device_common.cuh"
#include "internal.h"

namespace gbk {

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per pipeline wait

__device__ __forceinline__ void copy_elem(unsigned char *d, const unsigned char *s, int es) {
    if (es == 8) {
        *reinterpret_cast<unsigned long long *>(d) = *reinterpret_cast<const unsigned long long *>(s);
    } else if (es == 4) {
        *reinterpret_cast<unsigned int *>(d) = *reinterpret_cast<const unsigned int *>(s);
    } else {
        *reinterpret_cast<unsigned short *>(d) = *reinterpret_cast<const unsigned short *>(s);
    }
}

template <typename XT> __device__ __forceinline__ XT zero_of() { return XT(0); }

// A product rounded on its own (never fused into a following addition), so that the
// segmented passes round every product the same way whatever code surrounds it.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// hi + lo += t, compensated (TwoSum: hi takes the rounded sum, lo gathers its rounding
// errors).  A sum that is infinite or NaN carries no error term, so that hi + lo stays what the
// plain sum gives (an infinity would otherwise make the error term NaN).
template <typename AT>
__device__ __forceinline__ void carry_in(AT &hi, AT &lo, AT t) {
    const AT s_ = hi + t;
    const AT bp = s_ - hi;
    const AT err = (hi - (s_ - bp)) + (t - bp);
    lo += isfinite(s_) ? err : AT(0);
    hi = s_;
}

// carry records: (hi, lo) of the accumulation type, widened to FP64 by the zone fixup
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };
__device__ __forceinline__ float2 make_pair2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 make_pair2(double a, double b) { return make_double2(a, b); }

// KB consecutive vector entries at a 16-byte aligned address (KB >= 2), by vector loads
// through the read-only path.
template <typename XT, int KB> struct Gather {
    __device__ __forceinline__ static void run(const XT *src, XT (&w)[KB]) {
        static_assert(sizeof(XT) * KB % 16 == 0 || sizeof(XT) * KB == 8, "vector loads of whole 8/16 bytes");
        if constexpr (sizeof(XT) * KB == 8) {
            const uint2 q = __ldg(reinterpret_cast<const uint2 *>(src));
            const unsigned u[2] = {q.x, q.y};
            memcpy(w, u, 8);
        } else {
#pragma unroll
            for (int h = 0; h < (int)(sizeof(XT) * KB / 16); ++h) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(src) + h);
                const unsigned u[4] = {q.x, q.y, q.z, q.w};
                memcpy(reinterpret_cast<unsigned char *>(w) + 16 * h, u, 16);
            }
        }
    }
};

template <bool B> struct BoolC {
    static constexpr bool value = B;
};
struct RtBool {  // a flag known only at run time, passed where a BoolC may be
    bool value;
};

// WB: the most warps a launch of this instantiation may have (its register budget).
template <typename VT, typename XT, int MODE, int KB, bool SMEMV, int WB>
__global__ void __launch_bounds__(WB * 32, 1) stream_kernel(const __grid_constant__ StreamParams p) {
    using AT = typename Acc<VT>::type;
    constexpr bool SEGM = MODE == MODE_SEGDOT || MODE == MODE_VSEG;  // a segmented (dot-product) pass
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int kb = (MODE == MODE_DVALUES) ? 1 : p.kb;
    const int nvec = (MODE == MODE_DVALUES) ? 1 : p.kb;
    const int S = p.slots;
    const unsigned n_minor = static_cast<unsigned>(p.n_minor);

    uint64_t *myfull = reinterpret_cast<uint64_t *>(smem + p.vec_region_bytes) + warp * S;
    unsigned char *myslots = smem + p.vec_region_bytes + BAR_BYTES + (size_t)warp * S * p.slot_bytes;

    // Blocks: the grid's G BPC consecutive ranges of whole tiles, equal by the Sec. II rule
    // (BPC = 1 but for the windowed pass over row-sorted blocks); this CTA runs blocks
    // BPC g .. BPC g + BPC - 1 one after the other.  A block's tiles [ta, ta + nct) form nb
    // chunks of C tiles and then nct - nb C single-tile chunks.
    const int BPC = p.blocks_per_cta;
    const int GB = gridDim.x * BPC;
    const int tq = p.ntiles / GB, tr = p.ntiles % GB;
    const int C = p.chunk_tiles;
    auto big_chunks = [&](int n) { return (n - min(n, MAX_WARPS * C + MAX_WARPS)) / C; };
    // processors (chunks) before a block: a block of n tiles has big_chunks(n) + n - C big_chunks(n)
    auto chunks_of = [&](int n) { return n - (C - 1) * big_chunks(n); };
    int gb = 0, ta = 0, nb = 0, cnt = 0, nk = 0, toff = 0, chunk0 = 0;
    auto enter_block = [&](int hb) {
        gb = blockIdx.x * BPC + hb;
        ta = gb * tq + min(gb, tr);
        const int nct = tq + (gb < tr ? 1 : 0);
        nb = big_chunks(nct);
        cnt = nb / W + (warp < nb % W ? 1 : 0);   // C-tile chunks of this warp
        nk = nct / W + (warp < nct % W ? 1 : 0);  // tiles of this warp
        // first tail tile of this warp: the tiles of the warps before it less their C-tile chunks
        toff = (warp * (nct / W) + min(warp, nct % W)) - C * (warp * (nb / W) + min(warp, nb % W));
        chunk0 = gb * chunks_of(tq) + min(gb, tr) * (chunks_of(tq + 1) - chunks_of(tq));
    };
    auto tile_of = [&](int k) {  // tile of this warp's k-th tile of the block
        if constexpr (!SEGM) return ta + warp + k * W;  // no carries: the block's tiles round-robin
        return k < cnt * C ? ta + (warp + (k / C) * W) * C + k % C : ta + nb * C + toff + (k - cnt * C);
    };

    // this warp's slot barriers (used by this warp only)
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&myfull[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // ---- tile descriptors of this warp, 32 per batch: lane j holds tile 32 * batch + j: its
    // nzb, e_begin, flags and the next tile's nzb (d); the next tile's e_begin, the tile's
    // number and its chunk's processor number and place (e: proc << 2 | first | last << 1),
    // worked out here once per 32 tiles
    int4 dcur = make_int4(0, 0, 0, 0), dnxt = make_int4(0, 0, 0, 0);
    int4 ecur = make_int4(0, 0, 0, 0), enxt = make_int4(0, 0, 0, 0);
    auto load_batch = [&](int bi, int4 &d, int4 &e) {
        const int k = (bi << 5) + lane;
        if (k < nk) {
            const int t = tile_of(k);
            const TileMeta a = p.meta[t];
            const TileMeta b = p.meta[t + 1];
            d = make_int4(a.nzb, a.e_begin, a.flags, b.nzb);
            const bool in_big = k < cnt * C;
            const int q = k / C, o = k - q * C;
            const int first = in_big ? (o == 0) : 1;
            const int last = in_big ? (o == C - 1) : 1;
            const int proc = chunk0 + (in_big ? warp + q * W : nb + toff + (k - cnt * C));
            e = make_int4(b.e_begin, t, (proc << 2) | first | (last << 1), 0);
        }
    };
    int cb = 0;  // batch held in dcur
    // descriptor of this warp's tile k (its batch is cb or cb + 1)
    auto desc = [&](int k, int4 &d, int4 &e) {
        const bool c = (k >> 5) == cb;
        const int src = k & 31;
        d.x = __shfl_sync(FULL, c ? dcur.x : dnxt.x, src);
        d.y = __shfl_sync(FULL, c ? dcur.y : dnxt.y, src);
        d.z = __shfl_sync(FULL, c ? dcur.z : dnxt.z, src);
        d.w = __shfl_sync(FULL, c ? dcur.w : dnxt.w, src);
        e.x = __shfl_sync(FULL, c ? ecur.x : enxt.x, src);
        e.y = __shfl_sync(FULL, c ? ecur.y : enxt.y, src);
        e.z = __shfl_sync(FULL, c ? ecur.z : enxt.z, src);
    };
    // window [xbase, xbase + nxc) of the long vector covering segments i0..i1 (16-byte aligned)
    auto xwindow = [&](int i0, int i1, int &xbase, int &nxc) {
        xbase = 0;
        nxc = 0;
        if constexpr (!SEGM) {
            constexpr int xa = 16 / (int)sizeof(XT);
            const int last = min(i1, p.n_major - 1);
            if (last >= i0) {
                xbase = i0 & ~(xa - 1);
                nxc = ((last + 1 + xa - 1) & ~(xa - 1)) - xbase;
            }
        }
    };
    // Every lane copies one array for the whole kernel: lane 0 indices, 1 values,
    // 2 segment-start masks, 3.. long-vector windows (one per vector).  Its source,
    // element size and destination offset within a slot are fixed.
    const unsigned char *c_src = reinterpret_cast<const unsigned char *>(p.idx);
    int c_off = 0, c_len = p.nnz, c_es = 4;
    bool c_x = false;  // a long-vector window lane in use
    if (lane == 1) {
        c_src = static_cast<const unsigned char *>(p.vals);
        c_off = p.off_val;
        c_es = (int)sizeof(VT);
    } else if (lane == 2) {
        c_src = reinterpret_cast<const unsigned char *>(p.masks);
        c_off = p.off_mask;
        c_len = p.ntiles * p.mwp;
    } else if (SEGM && lane == 3) {  // the segmented modes: the tile's head-count prefix table
        c_src = reinterpret_cast<const unsigned char *>(p.pfx);
        c_off = p.off_pfx;
        c_len = p.ntiles * p.mwq;
        c_es = 2;
    } else if (lane >= 3) {
        const int b = lane - 3;
        c_src = static_cast<const unsigned char *>((MODE == MODE_DVALUES) ? p.vin[1] : p.vin[b < KB_MAX ? b : 0]);
        c_off = p.off_x + b * p.x_cap * (int)sizeof(XT);
        c_len = p.n_major;
        c_es = (int)sizeof(XT);
        c_x = !SEGM && b < nvec;
    }
    const int c_lim = c_len & ~(16 / c_es - 1);  // the array's last 16-byte boundary (in elements)
    // issue the copies of tile k into slot s
    auto issue = [&](int k, int s) {
        int4 d, e;
        desc(k, d, e);
        const int e1 = e.x;
        const int kb0 = d.x & ~7;
        const int ncov = ((d.w + 7) & ~7) - kb0;
        int xbase, nxc;
        xwindow(d.y, e1, xbase, nxc);
        int e0 = kb0, cnt = ncov;
        if (lane == 2) {
            e0 = e.y * p.mwp;
            cnt = p.mwp;
        } else if (SEGM && lane == 3) {
            e0 = e.y * p.mwq;
            cnt = p.mwq;
        } else if (lane >= 3) {
            e0 = xbase;
            cnt = (c_x && nxc <= p.x_cap) ? nxc : 0;
        }
        if (ncov < 0 || ncov > p.tile_cap) cnt = 0;
        unsigned char *dst = myslots + (size_t)s * p.slot_bytes + c_off;
        // the part below the array's last 16-byte boundary by bulk copy, the rest
        // (at most 15 bytes at the very end of an array) by plain loads
        const int end = e0 + cnt;
        const int bend = min(end, c_lim);
        const uint32_t bytes = bend > e0 ? static_cast<uint32_t>(bend - e0) * c_es : 0u;
        if (cnt > 0 && end > c_lim) {
            const int tl = min(end, c_len);
            for (int e = max(e0, c_lim); e < tl; ++e)
                copy_elem(dst + (size_t)(e - e0) * c_es, c_src + (size_t)e * c_es, c_es);
        }
        const uint32_t total = __reduce_add_sync(FULL, bytes);
        if (lane == 0) {  // the tile's header, read by this warp when it processes the tile
            int4 *hd = reinterpret_cast<int4 *>(myslots + (size_t)s * p.slot_bytes + p.off_hdr);
            hd[0] = d;
            hd[1] = make_int4(e1, xbase, nxc, e.z);
        }
        __syncwarp();
        // releases the header and the plain stores; the bulk bytes complete the phase
        if (lane == 0) mbar_arrive_expect_tx(&myfull[s], total);
        if (bytes) bulk_g2s(dst, c_src + (size_t)e0 * c_es, bytes, &myfull[s]);
    };

    // ---- the short (minor) vector on chip: accumulator (SCATTER) or input (SEGDOT / DVALUES):
    // the whole vector, or block gbk's window of it (row-sorted blocks; its first element is
    // 16-byte aligned).  Called by all threads; one vector goes by bulk copies on the barrier
    // sbar, whose phases sphase counts.
    uint64_t *sbar = reinterpret_cast<uint64_t *>(smem + p.vec_region_bytes + BAR_BYTES) - 1;
    uint32_t sphase = 0;
    // VSEG: the short vectors interleaved ([entry][VL], a whole entry VL * 4 bytes) follow the
    // lanes' scratch at the start of the region
    constexpr int VSCR_BYTES = WARPS_VSEG * 32 * 8 * 4;
    constexpr bool BULKV = SMEMV && (MODE == MODE_VSEG || (MODE != MODE_SCATTER && KB == 1));
    if (BULKV && threadIdx.x == 0) {
        mbar_init(sbar, 1);
        fence_mbar_init();
    }
    auto stage_vector = [&](int gbk) {
        if constexpr (SMEMV && MODE != MODE_SCATTER) {
            constexpr int EW = MODE == MODE_VSEG ? KB : 1;  // values per entry of the staged vector
            XT *vs = reinterpret_cast<XT *>(smem + (MODE == MODE_VSEG ? VSCR_BYTES : 0));
            int wb = 0, wl = p.n_minor;
            if (p.win) {
                const int2 w = p.win[gbk];
                wb = w.x;
                wl = min(w.y, p.n_minor);
            }
            if constexpr (BULKV) {
                // its 16-byte aligned part by bulk copies, the rest (under 16 bytes) by plain loads
                const XT *src = static_cast<const XT *>(p.vin[0]) + (size_t)wb * EW;
                constexpr int xa = (16 / (int)sizeof(XT) + EW - 1) / EW;  // entries per 16 bytes (at least 1)
                const int wbulk = wl & ~(xa - 1);
                if (threadIdx.x == 0 && wbulk > 0) {
                    mbar_arrive_expect_tx(sbar, static_cast<uint32_t>(wbulk) * EW * (uint32_t)sizeof(XT));
                    constexpr int piece = 32768 / (int)sizeof(XT);
                    const int total = wbulk * EW;
                    for (int o = 0; o < total; o += piece)
                        bulk_g2s(vs + o, src + o, static_cast<uint32_t>(min(piece, total - o)) * (uint32_t)sizeof(XT),
                                 sbar);
                }
                for (int i = wbulk * EW + threadIdx.x; i < wl * EW; i += blockDim.x) vs[i] = src[i];
                __syncthreads();  // the barrier's initialisation before anyone waits on it
                if (wbulk > 0) {
                    if (!mbar_wait_bounded(sbar, sphase & 1u, WAIT_LIMIT_NS)) {
                        if (threadIdx.x == 0) atomicOr(p.err, ERR_WAIT);
                        mbar_wait_bounded(sbar, sphase & 1u, WAIT_LIMIT_NS);  // let the copy land first
                    }
                    ++sphase;
                }
            } else {
                for (int i = threadIdx.x; i < wl; i += blockDim.x) {
#pragma unroll
                    for (int b = 0; b < KB; ++b)
                        vs[i * KB + b] = (b < kb) ? static_cast<const XT *>(p.vin[b])[wb + i] : zero_of<XT>();
                }
            }
        }
    };
    if constexpr (SMEMV && MODE == MODE_SCATTER) {
        AT *acc = reinterpret_cast<AT *>(smem);
        for (int i = threadIdx.x; i < p.n_minor * KB; i += blockDim.x) acc[i] = AT(0);
    }

    // the open segment at the start of the current chunk: its first segment, and whether that
    // began in the previous chunk (then its sum goes to the chunk's left record)
    int cfirst = -1;
    bool cleft = false;
    // first element of the current block's window of the input vector (row-sorted blocks)
    int vwin = 0;
    // running sum of the open segment (SEGDOT): compensated (hi + lo) in the accumulation
    // type, carried from one of this warp's tiles into the next while the segment runs on
    AT chi[KB], clo[KB];

    int s = 0;        // slot of the warp's next tile to consume
    uint32_t ph = 0;  // phase parity of that slot's barrier
    bool wfail = false;  // a staging wait of this warp timed out: it does no more work
    for (int hb = 0; hb < BPC; ++hb) {
    enter_block(hb);
    cb = 0;
    load_batch(0, dcur, ecur);
    load_batch(1, dnxt, enxt);
    if (!wfail)
        for (int k = 0; k < min(S, nk); ++k) issue(k, (s + k) % S);  // the first copies fly while the vector is staged
    if (hb == 0 || p.win) {
        if (hb > 0) __syncthreads();  // every warp is done with the previous block's window
        stage_vector(gb);
    }
    __syncthreads();
    cfirst = -1;
    cleft = false;
    vwin = (SEGM && p.win) ? p.win[gb].x : 0;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
        chi[b] = AT(0);
        clo[b] = AT(0);
    }

    for (int k = 0; k < nk && !wfail; ++k) {
        unsigned char *slot = myslots + (size_t)s * p.slot_bytes;
        bool ok = mbar_wait_bounded(&myfull[s], ph, WAIT_LIMIT_NS);
        ok = __all_sync(FULL, ok);
        if (!ok) {
            if (lane == 0) atomicOr(p.err, ERR_WAIT);
            // let the copies still in flight into this warp's slots land before leaving
            for (int q = 0; q < min(S, nk - k); ++q) {
                const int qs = s + q < S ? s + q : s + q - S;
                mbar_wait_bounded(&myfull[qs], s + q < S ? ph : ph ^ 1u, WAIT_LIMIT_NS);
            }
            wfail = true;
            break;
        }
        // tile header: first nonzero, first owned end event, flags, next tile's first
        // nonzero; next tile's first end event, long-vector window base and length
        const int4 d = reinterpret_cast<const int4 *>(slot + p.off_hdr)[0];
        const int4 d1 = reinterpret_cast<const int4 *>(slot + p.off_hdr)[1];
        const int kb0 = d.x & ~7;
        const int ncov = ((d.w + 7) & ~7) - kb0;
        if (ncov < 0 || ncov > p.tile_cap) {
            if (lane == 0) atomicOr(p.err, ERR_STRUCT);
        } else {
            {
                const int i0 = d.y, i1 = d1.x;
                // position of the tile in its chunk; the chunk's first segment started in the
                // previous chunk (left record) and its last continues in the next (right record)
                // by the flags of the chunk's first and last tiles
                const bool chunk_first = (d1.w & 1) != 0;
                const bool chunk_last = (d1.w & 2) != 0;
                const int proc = d1.w >> 2;
                if (chunk_first) {
                    cfirst = i0;
                    cleft = (d.z & 1) != 0;
                }
                const bool needRight = chunk_last && (d.z & 2) != 0;
                const bool dup = (d.z & 4) != 0;
                const int xbase = d1.y;
                const bool win = d1.z <= p.x_cap;
                const int rel_lo = d.x - kb0;
                const int rel_hi = d.w - kb0;
                const bool full = rel_lo == 0 && (rel_hi & 255) == 0;  // whole 256-position steps only
                const int32_t *idx_s = reinterpret_cast<const int32_t *>(slot);
                const unsigned char *val_s = slot + p.off_val;
                const uint32_t *mask_s = reinterpret_cast<const uint32_t *>(slot + p.off_mask);
                const XT *x_s = reinterpret_cast<const XT *>(slot + p.off_x);
                const uint16_t *pfx_s = reinterpret_cast<const uint16_t *>(slot + p.off_pfx);  // segmented modes
                const uint32_t mw = lane < p.mwp ? mask_s[lane] : 0u;
                bool idx_bad = false;  // an index outside the short vector was met in this tile

                // Emit the finished dot product of segment `col` for vector b (SEGDOT):
                // the chunk's first segment, when it started in the previous chunk, goes
                // to the chunk's left carry record (Sec. IV-A), the rest to out.
                using AT2 = typename Pair<AT>::type;
                auto emit = [&](int col, int b, AT value) {
                    if (cleft && col == cfirst)
                        static_cast<AT2 *>(p.rec_left)[(size_t)b * p.nproc + proc] = make_pair2(value, AT(0));
                    else
                        static_cast<XT *>(p.vout[b])[col] = static_cast<XT>(value);
                };
                // general path: the last segment j in [i0, i1] starting at or before staged position pos
                auto col_search = [&](int pos) -> int {
                    int lo = i0, hi = i1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (p.pptr[mid] - kb0 <= pos)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    return lo;
                };
                if constexpr (SEGM) {
                    if (dup) {  // empty segments ending in this tile get zero
                        for (int j = i0 + 1 + lane; j < i1; j += 32)
                            if (p.pptr[j + 1] == p.pptr[j]) {
#pragma unroll
                                for (int b = 0; b < KB; ++b)
                                    if (b < kb) static_cast<XT *>(p.vout[b])[j] = zero_of<XT>();
                            }
                    }
                }
                // head counts before every mask word: the segmented modes read them from the tile's
                // prefix table, the scatter pass counts them step by step
                int cnt_ex = 0, htotal = 0;
                if constexpr (SEGM) {
                    htotal = pfx_s[p.mwp];
                } else if constexpr (MODE == MODE_DVALUES) {
                    int incl = __popc(mw);
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int v = __shfl_up_sync(FULL, incl, d);
                        if (lane >= d) incl += v;
                    }
                    cnt_ex = incl - __popc(mw);
                    htotal = __shfl_sync(FULL, incl, 31);
                }

                // ---- DVALUES: 4 consecutive positions per lane, 128 per step
                auto run_steps4 = [&](auto fast_tag) {
                    const bool FAST = fast_tag.value;  // compile-time (BoolC) or run-time (RtBool)
                    const int nsteps = (rel_hi + 127) >> 7;
#pragma unroll 2
                    for (int stp = 0; stp < nsteps; ++stp) {
                        const int p0 = (stp << 7) + (lane << 2);
                        const int sh = (lane & 7) << 2;
                        const uint32_t mwl = __shfl_sync(FULL, mw, p0 >> 5);
                        const int cwl = __shfl_sync(FULL, cnt_ex, p0 >> 5);
                        const uint32_t hb = (mwl >> sh) & 0xFu;
                        const int base = cwl + __popc(mwl & ((1u << sh) - 1u));  // heads before p0
                        const int lo_cut = min(max(rel_lo - p0, 0), 4);
                        const int hi_cut = min(max(rel_hi - p0, 0), 4);
                        uint32_t vm = ((1u << hi_cut) - 1u) & ~((1u << lo_cut) - 1u);
                        int ix[4] = {0, 0, 0, 0};
                        if (vm) {
                            const int4 qi = reinterpret_cast<const int4 *>(idx_s)[p0 >> 2];
                            ix[0] = qi.x;
                            ix[1] = qi.y;
                            ix[2] = qi.z;
                            ix[3] = qi.w;
                            uint32_t bad = 0;
#pragma unroll
                            for (int e = 0; e < 4; ++e) bad |= (static_cast<unsigned>(ix[e]) >= n_minor ? 1u : 0u) << e;
                            if (bad & vm) atomicOr(p.err, ERR_INDEX);  // out-of-range entries are skipped
                            vm &= ~bad;
                        }
                        int cc = i0 + base;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            cc += (hb >> e) & 1u;
                            if ((vm >> e) & 1u) {
                                const int ce = FAST ? cc : col_search(p0 + e);
                                const XT xv = win ? x_s[ce - xbase] : static_cast<const XT *>(p.vin[1])[ce];
                                AT mv;
                                if constexpr (SMEMV) {
                                    mv = static_cast<AT>(reinterpret_cast<const XT *>(smem)[ix[e]]);
                                } else {
                                    mv = static_cast<AT>(__ldg(static_cast<const XT *>(p.vin[0]) + ix[e]));
                                }
                                static_cast<VT *>(p.vout[0])[kb0 + p0 + e] =
                                    from_d<VT>(static_cast<double>(mv * static_cast<AT>(xv)));
                            }
                        }
                    }
                };

                // Common prologue of the 8-wide steps: lane l takes positions p0 .. p0+7,
                // p0 = 256 * stp + 8 * l, staged with the staggered loads (register e holds
                // position e ^ (4 * sw)).  hb: positional segment-start bits of the lane,
                // base: segment starts of the tile before p0, vm: positional valid bits
                // (all set on the whole steps of a tile: WHOLE).
                const int sw = (lane >> 2) & 1;
                auto step_head = [&](auto full_tag, int stp, int &p0, uint32_t &hb, int &base, uint32_t &vm) {
                    constexpr bool WHOLE = decltype(full_tag)::value;
                    p0 = (stp << 8) + (lane << 3);
                    const int sh = (lane & 3) << 3;
                    const int wi = p0 >> 5;  // the lane's mask word
                    const uint32_t mwl = wi < p.mwp ? mask_s[wi] : 0u;
                    const int cwl = pfx_s[wi];
                    hb = (mwl >> sh) & 0xFFu;
                    base = cwl + __popc(mwl & ((1u << sh) - 1u));
                    if constexpr (WHOLE) {
                        vm = 0xFFu;
                    } else {
                        const int lo_cut = min(max(rel_lo - p0, 0), 8);
                        const int hi_cut = min(max(rel_hi - p0, 0), 8);
                        vm = ((1u << hi_cut) - 1u) & ~((1u << lo_cut) - 1u);
                    }
                };
                // indices and values of the lane's 8 positions (register order); returns the
                // register-order valid bits with out-of-range indices removed (and reported)
                auto step_load = [&](auto full_tag, auto check_tag, int p0, uint32_t vm_r, int (&ix)[8], AT (&va)[8]) -> uint32_t {
                    constexpr bool WHOLE = decltype(full_tag)::value;
                    constexpr bool CHECK = decltype(check_tag)::value;
                    if (!WHOLE) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            ix[e] = 0;
                            va[e] = AT(0);
                        }
                    }
                    if (WHOLE || vm_r) {
                        stag8_idx(idx_s, p0, sw, ix);
                        Stag8<VT, AT>::run(val_s, p0, sw, va);
                        if (!WHOLE) {
                            // positions outside the tile hold whatever the slot held before:
                            // zero them (a stale NaN or infinity times zero would not vanish)
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (!((vm_r >> e) & 1u)) {
                                    ix[e] = 0;
                                    va[e] = AT(0);
                                }
                        }
                        // out-of-range indices are clamped into the vector (never dereferenced
                        // outside it) and reported once per tile; a plan whose indices were
                        // validated skips this on its whole steps (the indices are borrowed
                        // unchanged)
                        if constexpr (CHECK) {
                            unsigned mx = 0;
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                mx = max(mx, static_cast<unsigned>(ix[e]));
                                ix[e] = static_cast<int>(min(static_cast<unsigned>(ix[e]), n_minor - 1u));
                            }
                            idx_bad |= mx >= n_minor;
                        }
                    }
                    return vm_r;
                };

                // ---- SCATTER: 256 positions per step, lane l taking positions l, l+32, .., l+224.
                // Consecutive lanes hold consecutive positions, whose rows (sorted within a
                // column) fall in different shared-memory banks far more often than the rows
                // of positions 8 apart: fewer conflicted atomic wavefronts.
                auto run_scatter = [&](auto fast_tag, auto win_tag, auto full_tag, auto check_tag) {
                    constexpr bool CHECK = decltype(check_tag)::value;
                    const bool FAST = fast_tag.value;  // compile-time (BoolC) or run-time (RtBool)
                    constexpr bool WIN = decltype(win_tag)::value;
                    constexpr bool WHOLE = decltype(full_tag)::value;
                    auto xval = [&](int b, int ce) -> AT {
                        if constexpr (WIN) {
                            return static_cast<AT>(x_s[b * p.x_cap + ce - xbase]);
                        } else {
                            return static_cast<AT>(static_cast<const XT *>(p.vin[b])[ce]);
                        }
                    };
                    auto add = [&](int row, int b, AT contrib) {
                        if constexpr (SMEMV) {
                            atomicAdd(reinterpret_cast<AT *>(smem) + row * KB + b, contrib);
                        } else {
                            atomicAdd(static_cast<double *>(p.part) + (size_t)b * p.n_minor + row,
                                      static_cast<double>(contrib));
                        }
                    };
                    const VT *vv = reinterpret_cast<const VT *>(val_s);
                    const uint32_t lane_le = FULL >> (31 - lane);  // bits 0..lane
                    const int nsteps = (rel_hi + 255) >> 8;
                    int cbr = 0;  // segment starts of the tile before the step
                    for (int stp = 0; stp < nsteps; ++stp) {
                        const int s0 = stp << 8;
                        // segment-start words of the step (positions s0 + 32e .. s0 + 32e + 31)
                        uint32_t w[8];
                        {
                            const uint4 qa = reinterpret_cast<const uint4 *>(mask_s)[2 * stp];
                            const uint4 qb = reinterpret_cast<const uint4 *>(mask_s)[2 * stp + 1];
                            w[0] = qa.x; w[1] = qa.y; w[2] = qa.z; w[3] = qa.w;
                            w[4] = qb.x; w[5] = qb.y; w[6] = qb.z; w[7] = qb.w;
                            if (!WHOLE) {
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    if ((stp << 3) + e >= p.mwp) w[e] = 0u;
                            }
                        }
                        const int cb = cbr;
                        // all loads of the step first (independent), then the additions
                        int row[8];
                        AT a[8];
                        uint32_t ok = 0xFFu;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int pos = s0 + (e << 5) + lane;
                            if (WHOLE || (pos >= rel_lo && pos < rel_hi)) {
                                row[e] = idx_s[pos];
                                a[e] = to_acc<AT>(vv[pos]);
                            } else {
                                row[e] = 0;
                                a[e] = AT(0);
                                ok &= ~(1u << e);
                            }
                        }
                        if constexpr (CHECK) {
                            // out-of-range rows are clamped into the accumulator and reported
                            unsigned mx = 0;
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                mx = max(mx, static_cast<unsigned>(row[e]));
                                row[e] = static_cast<int>(min(static_cast<unsigned>(row[e]), n_minor - 1u));
                            }
                            idx_bad |= mx >= n_minor;
                        }
                        if (FAST && (w[0] | w[1] | w[2] | w[3] | w[4] | w[5] | w[6] | w[7]) == 0u) {
                            // no segment starts in this step: every position is in segment i0 + cb
#pragma unroll
                            for (int b = 0; b < KB; ++b) {
                                if (b < kb) {
                                    const AT xv = xval(b, i0 + cb);
#pragma unroll
                                    for (int e = 0; e < 8; ++e)
                                        if (WHOLE || ((ok >> e) & 1u)) add(row[e], b, a[e] * xv);
                                }
                            }
                            continue;
                        }
                        int ce[8];
                        {
                            int pre = i0 + cb;
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                ce[e] = FAST ? pre + __popc(w[e] & lane_le) : col_search(s0 + (e << 5) + lane);
                                pre += __popc(w[e]);
                            }
                            cbr = pre - i0;  // (a step without segment starts leaves it as it was)
                        }
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            if (b < kb) {
                                AT xv[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) xv[e] = (WHOLE || ((ok >> e) & 1u)) ? xval(b, ce[e]) : AT(0);
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    if (WHOLE || ((ok >> e) & 1u)) add(row[e], b, a[e] * xv[e]);
                            }
                        }
                    }
                };

                // ---- SEGDOT: 8 positions per lane, 256 per step.  Finished segments are
                // emitted from a per-lane scratch of the values that close at each position,
                // kept in this lane's own (already consumed) slots of the staged step.
                AT *ev_base = (sizeof(AT) == 8) ? reinterpret_cast<AT *>(const_cast<unsigned char *>(val_s))
                                                : reinterpret_cast<AT *>(const_cast<int32_t *>(idx_s));
                // front of a step: segment-start bits, loads, products and the lane-local
                // inclusive prefix rr (position order, restarted at every head)
                auto seg_front = [&](auto full_tag, auto check_tag, int stp, int &p0, uint32_t &hb, int &base,
                                     AT (&rr)[8][KB]) {
                    constexpr bool WHOLE = decltype(full_tag)::value;
                    uint32_t vm;
                    step_head(full_tag, stp, p0, hb, base, vm);
                    int ix[8];
                    AT va[8];
                    const uint32_t vm_r = step_load(full_tag, check_tag, p0, rot4(vm, sw), ix, va);
                    if constexpr (!SMEMV && KB > 1) {
                        // several vectors in global memory, interleaved (vin[0][i * KB + b]): the
                        // KB entries of a nonzero's index come in one or two vector loads.  The
                        // positions run outside and the vectors inside; every vector's products
                        // and prefix sums are the same operations as in the other paths.
                        const XT *vt = static_cast<const XT *>(p.vin[0]);
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int r = e ^ (sw << 2);  // register of position e
                            const int ixe = sw ? ix[e ^ 4] : ix[e];
                            const AT vae = sw ? va[e ^ 4] : va[e];
                            XT wv[KB];
                            if (WHOLE || ((vm_r >> r) & 1u)) {
                                Gather<XT, KB>::run(vt + (size_t)(vwin + ixe) * KB, wv);
                            } else {
#pragma unroll
                                for (int b = 0; b < KB; ++b) wv[b] = zero_of<XT>();
                            }
#pragma unroll
                            for (int b = 0; b < KB; ++b) {
                                const AT pe = mul_rn(vae, static_cast<AT>(wv[b]));
                                rr[e][b] = (e == 0 || ((hb >> e) & 1u)) ? pe : rr[e > 0 ? e - 1 : 0][b] + pe;
                            }
                        }
                        return;
                    }
#pragma unroll
                    for (int b = 0; b < KB; ++b) {
                        AT pr[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            AT w_ = AT(0);
                            if (WHOLE || ((vm_r >> e) & 1u)) {
                                if constexpr (SMEMV) {
                                    w_ = static_cast<AT>(reinterpret_cast<const XT *>(smem)[ix[e] * KB + b]);
                                } else {
                                    w_ = static_cast<AT>(__ldg(static_cast<const XT *>(p.vin[b]) + vwin + ix[e]));
                                }
                            }
                            pr[e] = mul_rn(va[e], w_);
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const AT pe = sw ? pr[e ^ 4] : pr[e];
                            rr[e][b] = (e == 0 || ((hb >> e) & 1u)) ? pe : rr[e > 0 ? e - 1 : 0][b] + pe;
                        }
                    }
                };
                // warp segmented scan of the lanes' open sums (the o operator of Sec. IV-B):
                // returns the open sum at the end of this lane; Tex: at the end of the previous lane
                auto seg_scan = [&](unsigned bal, AT t, AT &Tex) -> AT {
                    const unsigned le = bal & (FULL >> (31 - lane));
                    const int seg_start = le ? (31 - __clz(le)) : 0;
                    AT T = t;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const AT v = __shfl_up_sync(FULL, T, d);
                        if (lane - d >= seg_start && lane >= d) T += v;
                    }
                    Tex = __shfl_up_sync(FULL, T, 1);
                    if (lane == 0) Tex = AT(0);
                    return T;
                };
                // back of a step for vector b: emit the segments closed in this lane, then
                // carry the open sum at the end of the step (T31) into (chi, clo)
                auto seg_back = [&](auto fast_tag, int b, unsigned bal, int p0, uint32_t hb, int base,
                                    const AT (&rr)[8][KB], AT Tex, AT T31) {
                    const bool FAST = fast_tag.value;  // compile-time (BoolC) or run-time (RtBool)
                    if (hb != 0u && b < kb) {
                        AT *ev = ev_base + p0;
                        // value closing at position e: the open sum up to e - 1 (0 at e = 0)
                        if constexpr (sizeof(AT) == 4) {
                            const float4 lo = make_float4(0.f, rr[0][b], rr[1][b], rr[2][b]);
                            const float4 hi = make_float4(rr[3][b], rr[4][b], rr[5][b], rr[6][b]);
                            float4 *q = reinterpret_cast<float4 *>(ev);
                            q[sw] = sw ? hi : lo;  // staggered like the loads
                            q[sw ^ 1] = sw ? lo : hi;
                        } else {
#pragma unroll
                            for (int e = 1; e < 8; ++e) ev[e] = rr[e - 1][b];
                        }
                        // the first head closes the segment flowing into the lane
                        const bool before = (bal & ((1u << lane) - 1u)) != 0u;
                        const AT lead = Tex + (before ? AT(0) : chi[b] + clo[b]);
                        uint32_t rem = hb;
                        int k = 0;
                        while (rem) {
                            const int e = __ffs(rem) - 1;
                            AT v = (e == 0) ? AT(0) : ev[e];
                            if (k == 0) v += lead;
                            emit(FAST ? i0 + base + k : col_search(p0 + e - 1), b, v);
                            rem &= rem - 1u;
                            ++k;
                        }
                    }
                    if (bal) {
                        chi[b] = T31;
                        clo[b] = AT(0);
                    } else {  // compensated addition of the step total
                        carry_in(chi[b], clo[b], T31);
                    }
                };
                // the open segment runs through a whole head-free step: add its total t (the
                // butterfly over the lanes' sums) to the carry, compensated
                auto carry_add = [&](int b, AT t) { carry_in(chi[b], clo[b], t); };
                auto seg_carry_total = [&](int b, AT t) {
#pragma unroll
                    for (int d = 16; d >= 1; d >>= 1) t += __shfl_xor_sync(FULL, t, d);
                    carry_add(b, t);
                };
                auto run_segdot8 = [&](auto fast_tag, auto full_tag, auto check_tag) {
                    const int nsteps = (rel_hi + 255) >> 8;
                    int stp = 0;
                    if constexpr (KB == 1 && sizeof(AT) == 4 && WB <= WARPS_REGS) {
                        // two steps at a time: their loads, products, lane prefixes and scans do
                        // not depend on each other and interleave; the carry passes from the
                        // first step to the second as in the one-step loop (the same operations
                        // in the same order)
                        for (; stp + 1 < nsteps; stp += 2) {
                            int p0a, p0b, basea, baseb;
                            uint32_t hba, hbb;
                            AT ra[8][KB], rb[8][KB];
                            seg_front(full_tag, check_tag, stp, p0a, hba, basea, ra);
                            seg_front(full_tag, check_tag, stp + 1, p0b, hbb, baseb, rb);
                            const unsigned bala = __ballot_sync(FULL, hba != 0u);
                            const unsigned balb = __ballot_sync(FULL, hbb != 0u);
                            if ((bala | balb) == 0u) {
                                AT ta = ra[7][0], tb = rb[7][0];
#pragma unroll
                                for (int d = 16; d >= 1; d >>= 1) {
                                    ta += __shfl_xor_sync(FULL, ta, d);
                                    tb += __shfl_xor_sync(FULL, tb, d);
                                }
                                carry_add(0, ta);
                                carry_add(0, tb);
                            } else if (bala != 0u && balb != 0u) {
                                AT Texa, Texb;
                                const AT Ta = seg_scan(bala, ra[7][0], Texa);
                                const AT Tb = seg_scan(balb, rb[7][0], Texb);
                                const AT T31a = __shfl_sync(FULL, Ta, 31);
                                const AT T31b = __shfl_sync(FULL, Tb, 31);
                                seg_back(fast_tag, 0, bala, p0a, hba, basea, ra, Texa, T31a);
                                seg_back(fast_tag, 0, balb, p0b, hbb, baseb, rb, Texb, T31b);
                            } else if (bala != 0u) {
                                AT Texa;
                                const AT Ta = seg_scan(bala, ra[7][0], Texa);
                                seg_back(fast_tag, 0, bala, p0a, hba, basea, ra, Texa, __shfl_sync(FULL, Ta, 31));
                                seg_carry_total(0, rb[7][0]);
                            } else {
                                seg_carry_total(0, ra[7][0]);
                                AT Texb;
                                const AT Tb = seg_scan(balb, rb[7][0], Texb);
                                seg_back(fast_tag, 0, balb, p0b, hbb, baseb, rb, Texb, __shfl_sync(FULL, Tb, 31));
                            }
                        }
                    }
                    for (; stp < nsteps; ++stp) {
                        int p0, base;
                        uint32_t hb;
                        AT rr[8][KB];
                        seg_front(full_tag, check_tag, stp, p0, hb, base, rr);
                        const unsigned bal = __ballot_sync(FULL, hb != 0u);
                        if (bal == 0u) {
#pragma unroll
                            for (int b = 0; b < KB; ++b) seg_carry_total(b, rr[7][b]);
                            continue;
                        }
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            AT Tex;
                            const AT T = seg_scan(bal, rr[7][b], Tex);
                            seg_back(fast_tag, b, bal, p0, hb, base, rr, Tex, __shfl_sync(FULL, T, 31));
                        }
                    }
                };


                // ---- VSEG: several vectors, one per lane of a lane group.  Lane g VL + bv carries
                // vector bv through the virtual lanes v = g + NG i (i < VL) of every 256-position
                // step, virtual lane v being the 8 positions 8v .. 8v + 7 that lane v takes in the
                // single-vector pass.  Each sum is formed with that pass's operations in its order:
                // the prefix of a virtual lane restarted at every head, the butterfly total of a
                // head-free step, the segmented Kogge-Stone scan over the 32 virtual lanes of a step
                // with heads (levels within a lane on registers, the others by shuffles across the
                // lane groups) and the compensated carry.  The vectors are read through L2 from an
                // interleaved copy, vin[0][i * VL + b].
                auto run_vseg = [&](auto fast_tag, auto full_tag, auto check_tag) {
                    constexpr int VL = KB;
                    constexpr int NG = 32 / VL;
                    static_assert(MODE != MODE_VSEG || (VL >= 4 && VL <= VL_MAX && 32 % VL == 0), "lane groups of 4 or 8");
                    constexpr bool WHOLE = decltype(full_tag)::value;
                    constexpr bool CHECK = decltype(check_tag)::value;
                    const bool FAST = fast_tag.value;  // compile-time (BoolC) or run-time (RtBool)
                    const int g = lane / VL;
                    const int bv = lane - g * VL;
                    const bool act = bv < kb;
                    const float *vt = static_cast<const float *>(p.vin[0]) + bv;  // in global memory
                    const float *vsm = reinterpret_cast<const float *>(smem + VSCR_BYTES) + bv;  // staged (SMEMV)
                    // this lane's 8-value scratch (the region before the staging slots)
                    AT *vscr = reinterpret_cast<AT *>(smem) + (warp * 32 + lane) * 8;
                    const int nsteps = (rel_hi + 255) >> 8;
                    for (int stp = 0; stp < nsteps; ++stp) {
                        // the step's segment-start words (positions 256 stp + 32 j ..), and its
                        // virtual lanes that hold a head (bit v)
                        uint32_t w[8];
                        {
                            const uint4 qa = reinterpret_cast<const uint4 *>(mask_s)[2 * stp];
                            const uint4 qb = reinterpret_cast<const uint4 *>(mask_s)[2 * stp + 1];
                            w[0] = qa.x; w[1] = qa.y; w[2] = qa.z; w[3] = qa.w;
                            w[4] = qb.x; w[5] = qb.y; w[6] = qb.z; w[7] = qb.w;
                            if (!WHOLE) {
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    if ((stp << 3) + e >= p.mwp) w[e] = 0u;
                            }
                        }
                        unsigned bal;
                        {
                            const int wi = (stp << 3) + (lane >> 2);
                            const uint32_t wl = (WHOLE || wi < p.mwp) ? mask_s[wi] : 0u;
                            bal = __ballot_sync(FULL, ((wl >> ((lane & 3) << 3)) & 0xFFu) != 0u);
                        }
                        // word of the step holding virtual lane i's bits (NG = 8: one of two)
                        auto word_of = [&](int i) -> uint32_t {
                            constexpr int NW = NG > 4 ? 2 : 1;
                            const int wlo = (NG * i) >> 2;
                            uint32_t wv = w[wlo];
                            if constexpr (NW > 1) {
                                if (((g + NG * i) >> 2) != wlo) wv = w[wlo + 1];
                            }
                            return wv;
                        };
                        auto heads_of = [&](int i) -> uint32_t {
                            return (word_of(i) >> (((g + NG * i) & 3) << 3)) & 0xFFu;
                        };
                        // heads of the tile before virtual lane i (the single-vector pass's base): the
                        // tile's heads before the step, the step's words before virtual lane i's word
                        // and the bits of that word below the virtual lane's byte
                        const int cbs = pfx_s[stp << 3];
                        auto base_of = [&](int i, const int (&pre)[8]) -> int {
                            const int v = g + NG * i;
                            int pw = pre[(NG * i) >> 2];
                            if constexpr (NG > 4) {
                                if (((g + NG * i) >> 2) != ((NG * i) >> 2)) pw = pre[((NG * i) >> 2) + 1];
                            }
                            return cbs + pw + __popc(word_of(i) & ((1u << ((v & 3) << 3)) - 1u));
                        };
                        auto word_prefix = [&](int (&pre)[8]) {
                            int a = 0;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                pre[j] = a;
                                a += __popc(w[j]);
                            }
                        };
                        // products of virtual lane i's 8 positions in position order (+0 outside the tile)
                        auto products = [&](int i, AT (&pe)[8]) {
                            const int p0 = (stp << 8) + ((g + NG * i) << 3);
                            uint32_t vm = 0xFFu;
                            if constexpr (!WHOLE) {
                                const int lo_cut = min(max(rel_lo - p0, 0), 8);
                                const int hi_cut = min(max(rel_hi - p0, 0), 8);
                                vm = ((1u << hi_cut) - 1u) & ~((1u << lo_cut) - 1u);
                            }
                            int ix[8];
                            AT va[8];
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                ix[e] = 0;
                                va[e] = AT(0);
                            }
                            if (WHOLE || vm) {
                                const int4 qa = reinterpret_cast<const int4 *>(idx_s)[p0 >> 2];
                                const int4 qb = reinterpret_cast<const int4 *>(idx_s)[(p0 >> 2) + 1];
                                ix[0] = qa.x; ix[1] = qa.y; ix[2] = qa.z; ix[3] = qa.w;
                                ix[4] = qb.x; ix[5] = qb.y; ix[6] = qb.z; ix[7] = qb.w;
                                Load8<VT, AT>::run(val_s, p0, va);
                                if (!WHOLE) {
#pragma unroll
                                    for (int e = 0; e < 8; ++e)
                                        if (!((vm >> e) & 1u)) {
                                            ix[e] = 0;
                                            va[e] = AT(0);
                                        }
                                }
                                if constexpr (CHECK) {
                                    unsigned mx = 0;
#pragma unroll
                                    for (int e = 0; e < 8; ++e) {
                                        mx = max(mx, static_cast<unsigned>(ix[e]));
                                        ix[e] = static_cast<int>(min(static_cast<unsigned>(ix[e]), n_minor - 1u));
                                    }
                                    idx_bad |= mx >= n_minor;
                                }
                            }
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                AT wv = AT(0);
                                if (act && (WHOLE || ((vm >> e) & 1u))) {
                                    if constexpr (SMEMV) {
                                        wv = vsm[ix[e] * VL];
                                    } else {
                                        wv = __ldg(vt + (size_t)(vwin + ix[e]) * VL);
                                    }
                                }
                                pe[e] = mul_rn(va[e], wv);
                            }
                        };
                        if (bal == 0u) {
                            // head-free step: the butterfly total (xor 16, 8, .., 1 over the virtual
                            // lanes: the levels within a lane first, then across the lane groups)
                            AT t[VL];
#pragma unroll
                            for (int i = 0; i < VL; ++i) {
                                AT pe[8];
                                products(i, pe);
                                AT r = pe[0];
#pragma unroll
                                for (int e = 1; e < 8; ++e) r = r + pe[e];
                                t[i] = r;
                            }
#pragma unroll
                            for (int h = VL / 2; h >= 1; h >>= 1) {
#pragma unroll
                                for (int i = 0; i < h; ++i) t[i] = t[i] + t[i + h];
                            }
                            AT tot = t[0];
#pragma unroll
                            for (int d = NG / 2; d >= 1; d >>= 1) tot = tot + __shfl_xor_sync(FULL, tot, d * VL);
                            carry_in(chi[0], clo[0], tot);
                            continue;
                        }
                        // step with heads: every virtual lane's open sum at its end (T), the open sum
                        // before its first head (F); segments closing at its later heads are emitted
                        // here, from the lane's scratch of the values that close at each position
                        AT T[VL], F[VL];
                        int pre[8];
                        word_prefix(pre);
#pragma unroll
                        for (int i = 0; i < VL; ++i) {
                            const uint32_t hb = heads_of(i);
                            AT pe[8];
                            products(i, pe);
                            AT rr[8];
                            rr[0] = pe[0];
#pragma unroll
                            for (int e = 1; e < 8; ++e) rr[e] = ((hb >> e) & 1u) ? pe[e] : rr[e - 1] + pe[e];
                            T[i] = rr[7];
                            F[i] = AT(0);
                            if (hb) {
                                // value closing at position e: the open sum up to e - 1 (0 at e = 0)
                                float4 *q = reinterpret_cast<float4 *>(vscr);
                                q[0] = make_float4(0.f, rr[0], rr[1], rr[2]);
                                q[1] = make_float4(rr[3], rr[4], rr[5], rr[6]);
                                F[i] = vscr[__ffs(hb) - 1];
                                uint32_t rem = hb & (hb - 1u);
                                if (act && rem) {
                                    const int p0 = (stp << 8) + ((g + NG * i) << 3);
                                    XT *o = static_cast<XT *>(p.vout[bv]);
                                    int col = FAST ? i0 + base_of(i, pre) : 0;
                                    while (rem) {  // a later head: the segment lies inside the virtual lane
                                        const int e = __ffs(rem) - 1;
                                        col = FAST ? col + 1 : col_search(p0 + e - 1);
                                        o[col] = static_cast<XT>(vscr[e]);
                                        rem &= rem - 1u;
                                    }
                                }
                            }
                        }
                        // segmented Kogge-Stone scan of the open sums over the 32 virtual lanes: at
                        // level d virtual lane v adds the sum of v - d when no head lies in
                        // (v - d, v] and v >= d (bit v of ok)
                        unsigned ok = ~bal & ~1u;
#pragma unroll
                        for (int lv = 0; lv < 5; ++lv) {
                            const int d = 1 << lv;
                            if (lv > 0) ok &= ok << (d >> 1);
                            if (ok == 0u) break;  // (warp-uniform) no virtual lane adds at this level or later
                            const unsigned okg = ok >> g;  // bit NG i: virtual lane g + NG i adds
                            if (d < NG) {
                                // from lane group (g - d) mod NG: its sum of the same i, or of i - 1
                                // when the distance wraps past group NG - 1
                                const bool wsrc = g + d >= NG;
                                const int src = ((g + NG - d) % NG) * VL + bv;
                                AT rv[VL];
#pragma unroll
                                for (int i = 0; i < VL; ++i)
                                    rv[i] = __shfl_sync(FULL, wsrc ? (i > 0 ? T[i > 0 ? i - 1 : 0] : AT(0)) : T[i], src);
#pragma unroll
                                for (int i = 0; i < VL; ++i)
                                    if ((okg >> (NG * i)) & 1u) T[i] = T[i] + rv[i];
                            } else {
                                const int dd = d / NG;
#pragma unroll
                                for (int i = VL - 1; i >= dd; --i)
                                    if ((okg >> (NG * i)) & 1u) T[i] = T[i] + T[i - dd];
                            }
                        }
                        // open sum at the end of virtual lane v - 1 (0 for v = 0)
                        AT Tex[VL];
                        {
                            const bool wsrc = g == NG - 1;
                            const int src = ((g + NG - 1) % NG) * VL + bv;
#pragma unroll
                            for (int i = 0; i < VL; ++i) {
                                if constexpr (NG > 1) {
                                    Tex[i] = __shfl_sync(FULL, wsrc ? (i > 0 ? T[i > 0 ? i - 1 : 0] : AT(0)) : T[i], src);
                                } else {
                                    Tex[i] = i > 0 ? T[i > 0 ? i - 1 : 0] : AT(0);
                                }
                            }
                            if (g == 0) Tex[0] = AT(0);
                        }
                        // the first head of each virtual lane closes the segment flowing into it
                        const AT cc = chi[0] + clo[0];
#pragma unroll
                        for (int i = 0; i < VL; ++i) {
                            const uint32_t hb = heads_of(i);
                            if (act && hb) {
                                const int v = g + NG * i;
                                const bool before = (bal & ((1u << v) - 1u)) != 0u;
                                const AT lead = Tex[i] + (before ? AT(0) : cc);
                                const AT val = F[i] + lead;
                                const int e = __ffs(hb) - 1;
                                emit(FAST ? i0 + base_of(i, pre) : col_search((stp << 8) + (v << 3) + e - 1), bv, val);
                            }
                        }
                        chi[0] = __shfl_sync(FULL, T[VL - 1], (NG - 1) * VL + bv);
                        clo[0] = AT(0);
                    }
                };

                if constexpr (SEGM) {
                    if constexpr (MODE == MODE_SEGDOT) {
                        if (full && !dup && !p.checked)
                            run_segdot8(BoolC<true>{}, BoolC<true>{}, BoolC<false>{});
                        else
                            run_segdot8(RtBool{!dup}, BoolC<false>{}, BoolC<true>{});
                    } else {
                        if (full && !dup && !p.checked)
                            run_vseg(BoolC<true>{}, BoolC<true>{}, BoolC<false>{});
                        else
                            run_vseg(RtBool{!dup}, BoolC<false>{}, BoolC<true>{});
                    }
                    // a segment whose end event lies in this tile is complete; the open one
                    // continues in the chunk's next tile (kept in chi, clo) or, at the end of
                    // the chunk, in the next chunk: right carry record
                    const int col_last = dup ? col_search(rel_hi - 1) : i0 + htotal;
                    if constexpr (MODE == MODE_VSEG) {
                        if (lane < kb) {  // lane group 0 holds every vector's carry (lane = vector)
                            const AT v = chi[0] + clo[0];
                            if (col_last < i1)
                                emit(col_last, lane, v);
                            else if (needRight)
                                static_cast<AT2 *>(p.rec_right)[(size_t)lane * p.nproc + proc] = make_pair2(chi[0], clo[0]);
                        }
                    } else if (lane == 0) {
                        for (int b = 0; b < kb; ++b) {
                            const AT v = chi[b] + clo[b];
                            if (col_last < i1)
                                emit(col_last, b, v);
                            else if (needRight)
                                static_cast<AT2 *>(p.rec_right)[(size_t)b * p.nproc + proc] = make_pair2(chi[b], clo[b]);
                        }
                    }
                    if (col_last < i1 || chunk_last) {  // nothing runs on into this warp's next tile
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            chi[b] = AT(0);
                            clo[b] = AT(0);
                        }
                    }
                } else if constexpr (MODE == MODE_SCATTER) {
                    if (win && full && !dup && !p.checked)
                        run_scatter(BoolC<true>{}, BoolC<true>{}, BoolC<true>{}, BoolC<false>{});
                    else if (win)
                        run_scatter(RtBool{!dup}, BoolC<true>{}, BoolC<false>{}, BoolC<true>{});
                    else
                        run_scatter(RtBool{!dup}, BoolC<false>{}, BoolC<false>{}, BoolC<true>{});
                } else {
                    run_steps4(RtBool{!dup});
                }
                if (__any_sync(FULL, idx_bad) && lane == 0) atomicOr(p.err, ERR_INDEX);
            }
        }
        // the slot is free: the tile S ahead goes into it.  Its reads have all returned
        // (their values were used); the segmented mode also wrote its scratch into the
        // slot, which the proxy fence orders before the bulk copy's writes.
        __syncwarp();
        if constexpr (MODE == MODE_SEGDOT) fence_proxy_async_smem();
        const int kn = k + S;
        if (kn < nk) {
            if ((kn >> 5) == cb + 2) {
                dcur = dnxt;
                ecur = enxt;
                ++cb;
                load_batch(cb + 1, dnxt, enxt);
            }
            issue(kn, s);
        }
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }

    }  // blocks of this CTA

    if constexpr (MODE == MODE_SCATTER && SMEMV) {
        __syncthreads();
        const AT *acc = reinterpret_cast<const AT *>(smem);
        AT *part = static_cast<AT *>(p.part);
        for (int b = 0; b < kb; ++b)
            for (int i = threadIdx.x; i < p.n_minor; i += blockDim.x)
                part[((size_t)blockIdx.x * kb + b) * p.n_minor + i] = acc[i * KB + b];
    }
}

// Host-side launch of one instantiation; raises its shared-memory limit once per device.
// Up to WARPS_REGS warps run a kernel compiled for 128 registers a thread; more warps
// (single-vector passes only) run one compiled for 80.
template <typename VT, typename XT, int MODE, int KB, bool SMEMV, int WB>
cudaError_t launch_wb(const LaunchArgs &a) {
    auto kern = stream_kernel<VT, XT, MODE, KB, SMEMV, WB>;
    static SmemLimit lim;
    const cudaError_t e = ensure_smem_limit(kern, lim, a.smem);
    if (e != cudaSuccess) return e;
    kern<<<a.grid, a.block, a.smem, a.stream>>>(a.sp);
    return cudaGetLastError();
}

template <typename VT, typename XT, int MODE, int KB, bool SMEMV>
cudaError_t launch_one(const LaunchArgs &a) {
    if constexpr (KB == 1) {
        if (a.block > WARPS_REGS * 32) return launch_wb<VT, XT, MODE, KB, SMEMV, MAX_WARPS>(a);
    }
    return launch_wb<VT, XT, MODE, KB, SMEMV, WARPS_REGS>(a);
}

// The instantiation for a pass of `mode` over kb vectors (kb rounded up to the template's).
// FP64 runs several vectors of a segmented pass with MODE_SEGDOT (on chip or interleaved in
// global memory); the other value types with MODE_VSEG (lane groups of 4 or 8, the vectors
// staged in shared memory when they fit, else read through L2).
template <typename VT, typename XT>
cudaError_t launch_mode(int mode, int kb, const LaunchArgs &a) {
    constexpr bool F64 = sizeof(VT) == 8;
    if (mode == MODE_DVALUES) {
        return a.smemv ? launch_one<VT, XT, MODE_DVALUES, 1, true>(a) : launch_one<VT, XT, MODE_DVALUES, 1, false>(a);
    }
    if (mode == MODE_VSEG) {
        if constexpr (F64) {
            return cudaErrorInvalidValue;
        } else {
            if (kb < 1 || kb > 8) return cudaErrorInvalidValue;
            if (a.smemv)
                return kb <= 4 ? launch_wb<VT, XT, MODE_VSEG, 4, true, WARPS_VSEG>(a)
                               : launch_wb<VT, XT, MODE_VSEG, 8, true, WARPS_VSEG>(a);
            return kb <= 4 ? launch_wb<VT, XT, MODE_VSEG, 4, false, WARPS_VSEG>(a)
                           : launch_wb<VT, XT, MODE_VSEG, 8, false, WARPS_VSEG>(a);
        }
    }
    if (mode == MODE_SCATTER) {
        if (!a.smemv) return kb == 1 ? launch_one<VT, XT, MODE_SCATTER, 1, false>(a) : cudaErrorInvalidValue;
        if (kb <= 1) return launch_one<VT, XT, MODE_SCATTER, 1, true>(a);
        if (kb <= 2) return launch_one<VT, XT, MODE_SCATTER, 2, true>(a);
        if (kb <= 4) return launch_one<VT, XT, MODE_SCATTER, 4, true>(a);
        return launch_one<VT, XT, MODE_SCATTER, 8, true>(a);
    }
    if (kb <= 1) return a.smemv ? launch_one<VT, XT, MODE_SEGDOT, 1, true>(a) : launch_one<VT, XT, MODE_SEGDOT, 1, false>(a);
    if constexpr (!F64) {
        return cudaErrorInvalidValue;  // several vectors: MODE_VSEG
    } else {
        if (!a.smemv) {  // interleaved in global memory (vin[0])
            if (kb <= 2) return launch_one<VT, XT, MODE_SEGDOT, 2, false>(a);
            if (kb <= 4) return launch_one<VT, XT, MODE_SEGDOT, 4, false>(a);
            return launch_one<VT, XT, MODE_SEGDOT, 8, false>(a);
        }
        if (kb <= 2) return launch_one<VT, XT, MODE_SEGDOT, 2, true>(a);
        if (kb <= 4) return launch_one<VT, XT, MODE_SEGDOT, 4, true>(a);
        return launch_one<VT, XT, MODE_SEGDOT, 8, true>(a);
    }
}

}  // namespace gbk
