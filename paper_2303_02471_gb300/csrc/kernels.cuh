// Device building blocks and kernel launchers of the column-wise SpGEMM.
//
// Every kernel walks the products of a column j of C the same way
// (Gustavson by columns, Section 2.1): for each stored B_kj, every stored
// A_ik gives the product A_ik * B_kj for row i.  The walk flattens the
// products of a chunk of B entries so that consecutive lanes take
// consecutive entries of an A column (coalesced), with the owning B entry
// found by a binary search over the chunk's prefix sums of Z^A_k.
#pragma once

#include <algorithm>

#include "spgemm_internal.cuh"

namespace spg {

struct BinOffsets { int64_t v[NBINS + 1]; };

// Products a lane of a group walk gathers before it consumes them.
constexpr int kGroupBatch = 2;

// Threads per CTA of the symbolic CTA-level kernels (several CTAs per SM).
constexpr int kSymCtaThreads = 256;

// Hash-table slots per output entry of a column in the numeric and backward
// phases, per cent (spg_config.table_slots_pct's default).
constexpr int kDefaultSlotsPct = 150;

// ------------------------------------------------------ L2 residency
// Gathers of A's rows and values carry an L2 evict-last policy: every column
// of B reads A's columns again, while C (and the kept flags) stream through
// L2 once and would otherwise push A out.
__device__ __forceinline__ uint64_t keep_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int32_t ld_keep(const int32_t *a, uint64_t p) {
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(p));
    return v;
}
__device__ __forceinline__ float ld_keep(const float *a, uint64_t p) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(p));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *a, uint64_t p) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(p));
    return v;
}

// ------------------------------------------------------------ group walk
// A group of G lanes (G divides 32) walks the products of B entries
// [p0, p1) in chunks of G entries.  f(row, product) runs once per product
// on the lane that owns it.  All lanes of the group must call this with the
// same arguments.
template <int G, bool VALS, typename VT, typename F>
__device__ __forceinline__ void group_products(unsigned mask, const int64_t *__restrict__ Acp,
                                               const int32_t *__restrict__ Arow,
                                               const VT *__restrict__ Aval,
                                               const int32_t *__restrict__ Brow,
                                               const VT *__restrict__ Bval, int64_t p0, int64_t p1,
                                               F &&f) {
    const int gl = threadIdx.x & (G - 1);
    const uint64_t pol = keep_policy();
    for (int64_t base = p0; base < p1; base += G) {
        const int64_t p = base + gl;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = Brow[p];
            a0 = Acp[k];
            z = static_cast<int>(Acp[k + 1] - a0);
            if (VALS) bv = Bval[p];
        }
        const int incl = group_incl_scan<G>(mask, z);
        const int total = __shfl_sync(mask, incl, G - 1, G);
        const int excl = incl - z;
        for (int q0 = 0; q0 < total; q0 += G * kGroupBatch) {
            int32_t rows[kGroupBatch];
            VT av[kGroupBatch], bvs[kGroupBatch];
#pragma unroll
            for (int u = 0; u < kGroupBatch; ++u) {
                const int q = q0 + u * G + gl;
                rows[u] = -1;
                if (q0 + u * G < total) {  // uniform over the group
                    int s = 0;
#pragma unroll
                    for (int step = G / 2; step > 0; step >>= 1) {
                        const int ex = __shfl_sync(mask, excl, s + step, G);
                        if (ex <= q) s += step;
                    }
                    const int64_t a0s = __shfl_sync(mask, a0, s, G);
                    const int exs = __shfl_sync(mask, excl, s, G);
                    if (VALS) bvs[u] = __shfl_sync(mask, bv, s, G);
                    if (q < total) {
                        const int64_t qa = a0s + (q - exs);
                        rows[u] = ld_keep(Arow + qa, pol);
                        if (VALS) av[u] = ld_keep(Aval + qa, pol);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kGroupBatch; ++u) {
                if (rows[u] >= 0) {
                    VT prod = VT(0);
                    if (VALS) prod = av[u] * bvs[u];
                    f(rows[u], prod);
                }
            }
        }
    }
}

// Products a thread of a walk gathers before it consumes them.
constexpr int kWalkBatch = 4;

// ------------------------------------------------------------- CTA walk
// Entries whose A column has at least this many entries are walked one
// 32-product window at a time with a single owner per window (and, in the
// value walk, a ring of windows); shorter ones share windows.  On R-MAT 16
// measured as fast as 24 or 32 or up to 2 % faster (a half-full window in
// the ring against the shared windows' search for their entries), 64 slower.
constexpr int kLongEntry = 16;
// Windows of a long entry in the register ring of the dense bin's value
// walk (cta_walk's AHEAD; other callers keep one): four 256-thread CTAs per
// SM leave 64 registers a thread, which hold five without spilling.
constexpr int kWalkAhead = 5;
// The same for the dense bin's flag walks (rows only, one register a window;
// eight 256-thread CTAs per SM leave the symbolic kernel 32 registers a
// thread): the symbolic phase's, and the numeric kernel's when no flags were
// kept (the single pass).
constexpr int kSymWalkAhead = 4;

// Inclusive block scan of four int32 counters packed as two int64 lanes
// (each half < 2^31); totals returned.  Two barriers.
__device__ __forceinline__ void cta_incl_scan4(int (&v)[4], int64_t *s_warp, int (&tot)[4]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = (int64_t)v[0] | ((int64_t)v[1] << 32);
    int64_t y = (int64_t)v[2] | ((int64_t)v[3] << 32);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t ox = __shfl_up_sync(0xffffffffu, x, d);
        const int64_t oy = __shfl_up_sync(0xffffffffu, y, d);
        if (lane >= d) {
            x += ox;
            y += oy;
        }
    }
    if (lane == 31) {
        s_warp[warp] = x;
        s_warp[32 + warp] = y;
    }
    __syncthreads();
    if (warp == 0) {
        int64_t a = lane < nw ? s_warp[lane] : 0, b = lane < nw ? s_warp[32 + lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t oa = __shfl_up_sync(0xffffffffu, a, d);
            const int64_t ob = __shfl_up_sync(0xffffffffu, b, d);
            if (lane >= d) {
                a += oa;
                b += ob;
            }
        }
        if (lane < nw) {
            s_warp[lane] = a;
            s_warp[32 + lane] = b;
        }
    }
    __syncthreads();
    const int64_t tx = s_warp[nw - 1], ty = s_warp[32 + nw - 1];
    if (warp > 0) {
        x += s_warp[warp - 1];
        y += s_warp[32 + warp - 1];
    }
    v[0] = (int)(x & 0xffffffff); v[1] = (int)(x >> 32);
    v[2] = (int)(y & 0xffffffff); v[3] = (int)(y >> 32);
    tot[0] = (int)(tx & 0xffffffff); tot[1] = (int)(tx >> 32);
    tot[2] = (int)(ty & 0xffffffff); tot[3] = (int)(ty >> 32);
}

// Shared scratch of the CTA walk: the non-empty B entries of a chunk, long
// entries first, then short ones.
template <typename VT>
struct WalkSmem {
    int *key;       // [blockDim] long: windows before it; short: products before it
    int *z;         // [blockDim] Z^A_k
    int64_t *a0;    // [blockDim] start of A column k
    VT *bv;         // [blockDim] B_kj
    int64_t *warp;  // [64]
};

template <typename VT>
__host__ __device__ inline size_t walk_smem_bytes(int threads) {
    return (size_t)threads * (16 + sizeof(VT)) + 64 * 8 + 32;
}

template <typename VT>
__device__ __forceinline__ WalkSmem<VT> carve_walk(unsigned char *p) {
    WalkSmem<VT> w;
    w.a0 = reinterpret_cast<int64_t *>(p); p += (size_t)blockDim.x * 8;
    w.warp = reinterpret_cast<int64_t *>(p); p += 64 * 8;
    w.key = reinterpret_cast<int *>(p); p += (size_t)blockDim.x * 4;
    w.z = reinterpret_cast<int *>(p); p += (size_t)blockDim.x * 4;
    p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    w.bv = reinterpret_cast<VT *>(p); p += (size_t)blockDim.x * sizeof(VT);
    p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    return w;
}

// The whole CTA walks the products of B entries [p0, p1) of one column
// (whose Op_j must be below 2^31).  Per chunk of blockDim entries, one block
// scan sorts the non-empty entries into long ones (Z^A_k >= kLongEntry) and
// short ones.  The work is cut into windows of 32 products, one per lane,
// with consecutive lanes on consecutive entries of an A column (coalesced):
//   * a long entry contributes ceil(Z^A_k / 32) windows of its own; the
//     window's owner is the same for all lanes and advances with a uniform
//     shared-memory scan;
//   * short entries are concatenated into windows that can span several
//     entries; with s the entry of the window's first product, entries
//     s+1..s+32 are loaded one per lane, the offsets of those that start in
//     the window are OR-reduced into a mask and lane l's owner is
//     s + popc(mask & bits 1..l).
// Every warp takes an equal contiguous share of the chunk's windows (balanced
// over products, not B entries); kWalkBatch windows are gathered before any
// product is consumed.  f(row, product) per product.  Contains barriers:
// every thread of the CTA must call it.
template <bool VALS, typename VT, int AHEAD = 1, typename F>
__device__ __forceinline__ void cta_walk(const int64_t *__restrict__ Acp, const int32_t *__restrict__ Arow,
                                         const VT *__restrict__ Aval, const int32_t *__restrict__ Brow,
                                         const VT *__restrict__ Bval, int64_t p0, int64_t p1,
                                         const WalkSmem<VT> &w, F &&f) {
    // windows gathered per lane before any is consumed: with values, short
    // entries take one at a time (the loop stays small enough not to spill);
    // long ones keep a ring of AHEAD windows in flight when the caller asks
    // for one (AHEAD > 1) or values are walked, else take kWalkBatch windows
    // at a time across entries
    constexpr int UB = VALS ? 1 : kWalkBatch;
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const uint64_t pol = keep_policy();
    for (int64_t base = p0; base < p1; base += T) {
        const int64_t p = base + threadIdx.x;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = Brow[p];
            a0 = Acp[k];
            z = (int)(Acp[k + 1] - a0);
            if (VALS) bv = Bval[p];
        }
        const bool lng = z >= kLongEntry;
        // counters: long windows, long entries, short products, short entries
        int v[4] = {lng ? (z + 31) >> 5 : 0, lng ? 1 : 0, lng ? 0 : z, (!lng && z > 0) ? 1 : 0};
        const int mine[4] = {v[0], v[1], v[2], v[3]};
        int tot[4];
        cta_incl_scan4(v, w.warp, tot);
        const int nl = tot[1];
        if (lng) {
            const int i = v[1] - 1;
            w.key[i] = v[0] - mine[0];
            w.z[i] = z;
            w.a0[i] = a0;
            if (VALS) w.bv[i] = bv;
        } else if (z > 0) {
            const int i = nl + v[3] - 1;
            w.key[i] = v[2] - mine[2];
            w.z[i] = z;
            w.a0[i] = a0;
            if (VALS) w.bv[i] = bv;
        }
        __syncthreads();
        const int WL = tot[0], nsh = tot[3], ZS = tot[2];
        const int WS = (ZS + 31) >> 5;
        const int64_t nwin = (int64_t)WL + WS;
        const int win0 = (int)(nwin * warp / nw), win1 = (int)(nwin * (warp + 1) / nw);
        // ---- long entries: windows [win0, min(win1, WL))
        {
            const int e1 = win1 < WL ? win1 : WL;
            if (win0 < e1) {
                int li = 0, hi = nl - 1;
                while (li < hi) {
                    const int mid = (li + hi + 1) >> 1;
                    if (w.key[mid] <= win0) li = mid; else hi = mid - 1;
                }
                if constexpr (UB == 1 || AHEAD > 1) {
                    // entry by entry: the entry's windows in [win, e_end)
                    // are one warp-uniform loop over idx = window * 32 + lane
                    // of its A column
                    for (int win = win0; win < e1; ++li) {
                        const int e_key = w.key[li], e_z = w.z[li];
                        const int nk = li + 1 < nl ? w.key[li + 1] : 0x7fffffff;
                        const int e_end = nk < e1 ? nk : e1;
                        const int64_t a0 = w.a0[li];
                        const int32_t *rp = Arow + a0;
                        const VT *vp = VALS ? Aval + a0 : nullptr;
                        const VT b = VALS ? w.bv[li] : VT(0);
                        const int i1 = (e_end - e_key) << 5;
                        // a ring of AHEAD windows in registers: slot d is
                        // consumed and refilled with the window AHEAD
                        // further on, so the gathers of the other slots stay
                        // in flight (the loop is unrolled by AHEAD, so the
                        // slots never move between registers)
                        int idx = ((win - e_key) << 5) + lane;
                        int32_t rq[AHEAD];
                        VT vq[AHEAD];
#pragma unroll
                        for (int d = 0; d < AHEAD; ++d) {
                            const int q = idx + 32 * d;
                            const bool in = q < i1 && q < e_z;
                            rq[d] = in ? ld_keep(rp + q, pol) : -1;
                            vq[d] = VALS && in ? ld_keep(vp + q, pol) : VT(0);
                        }
                        for (; idx < i1; idx += 32 * AHEAD) {
#pragma unroll
                            for (int d = 0; d < AHEAD; ++d) {
                                if (rq[d] >= 0) f(rq[d], VALS ? vq[d] * b : VT(0));
                                const int q = idx + 32 * (AHEAD + d);
                                const bool in = q < i1 && q < e_z;
                                rq[d] = in ? ld_keep(rp + q, pol) : -1;
                                vq[d] = VALS && in ? ld_keep(vp + q, pol) : VT(0);
                            }
                        }
                        win = e_end;
                    }
                } else {
                    // the owner is the same for every lane of a window: keep its
                    // entry in registers and reload only when it advances
                    int e_key = w.key[li], e_z = w.z[li];
                    int64_t e_a0 = w.a0[li];
                    VT e_b = VALS ? w.bv[li] : VT(0);
                    int next_key = li + 1 < nl ? w.key[li + 1] : 0x7fffffff;
                    for (int win = win0; win < e1; win += UB) {
                        int32_t rows[UB];
                        VT av[UB], bvs[UB];
    #pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            rows[u] = -1;
                            if (win + u < e1) {
                                while (next_key <= win + u) {
                                    ++li;
                                    e_key = next_key;
                                    e_z = w.z[li];
                                    e_a0 = w.a0[li];
                                    if (VALS) e_b = w.bv[li];
                                    next_key = li + 1 < nl ? w.key[li + 1] : 0x7fffffff;
                                }
                                const int idx = ((win + u - e_key) << 5) + lane;
                                if (idx < e_z) {
                                    const int64_t qa = e_a0 + idx;
                                    rows[u] = ld_keep(Arow + qa, pol);
                                    if (VALS) {
                                        av[u] = ld_keep(Aval + qa, pol);
                                        bvs[u] = e_b;
                                    }
                                }
                            }
                        }
    #pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            if (rows[u] >= 0) {
                                VT prod = VT(0);
                                if (VALS) prod = av[u] * bvs[u];
                                f(rows[u], prod);
                            }
                        }
                    }
                }
            }
        }
        // ---- short entries: windows [max(win0, WL), win1) of the concatenation
        {
            const int s0w = (win0 > WL ? win0 : WL) - WL, s1w = win1 - WL;
            if (s0w < s1w) {
                const int *sk = w.key + nl;
                const int64_t *sa = w.a0 + nl;
                const VT *sb = w.bv + nl;
                const int qs = s0w << 5;
                int s = 0, hi = nsh - 1;
                while (s < hi) {
                    const int mid = (s + hi + 1) >> 1;
                    if (sk[mid] <= qs) s = mid; else hi = mid - 1;
                }
                for (int win = s0w; win < s1w; win += UB) {
                    int32_t rows[UB];
                    VT av[UB], bvs[UB];
#pragma unroll
                    for (int u = 0; u < UB; ++u) {
                        rows[u] = -1;
                        if (win + u < s1w) {  // uniform over the warp
                            const int qf = (win + u) << 5;
                            const int cand = s + 1 + lane;
                            const int pos = cand < nsh ? sk[cand] - qf : 64;
                            const unsigned bits = __reduce_or_sync(0xffffffffu, pos < 32 ? (1u << pos) : 0u);
                            const int own = s + __popc(bits & upto);
                            const int q = qf + lane;
                            if (q < ZS) {
                                const int64_t qa = sa[own] + (q - sk[own]);
                                rows[u] = ld_keep(Arow + qa, pol);
                                if (VALS) {
                                    av[u] = ld_keep(Aval + qa, pol);
                                    bvs[u] = sb[own];
                                }
                            }
                            s += __popc(bits) + (__ballot_sync(0xffffffffu, pos == 32) ? 1 : 0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UB; ++u) {
                        if (rows[u] >= 0) {
                            VT prod = VT(0);
                            if (VALS) prod = av[u] * bvs[u];
                            f(rows[u], prod);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ bit selection
// Position of the k-th (0-based) set bit of b, for k < popc(b): a binary
// search over the halves of the word by their population counts.
__device__ __forceinline__ int select_bit(uint32_t b, int k) {
    int pos = 0;
#pragma unroll
    for (int width = 16; width > 0; width >>= 1) {
        const int c = __popc(b & ((1u << width) - 1u));
        if (k >= c) {
            k -= c;
            b >>= width;
            pos += width;
        }
    }
    return pos;
}

// ------------------------------------------------- two-level row bitmap
// For extracting a hash table's rows in ascending order in O(m / 1024 + n)
// per column: L0 has one bit per row, L1 one bit per non-zero L0 word.
// After marking, cta_list_words writes the indices of the non-zero L0 words
// in ascending order to `wlist` and returns their number; cta_expand_words
// then visits the rows in ascending order with their ranks and clears both
// levels.  Every thread must call both (they contain barriers).
__device__ __forceinline__ void mark_row(uint32_t *L0, uint32_t *L1, int32_t row) {
    const uint32_t bit = 1u << (row & 31);
    const uint32_t old = atomicOr(&L0[row >> 5], bit);
    if (old == 0u) atomicOr(&L1[row >> 10], 1u << ((row >> 5) & 31));
}

__device__ __forceinline__ int64_t cta_list_words(uint32_t *L1, int64_t W1, int32_t *wlist, int64_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // each warp owns a contiguous range of L1 words
    const int64_t per = ((W1 + nw - 1) / nw + 31) & ~int64_t(31);
    const int64_t w0 = (int64_t)warp * per < W1 ? (int64_t)warp * per : W1;
    const int64_t w1 = w0 + per < W1 ? w0 + per : W1;
    int64_t cnt = 0;
    for (int64_t w = w0 + lane; w < w1; w += 32) cnt += __popc(L1[w]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    int64_t off = 0, total = 0;
    for (int i = 0; i < nw; ++i) {
        const int64_t c = s_warp[i];
        if (i < warp) off += c;
        total += c;
    }
    for (int64_t base = w0; base < w1; base += 32) {
        const int64_t w = base + lane;
        uint32_t bits = w < w1 ? L1[w] : 0u;
        const int c = __popc(bits);
        int incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        int64_t pos = off + incl - c;
        if (w < w1) {
            L1[w] = 0u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                wlist[pos++] = (int32_t)(w * 32 + b);
            }
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncthreads();
    return total;
}

// Visits the rows of the K listed L0 words in ascending order: f(row, rank).
// Warps own contiguous ranges of the list; lanes expand consecutive words so
// consecutive lanes get consecutive ranks (coalesced writes).  Clears L0.
template <typename F>
__device__ __forceinline__ void cta_expand_words(uint32_t *L0, const int32_t *wlist, int64_t K, int64_t *s_warp,
                                                 F &&f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = ((K + nw - 1) / nw + 31) & ~int64_t(31);
    const int64_t k0 = (int64_t)warp * per < K ? (int64_t)warp * per : K;
    const int64_t k1 = k0 + per < K ? k0 + per : K;
    int64_t cnt = 0;
    for (int64_t i = k0 + lane; i < k1; i += 32) cnt += __popc(L0[wlist[i]]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if (lane == 0) s_warp[warp] = cnt;
    __syncthreads();
    int64_t off = 0;
    for (int i = 0; i < warp; ++i) off += s_warp[i];
    for (int64_t base = k0; base < k1; base += 32) {
        const int64_t i = base + lane;
        int32_t word = 0;
        uint32_t v = 0u;
        if (i < k1) {
            word = wlist[i];
            v = L0[word];
            L0[word] = 0u;
        }
        const int cntl = __popc(v);
        int incl = cntl;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const int S = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - cntl;
        for (int o0 = 0; o0 < S; o0 += 32) {
            const int o = o0 + lane;
            int s = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, excl, s + step);
                if (ex <= o) s += step;
            }
            uint32_t b = __shfl_sync(0xffffffffu, v, s);
            const int kk = o - __shfl_sync(0xffffffffu, excl, s);
            const int32_t ws = __shfl_sync(0xffffffffu, word, s);
            if (o < S) f(ws * 32 + select_bit(b, kk), off + o);
        }
        off += S;
    }
    __syncthreads();
}

// ------------------------------------------------------ bitmap ranking
// Dense flags of the SPA (Algorithm 1's SPA_flags) kept as a bitmap over the
// m rows, one uint2 per 32 rows: .x the bits, .y the number of set bits in
// all earlier words.  After cta_bitmap_prefix, the position of row i in the
// sorted column is rank(i) = .y + popc(.x & lanes below i).
__device__ __forceinline__ int32_t bitmap_rank(const uint2 *bm, int32_t row) {
    const uint2 w = bm[row >> 5];
    return (int32_t)w.y + __popc(w.x & ((1u << (row & 31)) - 1u));
}

// Exclusive prefix of popcounts over W words into .y; returns the total.
// The bits come from src[0..W) when src is given (a copy kept in global
// memory, written to .x on the way), else from .x.  A warp takes 256
// consecutive words as four rounds of 64, lane l holding words 2l and 2l+1
// of each round: loads and 16-byte stores are contiguous across the warp,
// and the four rounds' counts share one packed 64-bit warp scan (16 bits per
// round; a round counts at most 2048 bits).  Warps cover consecutive runs;
// one block-wide offset per pass.  Every thread must call it.
__device__ __forceinline__ int64_t cta_bitmap_prefix(uint2 *bm, int64_t W64, const uint32_t *src, int64_t *s_warp) {
    const int W = (int)W64;  // m < 2^31: words and counts are 32-bit
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // pair loads and 16-byte stores need aligned starts (uniform over the CTA)
    const bool vec = (reinterpret_cast<uintptr_t>(bm) & 15) == 0 &&
                     (src == nullptr || (reinterpret_cast<uintptr_t>(src) & 7) == 0);
    int carry = 0;
    for (int r0 = 0; r0 < W; r0 += 256 * nw) {
        const int wb = r0 + warp * 256 + 2 * lane;
        uint32_t b[8];
        uint64_t packed = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int w = wb + 64 * k;
            if (vec && w + 1 < W) {
                if (src) {
                    const uint2 u = *reinterpret_cast<const uint2 *>(src + w);
                    b[2 * k] = u.x;
                    b[2 * k + 1] = u.y;
                } else {
                    const uint4 u = *reinterpret_cast<const uint4 *>(bm + w);
                    b[2 * k] = u.x;
                    b[2 * k + 1] = u.z;
                }
            } else {
                b[2 * k] = w < W ? (src ? src[w] : bm[w].x) : 0u;
                b[2 * k + 1] = w + 1 < W ? (src ? src[w + 1] : bm[w + 1].x) : 0u;
            }
            packed |= (uint64_t)(__popc(b[2 * k]) + __popc(b[2 * k + 1])) << (16 * k);
        }
        const uint64_t mine = packed;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(0xffffffffu, packed, d);
            if (lane >= d) packed += o;
        }
        const uint64_t tot = __shfl_sync(0xffffffffu, packed, 31);
        const int wsum = (int)((tot & 0xffff) + ((tot >> 16) & 0xffff) + ((tot >> 32) & 0xffff) + (tot >> 48));
        if (lane == 31) s_warp[warp] = wsum;
        __syncthreads();
        int tw = lane < nw ? (int)s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, tw, d);
            if (lane >= d) tw += o;
        }
        const int before = __shfl_sync(0xffffffffu, tw, warp > 0 ? warp - 1 : 0);
        const int pass = __shfl_sync(0xffffffffu, tw, nw - 1);
        int base = carry + (warp > 0 ? before : 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int w = wb + 64 * k;
            const uint32_t y0 = (uint32_t)(base + (int)((packed >> (16 * k)) & 0xffff) - (int)((mine >> (16 * k)) & 0xffff));
            const uint32_t y1 = y0 + (uint32_t)__popc(b[2 * k]);
            if (vec && w + 1 < W) {
                *reinterpret_cast<uint4 *>(bm + w) = make_uint4(b[2 * k], y0, b[2 * k + 1], y1);
            } else {
                if (w < W) bm[w] = make_uint2(b[2 * k], y0);
                if (w + 1 < W) bm[w + 1] = make_uint2(b[2 * k + 1], y1);
            }
            base += (int)((tot >> (16 * k)) & 0xffff);
        }
        carry += pass;
        __syncthreads();
    }
    return carry;
}

// Writes out the set bits of bm[0..W) in ascending row order: the row at
// sorted position `rank` of the column is stored by put(rank, map(row))
// (bm[..].y must hold the prefix counts).  Warps take groups of kVisitGroup
// chunks of 32 words, the first group by warp index and the next ones from
// the shared counter *s_next, which must hold kVisitGroup * (number of warps)
// before a barrier that precedes the call (one shared atomic per 4096 rows).
// The ranks of a group are consecutive: each lane holds one word of a chunk
// and writes the word's rows, rank minus the group's first rank being the
// slot, into the warp's kVisitStage-entry slice of `stage`; the warp then
// stores the staged slots in order, one per lane, with kVisitUnroll map()
// look-ups in flight per lane before their stores, so the stores are
// coalesced and a group waits for few look-up latencies.  A group of more
// than kVisitStage rows goes through the slice in pieces.  stage:
// kVisitStage ints per warp of shared memory that nothing else uses during
// the call.  Clears the bits when `clear`.  No barrier inside.
// Chunks of 32 words a warp takes per grab in cta_bitmap_visit.
constexpr int kVisitGroup = 4;
// Rows a warp stages per piece in cta_bitmap_visit.
constexpr int kVisitStage = 160;
// Look-ups per lane issued before their stores in cta_bitmap_visit.
constexpr int kVisitUnroll = 4;

template <typename M, typename P>
__device__ __forceinline__ void cta_bitmap_visit(uint2 *bm, int64_t W64, bool clear, unsigned *s_next,
                                                 int32_t *stage, M &&map, P &&put) {
    // m < 2^31, so words, chunks and ranks all fit 32-bit indices
    const int W = (int)W64;
    const int lane = threadIdx.x & 31;
    const int nchunks = (W + 31) >> 5;
    int32_t *slots = stage + (threadIdx.x >> 5) * kVisitStage;
    // stores the slots of relative ranks [from, to), slot 0 holding `from`
    auto flush = [&](int32_t r0, int from, int to) {
        for (int o0 = from; o0 < to; o0 += 32 * kVisitUnroll) {
            int32_t out[kVisitUnroll];
#pragma unroll
            for (int u = 0; u < kVisitUnroll; ++u) {
                const int o = o0 + 32 * u + lane;
                out[u] = o < to ? map(slots[o - from]) : 0;
            }
#pragma unroll
            for (int u = 0; u < kVisitUnroll; ++u) {
                const int o = o0 + 32 * u + lane;
                if (o < to) put(r0 + o, out[u]);
            }
        }
    };
    for (int g = (threadIdx.x >> 5) * kVisitGroup; g < nchunks;) {
        const int gend = g + kVisitGroup < nchunks ? g + kVisitGroup : nchunks;
        // the group's first word exists (g < nchunks); its prefix count is
        // the group's first rank
        const int32_t r0 = (int32_t)bm[g << 5].y;
        int flushed = 0;  // relative ranks below this are stored
        int top = 0;      // relative end of the rows staged so far
        for (int c = g; c < gend; ++c) {
            const int wd = (c << 5) + lane;
            const uint2 v = wd < W ? bm[wd] : make_uint2(0u, 0u);
            if (clear && v.x) bm[wd].x = 0u;
            uint32_t bits = v.x;
            // lanes past W hold no bits
            int pos = wd < W ? (int)v.y - r0 : 0;
            const int32_t row0 = wd << 5;
            const int end = (int)__reduce_max_sync(0xffffffffu, (unsigned)(pos + __popc(bits)));
            for (;;) {
                const int lim = flushed + kVisitStage;
                while (bits && pos < lim) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    slots[pos - flushed] = row0 + b;
                    ++pos;
                }
                if (end <= lim) break;  // uniform over the warp
                __syncwarp();
                flush(r0, flushed, lim);
                __syncwarp();
                flushed = lim;
            }
            top = end > top ? end : top;
        }
        __syncwarp();
        flush(r0, flushed, top);
        __syncwarp();
        unsigned nc = 0;
        if (lane == 0) nc = atomicAdd(s_next, (unsigned)kVisitGroup);
        g = (int)__shfl_sync(0xffffffffu, nc, 0);
    }
}

// ------------------------------------------------------- bulk copies
// One-shot global -> shared bulk copies (TMA, cp.async.bulk) completing on
// an mbarrier in shared memory.  Addresses and sizes are multiples of 16
// bytes; the caller checks.  The wait gives up after kBulkWaitCycles.
constexpr long long kBulkWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Thread of the caller's choice: orders earlier generic accesses of the CTA
// (made visible by a barrier) before the copy, arms the barrier with the
// byte count and starts the copy.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

// Waits for the phase of the given parity to complete; false once `limit`
// cycles have passed (at once, without polling, when limit <= 0).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, long long limit = kBulkWaitCycles) {
    if (limit <= 0) return false;
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// ------------------------------------------------------------ launchers
// Row compaction.  Rows of A without entries have none in C = A B, so the
// forward passes may number only the rows that hold entries: mark[r] = 1 for
// every row of an entry (in range), an inclusive scan of mark gives the count,
// k_row_map writes map[r] (compact index or -1) and inv[compact] = r, and
// k_row_remap rewrites A's rows through map, reporting a row without a
// compact index (kDetailRowMap).
__global__ void k_row_mark(const int32_t *Arow, int64_t nnz, int64_t m, int64_t *mark);
__global__ void k_row_map(const int64_t *incl, int64_t m, int32_t *map, int32_t *inv);
__global__ void k_row_remap(const int32_t *Arow, int64_t nnz, const int32_t *map, int64_t m, int32_t *out,
                            Ctrl *ctrl);

// Mapped pinned host buffer of small device -> host reads, grown on demand
// (at least 64 KiB).
struct Mirror {
    void *host = nullptr;
    void *dev = nullptr;
    size_t cap = 0;
    ~Mirror();
    cudaError_t reserve(size_t need);
};

// Small device -> host reads (control blocks, counts): a one-CTA kernel
// copies src0[0..n0) and src1[0..n1) into the mapped pinned mirror `m` (NULL:
// one of the calling host thread for the current device), the stream is
// synchronised and the bytes are copied to dst0 / dst1.  No copy engine is
// used, so these reads are not queued behind large copies that the caller
// has in flight on other streams.
cudaError_t readback(Mirror *m, void *dst0, const void *src0, size_t n0, void *dst1, const void *src1, size_t n1,
                     cudaStream_t s);
cudaError_t launch_inclusive_scan(int64_t *x, int64_t n, int64_t *tile_sums, cudaStream_t s);
int64_t scan_tile_count(int64_t n);

__global__ void k_validate(const int64_t *cp, const int32_t *row, int64_t nrows, int64_t ncols,
                           int64_t nnz, int which, Ctrl *ctrl);
__global__ void k_count_bin(const int64_t *Bcp, const int32_t *Brow, const int64_t *Acp, int64_t nB,
                            int64_t t, int64_t hmax, int promote, int64_t mrows, int64_t mult, int64_t *op,
                            int64_t *Ccp, Ctrl *ctrl);
// Multiplier coprime to n (n >= 1) near n times the golden ratio's fraction,
// dealing the columns of k_count_bin over the warps.
int64_t column_deal_mult(int64_t n);
__global__ void k_slot_caps(const int64_t *op, int64_t nB, int64_t mrows, int64_t *caps);
// Single pass: C's entries from the slots (two launches: the first column
// of every tile of C's positions into tile_col, copy_tile_count(nnzC) ints,
// then the tiles).
cudaError_t launch_slot_copy(int64_t nB, int64_t nnzC, const int64_t *Ccp, const int64_t *soff, int32_t *tile_col,
                             const int32_t *srow, const void *sval, int32_t *Crow, void *Cval, int w, int sms,
                             cudaStream_t s);
int64_t copy_tile_count(int64_t n);
__global__ void k_bin_scatter(const int64_t *op, int64_t nB, int64_t t, int64_t hmax, int promote,
                              BinOffsets off, int32_t *bin_cols, Ctrl *ctrl);

// Geometry of one phase (symbolic / numeric / backward) of one bin.
struct Geo {
    int threads = 0;       // threads per CTA
    int grid = 0;          // CTAs
    size_t smem = 0;       // dynamic shared memory
    int64_t slots = 0;     // table slots per CTA (CTA hash bins, global bin)
    bool bm_global = false;  // dense flags bitmap in global scratch
    int64_t cap = 0;       // dense bin: values kept in shared memory up to this nnz
    bool prefetch = false;   // dense bin: next column's kept flags staged by a bulk copy
};

// Everything a bin kernel needs, passed by value.
struct BinTask {
    const int32_t *cols;  // this bin's column ids
    int64_t count;
    int bin;
    int shrink;           // table_shrink test knob
    int64_t m;            // rows of A / C
    int64_t W;            // bitmap words = ceil(m / 32)
    const int64_t *op;    // Op_j
    unsigned char *scratch;  // per-CTA global scratch (base)
    size_t scratch_stride;   // bytes per CTA
    Ctrl *ctrl;
    uint32_t *flag_cache;    // dense bin: W words per listed column, for the
    int64_t cache_cols;      //   first cache_cols columns of the bin's list
    long long wait_cycles;   // dense bin: limit of a wait for kept flags (<= 0: give up at once)
    // single pass: the numeric kernels write each column at its slot (the
    // column pointers passed in are the slot offsets, slot capacity
    // min(Op_j, m)) and its entry count to cnt_out[j + 1]; null otherwise
    // (the count is checked against the symbolic phase's)
    int64_t *cnt_out = nullptr;
    int slots_pct = kDefaultSlotsPct;  // hash-table slots per output entry, per cent
};

struct Operands {
    const int64_t *Acp; const int32_t *Arow; const void *Aval;
    const int64_t *Bcp; const int32_t *Brow; const void *Bval;
    const int32_t *Rmap = nullptr;  // C's row of a compact row (numeric)
};

// symbolic.cu
cudaError_t launch_symbolic_bin(const BinTask &t, const Operands &o, int64_t *Ccp, const Geo &g,
                                cudaStream_t s);
Geo symbolic_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                      int64_t max_op, int shrink, int64_t scratch_ctas);
// numeric.cu
cudaError_t launch_numeric_bin(const BinTask &t, const Operands &o, const int64_t *Ccp,
                               int32_t *Crow, void *Cval, int dtype, const Geo &g, cudaStream_t s);
Geo numeric_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                     int64_t maxnnz, int dtype, int slots_pct, int64_t scratch_ctas);
// backward.cu
cudaError_t launch_backward_bin(const BinTask &t, const Operands &o, const int64_t *Ccp,
                                const int32_t *Crow, const void *dC, void *dA, void *dB,
                                int dtype, const Geo &g, cudaStream_t s);
Geo backward_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                      int64_t maxnnz, int dtype, int slots_pct, int64_t scratch_ctas);

// Table slots of the global-memory hash bin for a column with Op_j = op in a
// matrix with m rows (symbolic: keys only, load <= 1/2).
__host__ __device__ inline int64_t global_sym_slots(int64_t op, int64_t m) {
    int64_t need = 2 * (op < m ? op : m);
    int64_t p = 64;
    while (p < need) p <<= 1;
    return p;
}
// Table slots for a column with n outputs (numeric / backward): pct per
// cent of n, rounded up to a multiple of 32, at least 64 (the default
// kDefaultSlotsPct keeps the load at most 2/3).
__host__ __device__ inline int64_t num_slots(int64_t n, int pct = kDefaultSlotsPct) {
    int64_t s = (n * pct + 99) / 100;
    s = (s + 31) & ~int64_t(31);
    return s < 64 ? 64 : s;
}

}  // namespace spg
