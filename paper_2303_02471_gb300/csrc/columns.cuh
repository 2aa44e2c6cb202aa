// Per-column bodies of the accumulators, shared by the per-bin kernels of a
// single product and by the persistent kernels of the batched form.
//
//   symbolic  nnz(C_j):   group hash table / CTA hash table / dense flags
//   numeric   C[:, j]:    group hash + register sort / CTA hash + two-level
//                         bitmap extraction / dense SPA with rank-indexed values
//   backward  dA, dB:     the forward's products, each looking up dC_ij
//
// "Group" functions run on G lanes (G divides 32; mask = the group's lanes);
// "CTA" functions contain barriers and must be called by every thread of the
// block.  Table slots, bitmaps and scratch are passed in by the caller, which
// decides where they live (shared memory or the CTA's global scratch).
#pragma once

#include "kernels.cuh"

namespace spg {

// Typed operand views of one product.
template <typename VT>
struct TOps {
    const int64_t *Acp;
    const int32_t *Arow;
    const VT *Aval;
    const int64_t *Bcp;
    const int32_t *Brow;
    const VT *Bval;
    // C's row of a (compact) row of the walk; nullptr: the same row
    const int32_t *Rmap = nullptr;

    __device__ __forceinline__ int32_t crow(int32_t r) const { return Rmap ? __ldg(Rmap + r) : r; }
};

template <typename VT>
__device__ __forceinline__ TOps<VT> typed(const Operands &o) {
    return TOps<VT>{o.Acp, o.Arow, static_cast<const VT *>(o.Aval), o.Bcp, o.Brow, static_cast<const VT *>(o.Bval),
                    o.Rmap};
}

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

// Bytes of a CTA hash table with `cap` slots plus its extraction word list.
template <typename VT>
__host__ __device__ inline size_t cta_table_bytes(int64_t cap) {
    return al16((size_t)cap * 4) + al16((size_t)cap * sizeof(VT)) + al16((size_t)cap * 4);
}

// ================================================================ symbolic
// Distinct rows of column j, counted by a group's key table of H slots
// (2 G R for Op_j <= G R).  Returns the count on every lane of the group.
template <int G, int R>
__device__ __forceinline__ int sym_group_column(unsigned mask, const TOps<float> &o, int32_t j, int32_t *keys,
                                                uint32_t H, bool &ovf) {
    const int gl = threadIdx.x & (G - 1);
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) keys[i * G + gl] = kEmptyKey;
    __syncwarp(mask);
    int cnt = 0;
    group_products<G, false, float>(mask, o.Acp, o.Arow, nullptr, o.Brow, nullptr, o.Bcp[j], o.Bcp[j + 1],
                                    [&](int32_t row, float) {
                                        bool fresh;
                                        if (hash_insert(keys, H, row, fresh) < 0) ovf = true;
                                        cnt += fresh;
                                    });
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) cnt += __shfl_xor_sync(mask, cnt, d, G);
    return cnt;
}

// Distinct rows of column j by a CTA key table of H slots.  s_cnt: a shared
// counter.  Returns the count on every thread.
__device__ __forceinline__ int64_t sym_cta_column(const TOps<float> &o, int32_t j, int32_t *keys, uint32_t H,
                                                  const WalkSmem<float> &w, unsigned long long *s_cnt, bool &ovf) {
    for (uint32_t s = threadIdx.x; s < H; s += blockDim.x) keys[s] = kEmptyKey;
    if (threadIdx.x == 0) *s_cnt = 0;
    __syncthreads();
    unsigned cnt = 0;
    cta_walk<false, float>(o.Acp, o.Arow, nullptr, o.Brow, nullptr, o.Bcp[j], o.Bcp[j + 1], w,
                           [&](int32_t row, float) {
                               bool fresh;
                               if (hash_insert(keys, H, row, fresh) < 0) ovf = true;
                               cnt += fresh;
                           });
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(s_cnt, (unsigned long long)cnt);
    __syncthreads();
    const int64_t r = (int64_t)*s_cnt;
    __syncthreads();
    return r;
}

// Distinct rows of column j by SPA flags: a row is new when its bit was
// still clear (Algorithm 1's counter).  `bm` (W words) must be zero on entry
// and is zero again on return; `keep` (W words, may be null) receives the
// flags for the numeric phase.
__device__ __forceinline__ int64_t sym_dense_column(const TOps<float> &o, int32_t j, uint32_t *bm, int64_t W,
                                                    uint32_t *keep, const WalkSmem<float> &w,
                                                    unsigned long long *s_cnt) {
    // (a dense column has B entries, so the walk's barriers order this reset
    // before every add below)
    if (threadIdx.x == 0) *s_cnt = 0;
    // the OR's old value is not needed: the rows are counted afterwards with
    // popcounts while the words are copied out and cleared
    cta_walk<false, float, kSymWalkAhead>(o.Acp, o.Arow, nullptr, o.Brow, nullptr, o.Bcp[j], o.Bcp[j + 1], w,
                                          [&](int32_t row, float) { atomicOr(&bm[row >> 5], 1u << (row & 31)); });
    unsigned long long cnt = 0;
    const bool vec = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(bm) & 15) == 0 &&
                     (!keep || (reinterpret_cast<uintptr_t>(keep) & 15) == 0);
    if (vec) {
        uint4 *b4 = reinterpret_cast<uint4 *>(bm);
        uint4 *k4 = reinterpret_cast<uint4 *>(keep);
        const int W4 = (int)(W >> 2);
        for (int i = threadIdx.x; i < W4; i += blockDim.x) {
            const uint4 v = b4[i];
            cnt += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            if (keep) __stcs(k4 + i, v);  // read back by the numeric phase only
            b4[i] = make_uint4(0u, 0u, 0u, 0u);
        }
    } else {
        for (int i = threadIdx.x; i < (int)W; i += blockDim.x) {
            const uint32_t v = bm[i];
            cnt += __popc(v);
            if (keep) keep[i] = v;
            bm[i] = 0u;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(s_cnt, cnt);
    __syncthreads();
    const int64_t r = (int64_t)*s_cnt;
    __syncthreads();
    return r;
}

// ================================================================= numeric
// Column j by a group: hash accumulation (Section 3.2) in a table of H <= 2 G R
// slots, compaction, register bitonic sort, write at c0.  Returns false if
// the count differs from nn (with cnt_out: exceeds nn, the slot size; the
// count is then written to cnt_out[j + 1]).
template <int G, int R, typename VT>
__device__ __forceinline__ bool num_group_column(unsigned mask, const TOps<VT> &o, int32_t j, int64_t c0,
                                                 int64_t nn, int32_t *keys, VT *vals, uint32_t H, int32_t *Crow,
                                                 VT *Cval, bool &ovf, int64_t *cnt_out = nullptr) {
    const int gl = threadIdx.x & (G - 1);
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        keys[i * G + gl] = kEmptyKey;
        vals[i * G + gl] = VT(0);
    }
    __syncwarp(mask);
    group_products<G, true, VT>(mask, o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1],
                                [&](int32_t row, VT prod) {
                                    bool fresh;
                                    const int32_t slot = hash_insert(keys, H, row, fresh);
                                    if (slot < 0) ovf = true;
                                    else atomicAdd(&vals[slot], prod);
                                });
    __syncwarp(mask);
    // compact the occupied slots to the front of the table
    int32_t kk[2 * R];
    VT vv[2 * R];
    int pos[2 * R];
    int n = 0;
    const unsigned lane_base = (threadIdx.x & 31) & ~(G - 1);
    const unsigned below = (1u << gl) - 1u;
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        kk[i] = keys[i * G + gl];
        vv[i] = vals[i * G + gl];
        const bool occ = kk[i] != kEmptyKey;
        unsigned b = __ballot_sync(mask, occ) >> lane_base;
        if (G < 32) b &= (1u << (G & 31)) - 1u;
        pos[i] = occ ? n + __popc(b & below) : -1;
        n += __popc(b);
    }
    __syncwarp(mask);
#pragma unroll
    for (int i = 0; i < 2 * R; ++i)
        if (pos[i] >= 0 && pos[i] < G * R) {
            keys[pos[i]] = kk[i];
            vals[pos[i]] = vv[i];
        }
    __syncwarp(mask);
    int32_t key[R];
    VT val[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * G + gl;
        if (e < n) {
            key[r] = keys[e];
            val[r] = vals[e];
        } else {
            key[r] = 0x7fffffff;
            val[r] = VT(0);
        }
    }
    group_bitonic_sort<G, R, VT>(mask, key, val);
    if (cnt_out) {
        if (n > nn || n > G * R) return false;
        if (gl == 0) cnt_out[j + 1] = n;
    } else if (nn != n || n > G * R) {
        return false;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = r * G + gl;
        if (e < n) {
            Crow[c0 + e] = o.crow(key[r]);
            Cval[c0 + e] = val[r];
        }
    }
    return true;
}

// Column j by a CTA: hash accumulation in H slots, then the occupied rows are
// marked in the two-level bitmap (L0 W words, L1 ceil(W / 32) words, both
// zero on entry and on return) and written in ascending order with their
// values.  s_occ: shared counter.  Returns false on a count mismatch.
template <typename VT>
__device__ __forceinline__ bool num_cta_column(const TOps<VT> &o, int32_t j, int64_t c0, int64_t nn,
                                               int32_t *keys, VT *vals, int32_t *wlist, uint32_t H, uint32_t *L0,
                                               uint32_t *L1, int64_t W, const WalkSmem<VT> &w, unsigned *s_occ,
                                               int64_t *s_warp, int32_t *Crow, VT *Cval, bool &ovf,
                                               int64_t *cnt_out = nullptr) {
    for (uint32_t s = threadIdx.x; s < H; s += blockDim.x) {
        keys[s] = kEmptyKey;
        vals[s] = VT(0);
    }
    if (threadIdx.x == 0) *s_occ = 0;
    __syncthreads();
    cta_walk<true, VT>(o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1], w,
                       [&](int32_t row, VT prod) {
                           bool fresh;
                           const int32_t slot = hash_insert(keys, H, row, fresh);
                           if (slot < 0) ovf = true;
                           else atomicAdd(&vals[slot], prod);
                       });
    unsigned occ = 0;
    for (uint32_t s = threadIdx.x; s < H; s += blockDim.x) {
        const int32_t key = keys[s];
        if (key != kEmptyKey) {
            mark_row(L0, L1, key);
            ++occ;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) occ += __shfl_xor_sync(0xffffffffu, occ, d);
    if ((threadIdx.x & 31) == 0 && occ) atomicAdd(s_occ, occ);
    __syncthreads();
    const int64_t found = (int64_t)*s_occ;
    // single pass: nn is the slot size, the count is written
    const bool ok = cnt_out ? found <= nn : found == nn;
    if (cnt_out && ok && threadIdx.x == 0) cnt_out[j + 1] = found;
    const int64_t K = cta_list_words(L1, (W + 31) / 32, wlist, s_warp);
    cta_expand_words(L0, wlist, K, s_warp, [&](int32_t row, int64_t rank) {
        const int32_t slot = hash_find(keys, H, row);
        if (ok && slot >= 0) {
            Crow[c0 + rank] = o.crow(row);
            Cval[c0 + rank] = vals[slot];
        }
    });
    return ok;
}

// Column j by the dense SPA (Algorithm 1): flags as a bitmap (from `keep`
// when the symbolic phase kept them, else a first product walk), prefix
// counts, then every product is added at its row's position in the sorted
// column, and the rows are written in ascending order.  The sums of the
// first `cap` positions live in shared memory (s_acc), the others in place
// in C, so the shared-memory and the L2 atomic units both take products.
// bm (W uint2) is zero on entry and on return.  after_prefix() runs on
// every thread once the flags (and `keep`) have been read.  Returns false on
// a count mismatch.
template <typename VT, typename AP>
__device__ __forceinline__ bool num_dense_column(const TOps<VT> &o, int32_t j, int64_t c0, int64_t nn, uint2 *bm,
                                                 int64_t W, const uint32_t *keep, VT *s_acc, int64_t cap,
                                                 const WalkSmem<VT> &w, int64_t *s_warp, unsigned *s_next,
                                                 int32_t *Crow, VT *Cval, AP &&after_prefix,
                                                 int64_t *cnt_out = nullptr) {
    // the previous user of *s_next finished before the caller's last barrier
    if (threadIdx.x == 0) *s_next = (blockDim.x >> 5) * kVisitGroup;
    // flags kept from the symbolic phase are read straight into the prefix
    // pass; otherwise the walk sets them again
    if (!keep)
        cta_walk<false, VT, kSymWalkAhead>(o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1], w,
                            [&](int32_t row, VT) { atomicOr(&bm[row >> 5].x, 1u << (row & 31)); });
    const int64_t total = cta_bitmap_prefix(bm, W, keep, s_warp);
    after_prefix();
    // single pass: nn is the slot size, the count is written
    if (cnt_out ? total > nn : total != nn) {
        // the pattern changed since the symbolic phase: the caller reports
        // it and the column is left unwritten
        for (int i = threadIdx.x; i < (int)W; i += blockDim.x) bm[i].x = 0u;
        __syncthreads();
        return false;
    }
    if (cnt_out) {
        if (threadIdx.x == 0) cnt_out[j + 1] = total;
        nn = total;
    }
    // nn <= m < 2^31: positions are 32-bit
    const int32_t n32 = (int32_t)nn;
    // double sums always go to C in place (cap is 0 for them): a compile-time
    // 0 drops the shared-memory path and its registers from that kernel
    const int32_t ns = sizeof(VT) == 8 ? 0 : (int32_t)(nn < cap ? nn : cap);
    VT *gacc = Cval + c0;
    int32_t *crow = Crow + c0;
    // the extraction stages rows in the walk's scratch, free once cta_walk
    // has returned (it ends with a barrier): 20 bytes per thread
    static_assert(kVisitStage * 4 <= 32 * (16 + sizeof(float)), "visit staging exceeds the walk scratch");
    int32_t *stage = reinterpret_cast<int32_t *>(w.a0);
    for (int32_t i = threadIdx.x; i < ns; i += blockDim.x) s_acc[i] = VT(0);
    for (int32_t i = ns + threadIdx.x; i < n32; i += blockDim.x) gacc[i] = VT(0);
    __syncthreads();
    if (ns == 0) {  // every sum in C (uniform over the CTA)
        cta_walk<true, VT, kWalkAhead>(o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1], w,
                           [&](int32_t row, VT prod) { atomicAdd(&gacc[bitmap_rank(bm, row)], prod); });
        cta_bitmap_visit(bm, W, true, s_next, stage, [&](int32_t row) { return o.crow(row); },
                         [&](int32_t rank, int32_t r) { crow[rank] = r; });
    } else {
        cta_walk<true, VT, kWalkAhead>(o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1], w,
                           [&](int32_t row, VT prod) {
                               const int32_t r = bitmap_rank(bm, row);
                               if (r < ns) atomicAdd(&s_acc[r], prod);
                               else atomicAdd(&gacc[r], prod);
                           });
        cta_bitmap_visit(bm, W, true, s_next, stage, [&](int32_t row) { return o.crow(row); },
                         [&](int32_t rank, int32_t r) {
                             crow[rank] = r;
                             if (rank < ns) gacc[rank] = s_acc[rank];
                         });
    }
    __syncthreads();
    return true;
}

// ================================================================ backward
// One product of the backward walk for a lane group of width G: the lane's A
// entry qa (row, a), the owning B entry p (global index, or -1 for an idle
// lane) and b = B_kj.  Adds b * dC_ij to dA[qa] and reduces a * dC_ij over
// lanes of the same p (owners are non-decreasing across the group's lanes)
// before one add to dB[p].  Every lane of the group calls it from the same
// call site.
template <int G, typename VT, typename L>
__device__ __forceinline__ void bwd_product(unsigned mask, int32_t row, VT a, VT b, int64_t qa, int64_t p, VT *dA,
                                            VT *dB, L &&lookup) {
    const int gl = threadIdx.x & (G - 1);
    VT g = VT(0);
    if (p >= 0) g = lookup(row);
    if (p >= 0 && dA) atomicAdd(&dA[qa], b * g);
    if (!dB) return;
    VT v = p >= 0 ? a * g : VT(0);
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const VT o = __shfl_up_sync(mask, v, d, G);
        const int64_t po = __shfl_up_sync(mask, p, d, G);
        if (gl >= d && po == p) v += o;
    }
    const int64_t pn = __shfl_down_sync(mask, p, 1, G);
    if (p >= 0 && (gl == G - 1 || pn != p)) atomicAdd(&dB[p], v);
}

// Lanes of a group of G cover column j's products like group_products;
// every lane of the group calls step(row, a, b, qa, p) once per round from a
// single call site (p = -1 when the lane is idle).
template <int G, typename VT, typename S>
__device__ __forceinline__ void group_walk_bwd(unsigned mask, const TOps<VT> &o, int64_t p0, int64_t p1, S &&step) {
    const int gl = threadIdx.x & (G - 1);
    for (int64_t base = p0; base < p1; base += G) {
        const int64_t p = base + gl;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = o.Brow[p];
            a0 = o.Acp[k];
            z = static_cast<int>(o.Acp[k + 1] - a0);
            bv = o.Bval[p];
        }
        const int incl = group_incl_scan<G>(mask, z);
        const int total = __shfl_sync(mask, incl, G - 1, G);
        const int excl = incl - z;
        for (int q0 = 0; q0 < total; q0 += G) {
            const int q = q0 + gl;
            int s = 0;
#pragma unroll
            for (int st = G / 2; st > 0; st >>= 1) {
                const int ex = __shfl_sync(mask, excl, s + st, G);
                if (ex <= q) s += st;
            }
            const int64_t a0s = __shfl_sync(mask, a0, s, G);
            const int exs = __shfl_sync(mask, excl, s, G);
            const VT bvs = __shfl_sync(mask, bv, s, G);
            const bool on = q < total;
            const int64_t qa = on ? a0s + (q - exs) : 0;
            const int32_t row = on ? o.Arow[qa] : 0;
            const VT av = on ? o.Aval[qa] : VT(0);
            step(row, av, bvs, qa, on ? base + s : (int64_t)-1);
        }
    }
}

// Same chunking and window split as cta_walk (one list of non-empty entries);
// every lane of a warp calls step(...) once per window from a single call
// site (p = -1 when idle), so the segmented reduction is warp-wide.
// pidx: blockDim ints of shared memory.  Contains barriers.
template <typename VT, typename S>
__device__ __forceinline__ void cta_walk_bwd(const TOps<VT> &o, int64_t p0, int64_t p1, const WalkSmem<VT> &w,
                                             int32_t *pidx, S &&step) {
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    for (int64_t base = p0; base < p1; base += T) {
        const int64_t p = base + threadIdx.x;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = o.Brow[p];
            a0 = o.Acp[k];
            z = (int)(o.Acp[k + 1] - a0);
            bv = o.Bval[p];
        }
        int v[4] = {z, z > 0 ? 1 : 0, 0, 0};
        const int mz = z;
        int tot[4];
        cta_incl_scan4(v, w.warp, tot);
        if (z > 0) {
            const int i = v[1] - 1;
            w.key[i] = v[0] - mz;
            w.a0[i] = a0;
            w.bv[i] = bv;
            pidx[i] = (int32_t)threadIdx.x;
        }
        __syncthreads();
        const int total = tot[0], nz = tot[1];
        const int nwin = (total + 31) >> 5;
        const int win0 = (int)((int64_t)nwin * warp / nw), win1 = (int)((int64_t)nwin * (warp + 1) / nw);
        if (win0 < win1) {
            const int qs = win0 << 5;
            int s = 0, hi = nz - 1;
            while (s < hi) {
                const int mid = (s + hi + 1) >> 1;
                if (w.key[mid] <= qs) s = mid; else hi = mid - 1;
            }
            for (int win = win0; win < win1; ++win) {
                const int qf = win << 5;
                const int cand = s + 1 + lane;
                const int pos = cand < nz ? w.key[cand] - qf : 64;
                const unsigned bits = __reduce_or_sync(0xffffffffu, pos < 32 ? (1u << pos) : 0u);
                const int own = s + __popc(bits & upto);
                const int q = qf + lane;
                const bool on = q < total;
                const int64_t qa = on ? w.a0[own] + (q - w.key[own]) : 0;
                const int32_t row = on ? o.Arow[qa] : 0;
                const VT av = on ? o.Aval[qa] : VT(0);
                step(row, av, on ? w.bv[own] : VT(0), qa, on ? base + pidx[own] : (int64_t)-1);
                s += __popc(bits) + (__ballot_sync(0xffffffffu, pos == 32) ? 1 : 0);
            }
        }
        __syncthreads();
    }
}

// Backward of column j by a group: dC[:, j] into the group's table (H slots).
template <int G, typename VT>
__device__ __forceinline__ bool bwd_group_column(unsigned mask, const TOps<VT> &o, int32_t j, int64_t c0, int64_t c1,
                                                 const int32_t *Crow, const VT *dC, int32_t *keys, VT *vals,
                                                 uint32_t H, VT *dA, VT *dB) {
    const int gl = threadIdx.x & (G - 1);
    for (uint32_t i = gl; i < H; i += G) keys[i] = kEmptyKey;
    __syncwarp(mask);
    bool ok = true;
    for (int64_t e = c0 + gl; e < c1; e += G) {
        bool fresh;
        const int32_t slot = hash_insert(keys, H, Crow[e], fresh);
        if (slot >= 0) vals[slot] = dC[e];
        else ok = false;
    }
    __syncwarp(mask);
    auto lookup = [&](int32_t row) -> VT {
        const int32_t slot = hash_find(keys, H, row);
        return slot >= 0 ? vals[slot] : VT(0);
    };
    group_walk_bwd<G, VT>(mask, o, o.Bcp[j], o.Bcp[j + 1], [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
        bwd_product<G, VT>(mask, row, a, b, qa, p, dA, dB, lookup);
    });
    return ok;
}

// Backward of column j by a CTA with a hash table of H slots for dC[:, j].
template <typename VT>
__device__ __forceinline__ bool bwd_cta_column(const TOps<VT> &o, int32_t j, int64_t c0, int64_t nn,
                                               const int32_t *Crow, const VT *dC, int32_t *keys, VT *vals,
                                               uint32_t H, const WalkSmem<VT> &w, int32_t *pidx, VT *dA, VT *dB) {
    for (uint32_t s = threadIdx.x; s < H; s += blockDim.x) keys[s] = kEmptyKey;
    __syncthreads();
    bool ok = true;
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
        bool fresh;
        const int32_t slot = hash_insert(keys, H, Crow[c0 + e], fresh);
        if (slot >= 0) vals[slot] = dC[c0 + e];
        else ok = false;
    }
    __syncthreads();
    auto lookup = [&](int32_t row) -> VT {
        const int32_t slot = hash_find(keys, H, row);
        return slot >= 0 ? vals[slot] : VT(0);
    };
    cta_walk_bwd<VT>(o, o.Bcp[j], o.Bcp[j + 1], w, pidx, [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
        bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
    });
    return ok;
}

// Backward of column j through the dense flags: C's rows of the column set
// the bitmap (W uint2, zero on entry and on return) whose prefix counts give
// the position of dC_ij; dC[:, j] is copied to s_dc when it fits (cap).
template <typename VT>
__device__ __forceinline__ void bwd_dense_column(const TOps<VT> &o, int32_t j, int64_t c0, int64_t nn,
                                                 const int32_t *Crow, const VT *dC, uint2 *bm, int64_t W, VT *s_dc,
                                                 int64_t cap, const WalkSmem<VT> &w, int32_t *pidx, int64_t *s_warp,
                                                 VT *dA, VT *dB) {
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int32_t r = Crow[c0 + e];
        atomicOr(&bm[r >> 5].x, 1u << (r & 31));
    }
    __syncthreads();
    cta_bitmap_prefix(bm, W, nullptr, s_warp);
    const bool in_smem = nn <= cap;
    if (in_smem)
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) s_dc[e] = dC[c0 + e];
    __syncthreads();
    if (in_smem) {
        auto lookup = [&](int32_t row) -> VT { return s_dc[bitmap_rank(bm, row)]; };
        cta_walk_bwd<VT>(o, o.Bcp[j], o.Bcp[j + 1], w, pidx, [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
            bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
        });
    } else {
        const VT *gdc = dC + c0;
        auto lookup = [&](int32_t row) -> VT { return gdc[bitmap_rank(bm, row)]; };
        cta_walk_bwd<VT>(o, o.Bcp[j], o.Bcp[j + 1], w, pidx, [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
            bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
        });
    }
    for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) bm[Crow[c0 + e] >> 5].x = 0u;
    __syncthreads();
}

}  // namespace spg
