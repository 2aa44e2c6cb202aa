// Batched form: nb independent products C_i = A_i x B_i of uneven sizes and
// mixed dtypes.  The columns of all products form one column space (product
// i owns global columns [col0_i, col0_i + n_i)); Op_j and the bins are taken
// over that space, and each phase runs as ONE persistent kernel whose blocks
// pop work items from a global counter:
//   * a CTA item is one column of a CTA hash bin or of the dense bin;
//   * a group item is blockDim / G columns of a warp-group bin;
//   * in the symbolic and numeric phases, when no product has more than
//     32 * kWarpDenseWords rows, a dense item is blockDim / 32 columns of
//     the dense bin, one per warp.
// Items are ordered heaviest first (dense, then CTA bins from the largest,
// then the group bins), the GPU form of processing columns by decreasing
// Op_j (Section 3.1).  Per-column work is the same device code as the
// single-product kernels (columns.cuh); every product keeps its own dtype.
// The numeric launch can be captured into a CUDA graph and replayed.
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "columns.cuh"
#include "handle.cuh"

namespace spg {

// One product of the batch, in device memory.
struct BProb {
    const int64_t *Acp;
    const int32_t *Arow;
    const void *Aval;
    const int64_t *Bcp;
    const int32_t *Brow;
    const void *Bval;
    int64_t *Ccp;  // into the concatenated column pointers
    int32_t *Crow;
    void *Cval;
    const void *dC;
    void *dA;
    void *dB;
    int64_t m;     // rows of A and C
    int64_t n;     // columns of B and C
    int64_t col0;  // first global column
    int64_t t;     // H-HASH threshold of this product
    int32_t dtype;
    int32_t pad;
};

constexpr int kMaxItemBins = NBINS;

// Item layout of a persistent launch (passed by value).
struct BItems {
    int64_t off[kMaxItemBins + 1];  // item offsets per bin in launch order
    int32_t order[kMaxItemBins];    // bin of each item range
    int64_t nitems;
    int nranges;
    int dense_warp;  // dense items are groups of one column per warp
};

struct BTask {
    const BProb *prob;
    const int64_t *col0s;  // [nb + 1] first global column of every product
    int nb;
    const int32_t *cols;   // bin lists of global columns
    BinOffsets boff;       // list offsets per bin
    unsigned long long *hist;
    Ctrl *ctrl;
    int64_t hmax;          // hash_cta_max
    int64_t cap_cta;       // CTA hash table slots
    int64_t cap_dense;     // dense values kept in shared memory
    int64_t Wmax;          // largest bitmap (words) of a product with CTA-level columns
    int64_t cap_sym;       // symbolic CTA key table slots
    const int64_t *op;     // Op of every global column
    int shrink;
    int promote;           // group_promote: lane-group bins moved up
    int slots_pct;         // numeric / backward table slots per output entry, per cent
    unsigned long long *counter;
    // flags of per-warp dense columns kept from the symbolic phase: column k
    // of the dense list owns words [coff[k], coff[k] + W) of `cache` when
    // they end within cache_words (cache null: nothing kept)
    const int64_t *coff;
    uint32_t *cache;
    int64_t cache_words;
};

__device__ __forceinline__ int find_prob(const int64_t *col0s, int nb, int64_t g) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (col0s[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename VT>
__device__ __forceinline__ TOps<VT> prob_ops(const BProb &P) {
    return TOps<VT>{P.Acp, P.Arow, static_cast<const VT *>(P.Aval), P.Bcp, P.Brow, static_cast<const VT *>(P.Bval)};
}

// --------------------------------------------------------- count + bins
__global__ void k_bcount(BTask b, int64_t ntot, int64_t *op) {
    __shared__ unsigned long long s_hist[NBINS], s_max[NBINS], s_prod[NBINS], s_nb[NBINS];
    if (threadIdx.x < NBINS) s_hist[threadIdx.x] = s_max[threadIdx.x] = s_prod[threadIdx.x] = s_nb[threadIdx.x] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += stride) {
        const int p = find_prob(b.col0s, b.nb, g);
        const BProb &P = b.prob[p];
        const int64_t j = g - P.col0;
        const int64_t p0 = P.Bcp[j], p1 = P.Bcp[j + 1];
        int64_t s = 0;
        for (int64_t q = p0; q < p1; ++q) {
            const int32_t k = P.Brow[q];
            s += P.Acp[k + 1] - P.Acp[k];
        }
        op[g] = s;
        const int bin = bin_of(s, P.t, b.hmax, b.promote);
        atomicAdd(&s_hist[bin], 1ULL);
        atomicMax(&s_max[bin], (unsigned long long)s);
        if (s) atomicAdd(&s_prod[bin], (unsigned long long)s);
        if (p1 > p0) atomicAdd(&s_nb[bin], (unsigned long long)(p1 - p0));
        if (bin == BIN_EMPTY) P.Ccp[j + 1] = 0;
        if (j == 0) P.Ccp[0] = 0;
    }
    __syncthreads();
    if (threadIdx.x < NBINS && s_hist[threadIdx.x]) {
        atomicAdd(&b.ctrl->hist[threadIdx.x], s_hist[threadIdx.x]);
        atomicMax(&b.ctrl->maxop[threadIdx.x], s_max[threadIdx.x]);
        atomicAdd(&b.ctrl->binprod[threadIdx.x], s_prod[threadIdx.x]);
        atomicAdd(&b.ctrl->binnnzb[threadIdx.x], s_nb[threadIdx.x]);
        atomicAdd(&b.ctrl->products, s_prod[threadIdx.x]);
    }
}

// Flag words of every dense-list column (coff[k + 1]; coff[0] = 0): a scan
// then gives each column its place in the kept-flag cache.
__global__ void k_bcache_words(BTask b, int64_t ndense, int64_t *coff) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ndense; k += stride) {
        const int64_t g = b.cols[b.boff.v[BIN_DENSE] + k];
        const BProb &P = b.prob[find_prob(b.col0s, b.nb, g)];
        coff[k + 1] = (P.m + 31) / 32;
        if (k == 0) coff[0] = 0;
    }
}

__global__ void k_bscatter(BTask b, int64_t ntot, const int64_t *op, int32_t *cols) {
    __shared__ unsigned int s_cnt[NBINS];
    __shared__ unsigned long long s_base[NBINS];
    if (threadIdx.x < NBINS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bin = -1;
    unsigned r = 0;
    if (g < ntot) {
        const int p = find_prob(b.col0s, b.nb, g);
        bin = bin_of(op[g], b.prob[p].t, b.hmax, b.promote);
        if (bin != BIN_EMPTY) r = atomicAdd(&s_cnt[bin], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NBINS && s_cnt[threadIdx.x])
        s_base[threadIdx.x] = atomicAdd(&b.ctrl->fill[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
    __syncthreads();
    if (bin > BIN_EMPTY) cols[b.boff.v[bin] + (int64_t)s_base[bin] + r] = (int32_t)g;
}

// CSC checks over a list of matrices (the A's or the B's of the batch):
// colptr[0] = 0, colptr[n] = nnz, non-decreasing, rows in range.
struct VMat {
    const int64_t *cp;
    const int32_t *row;
    int64_t nrows, ncols, nnz, col0;
};

__global__ void k_bvalidate(const VMat *mats, int nm, const int64_t *col0s, int64_t ntot, int which, Ctrl *ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ntot; g += stride) {
        const int i = find_prob(col0s, nm, g);
        const VMat &M = mats[i];
        const int64_t j = g - M.col0;
        const int64_t c = M.cp[j], c1 = M.cp[j + 1];
        bool bad = c1 < c || c < 0 || c1 > M.nnz || (j == 0 && c != 0) || (j == M.ncols - 1 && c1 != M.nnz);
        if (!bad)
            for (int64_t e = c; e < c1; ++e) {
                const int32_t r = M.row[e];
                if (r < 0 || (int64_t)r >= M.nrows) { bad = true; break; }
            }
        if (bad) set_error(ctrl, SPG_ERR_INVALID, which, g);
    }
}

// Zero dA and dB of every product before the backward adds into them.
__global__ void k_bzero(BTask b, const int64_t *aoff, const int64_t *boff_e, int64_t na, int64_t nbe) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < na + nbe; e += stride) {
        const bool isA = e < na;
        const int64_t x = isA ? e : e - na;
        const int p = find_prob(isA ? aoff : boff_e, b.nb, x);
        const BProb &P = b.prob[p];
        void *d = isA ? P.dA : P.dB;
        if (!d) continue;
        const int64_t k = x - (isA ? aoff[p] : boff_e[p]);
        if (P.dtype == SPG_F64) static_cast<double *>(d)[k] = 0.0;
        else static_cast<float *>(d)[k] = 0.0f;
    }
}

// Concatenated column pointers: after the global scan, subtract each
// product's base (the running total before its segment).
__global__ void k_bbase(BTask b, const int64_t *ccp_all, int64_t *base) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < b.nb) base[p] = ccp_all[b.prob[p].Ccp - ccp_all];
}

__global__ void k_bfix(BTask b, int64_t *ccp_all, int64_t total, const int64_t *base, const int64_t *segs,
                       int64_t *nnz) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int p = find_prob(segs, b.nb, e);
        ccp_all[e] -= base[p];
        if (e == segs[p] + b.prob[p].n) nnz[p] = ccp_all[e];
    }
}

// ---------------------------------------------------- persistent kernels
// Smem layout of a CTA item: [walk][table | L0 | L1 | wlist] or [walk][bm | acc].
struct ItemRef {
    int bin;
    int64_t idx;  // index in the bin's range
};

__device__ __forceinline__ ItemRef item_ref(const BItems &it, int64_t item) {
    ItemRef r{-1, 0};
    for (int k = 0; k < it.nranges; ++k)
        if (item < it.off[k + 1]) {
            r.bin = it.order[k];
            r.idx = item - it.off[k];
            return r;
        }
    return r;
}

// ------------------------------------------------------ warp-dense items
// When every product's dense flags are short (at most kWarpDenseWords words),
// a dense column is worked by one warp, with its own flags in shared memory
// and warp-level synchronisation only: the column's fixed cost (clearing,
// prefix, extraction) is small and no CTA barrier is paid per column.
constexpr int64_t kWarpDenseWords = 1024;

// Position of row among the flagged rows of its column: the word's prefix
// count plus the flags below it in the word.
__device__ __forceinline__ int32_t warp_dense_rank(const uint2 *bm, int32_t row) {
    const uint2 e = bm[row >> 5];
    return (int32_t)e.y + __popc(e.x & ((1u << (row & 31)) - 1u));
}

// nnz of column j: flags set by the warp's product walk, then counted (and
// copied to `keep` when it is not null).
__device__ __forceinline__ int64_t warp_dense_symbolic(const TOps<float> &o, int32_t j, uint32_t *bm, int W,
                                                       uint32_t *keep) {
    const int lane = threadIdx.x & 31;
    for (int w = lane; w < W; w += 32) bm[w] = 0u;
    __syncwarp();
    group_products<32, false, float>(0xffffffffu, o.Acp, o.Arow, nullptr, o.Brow, nullptr, o.Bcp[j], o.Bcp[j + 1],
                                     [&](int32_t row, float) { atomicOr(&bm[row >> 5], 1u << (row & 31)); });
    __syncwarp();
    int64_t cnt = 0;
    for (int w = lane; w < W; w += 32) {
        const uint32_t x = bm[w];
        cnt += __popc(x);
        if (keep) keep[w] = x;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    return cnt;
}

// Column j by the dense SPA in one warp: flags (read from `keep` when the
// symbolic phase kept them, else set by a product walk), prefix counts (each
// lane a contiguous run of words, one warp scan), every product added at its
// row's position in place in C, then the rows written in order.  False on a
// count mismatch.
template <typename VT>
__device__ __forceinline__ bool warp_dense_numeric(const TOps<VT> &o, int32_t j, int64_t c0, int64_t nn, uint2 *bm,
                                                   int W, const uint32_t *keep, int32_t *Crow, VT *Cval) {
    const int lane = threadIdx.x & 31;
    if (keep) {
        // four loads in flight per lane before their stores (the kept flags
        // come from DRAM)
        for (int w0 = lane; w0 < W; w0 += 128) {
            uint32_t x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = w0 + 32 * u < W ? __ldg(keep + w0 + 32 * u) : 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (w0 + 32 * u < W) bm[w0 + 32 * u] = make_uint2(x[u], 0u);
        }
    } else {
        for (int w = lane; w < W; w += 32) bm[w] = make_uint2(0u, 0u);
        __syncwarp();
        group_products<32, false, VT>(0xffffffffu, o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1],
                                      [&](int32_t row, VT) { atomicOr(&bm[row >> 5].x, 1u << (row & 31)); });
    }
    __syncwarp();
    // an odd run per lane: the lanes' words fall in different shared-memory banks
    const int per = ((W + 31) >> 5) | 1;
    const int w0 = lane * per < W ? lane * per : W;
    const int w1 = w0 + per < W ? w0 + per : W;
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(bm[w].x);
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int run = incl - cnt;
    for (int w = w0; w < w1; ++w) {
        const uint32_t x = bm[w].x;
        bm[w].y = (uint32_t)run;
        run += __popc(x);
    }
    __syncwarp();
    if ((int64_t)total != nn) return false;
    VT *gacc = Cval + c0;
    int32_t *crow = Crow + c0;
    for (int i = lane; i < total; i += 32) gacc[i] = VT(0);
    __syncwarp();
    group_products<32, true, VT>(0xffffffffu, o.Acp, o.Arow, o.Aval, o.Brow, o.Bval, o.Bcp[j], o.Bcp[j + 1],
                                 [&](int32_t row, VT prod) { atomicAdd(&gacc[warp_dense_rank(bm, row)], prod); });
    for (int w = lane; w < W; w += 32) {
        uint32_t bits = bm[w].x;
        int32_t r = (int32_t)bm[w].y;
        while (bits) {
            const int q = __ffs(bits) - 1;
            bits &= bits - 1u;
            crow[r++] = (w << 5) + q;
        }
    }
    return true;
}

// Item idx of the dense bin in warp form: warp w of the CTA takes dense
// column idx * (warps per CTA) + w.
template <int phase>
__device__ __noinline__ void bdense_warp_item(const BTask &b, int64_t idx, unsigned char *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t k = idx * nw + warp;
    if (k >= (int64_t)b.hist[BIN_DENSE]) return;
    const int64_t g = b.cols[b.boff.v[BIN_DENSE] + k];
    const int p = find_prob(b.col0s, b.nb, g);
    const BProb &P = b.prob[p];
    const int64_t j = g - P.col0;
    const int W = (int)((P.m + 31) / 32);
    uint32_t *keep = nullptr;
    if (b.cache && b.coff[k] + W <= b.cache_words) keep = b.cache + b.coff[k];
    if (phase == 0) {
        uint32_t *bm = reinterpret_cast<uint32_t *>(smem + (size_t)warp * al16((size_t)b.Wmax * 4));
        const TOps<float> o{P.Acp, P.Arow, nullptr, P.Bcp, P.Brow, nullptr};
        const int64_t cnt = warp_dense_symbolic(o, (int32_t)j, bm, W, keep);
        if (lane == 0) {
            P.Ccp[j + 1] = cnt;
            atomicMax(&b.ctrl->maxnnz[BIN_DENSE], (unsigned long long)cnt);
            atomicAdd(&b.ctrl->binnnz[BIN_DENSE], (unsigned long long)cnt);
        }
    } else {
        uint2 *bm = reinterpret_cast<uint2 *>(smem + (size_t)warp * al16((size_t)b.Wmax * 8));
        const int64_t c0 = P.Ccp[j], nn = P.Ccp[j + 1] - c0;
        const bool ok = P.dtype == SPG_F64
                            ? warp_dense_numeric<double>(prob_ops<double>(P), (int32_t)j, c0, nn, bm, W, keep,
                                                         P.Crow, static_cast<double *>(P.Cval))
                            : warp_dense_numeric<float>(prob_ops<float>(P), (int32_t)j, c0, nn, bm, W, keep,
                                                        P.Crow, static_cast<float *>(P.Cval));
        if (!ok && lane == 0) set_error(b.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + BIN_DENSE, j);
    }
}

template <int G, int R, typename VT>
__device__ __forceinline__ void bnum_group(const BTask &b, const BProb &P, int64_t j, unsigned char *smem,
                                           int bin) {
    constexpr int H = 2 * G * R;
    const int NG = blockDim.x / G;
    const int grp = threadIdx.x / G;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * H;
    // value slots of a group are strided by 8 bytes whatever the dtype: groups
    // of one tile may belong to products of different dtypes
    VT *vals = reinterpret_cast<VT *>(smem + al16((size_t)NG * H * 4) + (size_t)grp * H * 8);
    uint32_t Hj = (uint32_t)H >> b.shrink;
    if (Hj < 1) Hj = 1;
    const int64_t c0 = P.Ccp[j];
    bool ovf = false;
    const bool ok = num_group_column<G, R, VT>(group_mask(G), prob_ops<VT>(P), (int32_t)j, c0, P.Ccp[j + 1] - c0,
                                               keys, vals, Hj, P.Crow, static_cast<VT *>(P.Cval), ovf);
    if (ovf) set_error(b.ctrl, SPG_ERR_TABLE_OVERFLOW, bin, j);
    if (!ok) set_error(b.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + bin, j);
}

template <typename VT>
__device__ __noinline__ void bnum_cta(const BTask &b, const BProb &P, int64_t j, unsigned char *smem,
                                         int64_t *s_warp, unsigned *s_occ, int bin) {
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    unsigned char *p = smem + walk_smem_bytes<VT>(blockDim.x);
    const int64_t W = (P.m + 31) / 32;
    const int64_t c0 = P.Ccp[j], nn = P.Ccp[j + 1] - c0;
    if (bin == BIN_DENSE) {
        uint2 *bm = reinterpret_cast<uint2 *>(p);
        VT *acc = reinterpret_cast<VT *>(p + al16((size_t)b.Wmax * 8));
        for (int64_t i = threadIdx.x; i < W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
        __syncthreads();
        // double sums go to C in place (RED.F64 beats shared-memory f64
        // atomics on GB300); float sums stay in shared memory
        const int64_t cap = sizeof(VT) == 8 ? 0 : b.cap_dense;
        const bool ok = num_dense_column<VT>(prob_ops<VT>(P), (int32_t)j, c0, nn, bm, W, nullptr, acc, cap, w,
                                             s_warp, s_occ, P.Crow, static_cast<VT *>(P.Cval), []() {});
        if (!ok && threadIdx.x == 0) set_error(b.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + bin, j);
        return;
    }
    const int64_t cap = b.cap_cta;
    int32_t *keys = reinterpret_cast<int32_t *>(p);
    VT *vals = reinterpret_cast<VT *>(p + al16((size_t)cap * 4));
    int32_t *wlist = reinterpret_cast<int32_t *>(p + al16((size_t)cap * 4) + al16((size_t)cap * sizeof(VT)));
    uint32_t *L0 = reinterpret_cast<uint32_t *>(p + cta_table_bytes<VT>(cap));
    uint32_t *L1 = reinterpret_cast<uint32_t *>(p + cta_table_bytes<VT>(cap) + al16((size_t)b.Wmax * 4));
    for (int64_t i = threadIdx.x; i < W; i += blockDim.x) L0[i] = 0u;
    for (int64_t i = threadIdx.x; i < (W + 31) / 32; i += blockDim.x) L1[i] = 0u;
    __syncthreads();
    int64_t want = num_slots(nn, b.slots_pct);
    if (want > cap) want = cap;
    uint32_t H = (uint32_t)(want >> b.shrink);
    if (H < 1) H = 1;
    bool ovf = false;
    const bool ok = num_cta_column<VT>(prob_ops<VT>(P), (int32_t)j, c0, nn, keys, vals, wlist, H, L0, L1, W, w,
                                       s_occ, s_warp, P.Crow, static_cast<VT *>(P.Cval), ovf);
    if (ovf) set_error(b.ctrl, SPG_ERR_TABLE_OVERFLOW, bin, j);
    if (!ok && threadIdx.x == 0) set_error(b.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + bin, j);
}

// Group items: blockDim / G columns of one warp bin; each group may belong
// to a different product (and dtype).
template <int G, int R>
__device__ __forceinline__ void bgroup_item(const BTask &b, int bin, int64_t idx, unsigned char *smem, int phase) {
    const int NG = blockDim.x / G;
    const int64_t ci = idx * NG + threadIdx.x / G;
    const int64_t count = (int64_t)b.hist[bin];
    if (ci >= count) return;
    const int64_t g = b.cols[b.boff.v[bin] + ci];
    const int p = find_prob(b.col0s, b.nb, g);
    const BProb &P = b.prob[p];
    const int64_t j = g - P.col0;
    if (phase == 0) {  // symbolic
        constexpr int H = 2 * G * R;
        int32_t *keys = reinterpret_cast<int32_t *>(smem) + (threadIdx.x / G) * H;
        uint32_t Hj = (uint32_t)H >> b.shrink;
        if (Hj < 1) Hj = 1;
        bool ovf = false;
        const TOps<float> o{P.Acp, P.Arow, nullptr, P.Bcp, P.Brow, nullptr};
        const int cnt = sym_group_column<G, R>(group_mask(G), o, (int32_t)j, keys, Hj, ovf);
        if (ovf) set_error(b.ctrl, SPG_ERR_TABLE_OVERFLOW, bin, g);
        if ((threadIdx.x & (G - 1)) == 0) {
            P.Ccp[j + 1] = cnt;
            atomicMax(&b.ctrl->maxnnz[bin], (unsigned long long)cnt);
            atomicAdd(&b.ctrl->binnnz[bin], (unsigned long long)cnt);
        }
    } else if (phase == 1) {  // numeric
        if (P.dtype == SPG_F64) bnum_group<G, R, double>(b, P, j, smem, bin);
        else bnum_group<G, R, float>(b, P, j, smem, bin);
    } else {  // backward
        constexpr int H = 2 * G * R;
        const int grp = threadIdx.x / G;
        int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * H;
        unsigned char *vb = smem + al16((size_t)NG * H * 4);
        bool ok;
        if (P.dtype == SPG_F64)
            ok = bwd_group_column<G, double>(group_mask(G), prob_ops<double>(P), (int32_t)j, P.Ccp[j], P.Ccp[j + 1],
                                             P.Crow, static_cast<const double *>(P.dC), keys,
                                             reinterpret_cast<double *>(vb + (size_t)grp * H * 8), (uint32_t)H,
                                             static_cast<double *>(P.dA), static_cast<double *>(P.dB));
        else
            ok = bwd_group_column<G, float>(group_mask(G), prob_ops<float>(P), (int32_t)j, P.Ccp[j], P.Ccp[j + 1],
                                            P.Crow, static_cast<const float *>(P.dC), keys,
                                            reinterpret_cast<float *>(vb + (size_t)grp * H * 8), (uint32_t)H,
                                            static_cast<float *>(P.dA), static_cast<float *>(P.dB));
        if (!ok) set_error(b.ctrl, SPG_ERR_TABLE_OVERFLOW, bin, g);
    }
}

__device__ __noinline__ void bgroup_dispatch(const BTask &b, int bin, int64_t idx, unsigned char *smem, int phase) {
    switch (bin - BIN_WARP0) {
        case 0: bgroup_item<warp_bin_G(0), warp_bin_R(0)>(b, bin, idx, smem, phase); break;
        case 1: bgroup_item<warp_bin_G(1), warp_bin_R(1)>(b, bin, idx, smem, phase); break;
        case 2: bgroup_item<warp_bin_G(2), warp_bin_R(2)>(b, bin, idx, smem, phase); break;
        case 3: bgroup_item<warp_bin_G(3), warp_bin_R(3)>(b, bin, idx, smem, phase); break;
        case 4: bgroup_item<warp_bin_G(4), warp_bin_R(4)>(b, bin, idx, smem, phase); break;
        default: bgroup_item<warp_bin_G(5), warp_bin_R(5)>(b, bin, idx, smem, phase); break;
    }
}

// phase 0: symbolic, 1: numeric, 2: backward.  One launch per phase.
// One instantiation per phase, so each carries only its own code paths
// (and registers).
template <int phase>
__global__ void __launch_bounds__(512, 2) k_batched(BTask b, BItems it) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_item;
    __shared__ int64_t s_warp[32];
    __shared__ unsigned s_occ;
    __shared__ unsigned long long s_cnt;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(b.counter, 1ULL);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= it.nitems) break;
        const ItemRef r = item_ref(it, item);
        if (r.bin >= BIN_WARP0 && r.bin < BIN_CTA0) {
            bgroup_dispatch(b, r.bin, r.idx, smem, phase);
        } else if (phase < 2 && r.bin == BIN_DENSE && it.dense_warp) {
            if constexpr (phase < 2) bdense_warp_item<phase>(b, r.idx, smem);
        } else {
            const int64_t g = b.cols[b.boff.v[r.bin] + r.idx];
            const int p = find_prob(b.col0s, b.nb, g);
            const BProb &P = b.prob[p];
            const int64_t j = g - P.col0;
            const int64_t W = (P.m + 31) / 32;
            if (phase == 0) {
                const WalkSmem<float> w = carve_walk<float>(smem);
                unsigned char *q = smem + walk_smem_bytes<float>(blockDim.x);
                const TOps<float> o{P.Acp, P.Arow, nullptr, P.Bcp, P.Brow, nullptr};
                int64_t cnt;
                if (r.bin == BIN_DENSE) {
                    uint32_t *bm = reinterpret_cast<uint32_t *>(q);
                    for (int64_t i = threadIdx.x; i < W; i += blockDim.x) bm[i] = 0u;
                    __syncthreads();
                    cnt = sym_dense_column(o, (int32_t)j, bm, W, nullptr, w, &s_cnt);
                } else {
                    int64_t H = global_sym_slots(b.op[g], P.m);
                    if (H > b.cap_sym) H = b.cap_sym;
                    uint32_t Hs = (uint32_t)(H >> b.shrink);
                    if (Hs < 1) Hs = 1;
                    bool ovf = false;
                    cnt = sym_cta_column(o, (int32_t)j, reinterpret_cast<int32_t *>(q), Hs, w, &s_cnt, ovf);
                    if (ovf) set_error(b.ctrl, SPG_ERR_TABLE_OVERFLOW, r.bin, g);
                }
                if (threadIdx.x == 0) {
                    P.Ccp[j + 1] = cnt;
                    atomicMax(&b.ctrl->maxnnz[r.bin], (unsigned long long)cnt);
                    atomicAdd(&b.ctrl->binnnz[r.bin], (unsigned long long)cnt);
                }
            } else if (phase == 1) {
                if (P.dtype == SPG_F64) bnum_cta<double>(b, P, j, smem, s_warp, &s_occ, r.bin);
                else bnum_cta<float>(b, P, j, smem, s_warp, &s_occ, r.bin);
            } else {
                const int64_t c0 = P.Ccp[j], nn = P.Ccp[j + 1] - c0;
                if (P.dtype == SPG_F64) {
                    const WalkSmem<double> w = carve_walk<double>(smem);
                    unsigned char *q = smem + walk_smem_bytes<double>(blockDim.x);
                    int32_t *pidx = reinterpret_cast<int32_t *>(q);
                    q += al16((size_t)blockDim.x * 4);
                    uint2 *bm = reinterpret_cast<uint2 *>(q);
                    double *dc = reinterpret_cast<double *>(q + al16((size_t)b.Wmax * 8));
                    for (int64_t i = threadIdx.x; i < W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
                    __syncthreads();
                    bwd_dense_column<double>(prob_ops<double>(P), (int32_t)j, c0, nn, P.Crow,
                                             static_cast<const double *>(P.dC), bm, W, dc, b.cap_dense, w, pidx,
                                             s_warp, static_cast<double *>(P.dA), static_cast<double *>(P.dB));
                } else {
                    const WalkSmem<float> w = carve_walk<float>(smem);
                    unsigned char *q = smem + walk_smem_bytes<float>(blockDim.x);
                    int32_t *pidx = reinterpret_cast<int32_t *>(q);
                    q += al16((size_t)blockDim.x * 4);
                    uint2 *bm = reinterpret_cast<uint2 *>(q);
                    float *dc = reinterpret_cast<float *>(q + al16((size_t)b.Wmax * 8));
                    for (int64_t i = threadIdx.x; i < W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
                    __syncthreads();
                    bwd_dense_column<float>(prob_ops<float>(P), (int32_t)j, c0, nn, P.Crow,
                                            static_cast<const float *>(P.dC), bm, W, dc, b.cap_dense, w, pidx,
                                            s_warp, static_cast<float *>(P.dA), static_cast<float *>(P.dB));
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace spg

// ====================================================================== host
using namespace spg;

namespace {

size_t al256b(size_t v) { return (v + 255) & ~size_t(255); }

struct BLayout {
    size_t ctrl, prob, col0s, segs, base, nnz, aoff, boffe, vA, vB, acol0, op, cols, tiles, coff, cache, total;
};

// Bytes of kept dense flags of a batch: only when its dense columns run one
// per warp (every product at most 32 * kWarpDenseWords rows), at most the
// flags of every column, at most cfg.dense_cache_bytes.
size_t batch_cache_bytes(int nb, const spg_csc *A, const spg_csc *B, const spg_config &c) {
    int64_t mmax = 0, words = 0;
    for (int i = 0; i < nb; ++i) {
        mmax = std::max<int64_t>(mmax, A[i].nrows);
        words += B[i].ncols * ceil_div(A[i].nrows, 32);
    }
    if (c.dense_cache_bytes <= 0 || ceil_div(mmax, 32) > kWarpDenseWords) return 0;
    return (size_t)std::min<int64_t>(words, c.dense_cache_bytes / 4) * 4;
}

BLayout blayout(int nb, int64_t ntot, int64_t ntotA, int64_t ncp, size_t cache_bytes) {
    BLayout L{};
    size_t off = 0;
    L.ctrl = off; off = al256b(off + sizeof(Ctrl));
    L.prob = off; off = al256b(off + (size_t)nb * sizeof(BProb));
    L.col0s = off; off = al256b(off + (size_t)(nb + 1) * 8);
    L.segs = off; off = al256b(off + (size_t)(nb + 1) * 8);
    L.base = off; off = al256b(off + (size_t)nb * 8);
    L.nnz = off; off = al256b(off + (size_t)nb * 8);
    L.aoff = off; off = al256b(off + (size_t)(nb + 1) * 8);
    L.boffe = off; off = al256b(off + (size_t)(nb + 1) * 8);
    L.vA = off; off = al256b(off + (size_t)nb * sizeof(VMat));
    L.vB = off; off = al256b(off + (size_t)nb * sizeof(VMat));
    L.acol0 = off; off = al256b(off + (size_t)(nb + 1) * 8);
    L.op = off; off = al256b(off + (size_t)ntot * 8);
    L.cols = off; off = al256b(off + (size_t)ntot * 4);
    L.tiles = off; off = al256b(off + (size_t)scan_tile_count(ncp) * 8);
    L.coff = off; off = al256b(off + (cache_bytes ? (size_t)(ntot + 1) * 8 : 0));
    L.cache = off; off = al256b(off + cache_bytes);
    L.total = off;
    (void)ntotA;
    return L;
}

int64_t prob_t(const spg_config &c, int64_t m) {
    // the batched kernels have no global-memory hash tables: t <= hmax + 1
    int64_t t = c.t;
    if (t < 0) {
        t = (m + 127) / 128;
        if (t < 257) t = 257;
    }
    if (t > (int64_t)c.hash_cta_max + 1) t = (int64_t)c.hash_cta_max + 1;
    return t;
}

}  // namespace

struct spg_bplan {
    spg_handle *h = nullptr;  // read-backs through the handle's buffer (NULL: the thread's)
    int nb = 0;
    int device = 0;
    int sms = 1;
    size_t smem_optin = 0;
    spg_config cfg{};
    unsigned char *ws = nullptr;
    BLayout L{};
    int64_t ntot = 0, ncp = 0, na = 0, nbe = 0;
    std::vector<BProb> prob;  // host copy of the problem table
    std::vector<int64_t> nnz;
    Ctrl host{};
    BinOffsets off{};
    int64_t Wmax = 0, mmax = 0;
    int64_t cache_words = 0;  // kept dense flags (0: none)
    int threads = 256;
    bool any_f64 = false;
    // numeric graph
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<BProb> graph_prob;
    int64_t launches_sym = 0;
    ~spg_bplan() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
    }
    Ctrl *ctrl() const { return reinterpret_cast<Ctrl *>(ws + L.ctrl); }
    BTask task() const {
        BTask b{};
        b.prob = reinterpret_cast<const BProb *>(ws + L.prob);
        b.col0s = reinterpret_cast<const int64_t *>(ws + L.col0s);
        b.nb = nb;
        b.cols = reinterpret_cast<const int32_t *>(ws + L.cols);
        b.boff = off;
        b.hist = ctrl()->hist;
        b.ctrl = ctrl();
        b.hmax = cfg.hash_cta_max;
        b.op = reinterpret_cast<const int64_t *>(ws + L.op);
        b.shrink = cfg.table_shrink;
        b.promote = cfg.group_promote;
        b.slots_pct = cfg.table_slots_pct;
        b.counter = &ctrl()->work[0];
        b.Wmax = Wmax;
        if (cache_words > 0) {
            b.coff = reinterpret_cast<const int64_t *>(ws + L.coff);
            b.cache = reinterpret_cast<uint32_t *>(ws + L.cache);
            b.cache_words = cache_words;
        }
        return b;
    }
};

namespace {

// Dense columns of the forward phases are worked one per warp when every
// product's flags fit kWarpDenseWords words.
bool warp_dense(const spg_bplan &P, int phase) {
    return phase < 2 && P.host.hist[BIN_DENSE] != 0 && P.Wmax <= kWarpDenseWords;
}

// Items of a phase, heaviest first.
BItems make_items(const spg_bplan &P, int threads, int phase) {
    BItems it{};
    int k = 0;
    int64_t acc = 0;
    it.off[0] = 0;
    auto add = [&](int bin, int64_t n) {
        if (n <= 0) return;
        it.order[k] = bin;
        acc += n;
        it.off[++k] = acc;
    };
    it.dense_warp = warp_dense(P, phase) ? 1 : 0;
    add(BIN_DENSE, it.dense_warp ? ceil_div((int64_t)P.host.hist[BIN_DENSE], threads / 32)
                                 : (int64_t)P.host.hist[BIN_DENSE]);
    for (int c = kNumCtaBins - 1; c >= 0; --c) add(BIN_CTA0 + c, (int64_t)P.host.hist[BIN_CTA0 + c]);
    for (int w = kNumWarpBins - 1; w >= 0; --w) {
        const int NG = threads / warp_bin_G(w);
        add(BIN_WARP0 + w, ceil_div((int64_t)P.host.hist[BIN_WARP0 + w], NG));
    }
    it.nranges = k;
    it.nitems = acc;
    return it;
}

// Shared memory of a phase's persistent launch (the largest item kind present).
size_t phase_smem(const spg_bplan &P, int phase, int threads, int64_t &cap_cta, int64_t &cap_dense, int64_t &cap_sym) {
    const size_t w = P.any_f64 ? 8 : 4;
    const size_t walk = P.any_f64 ? walk_smem_bytes<double>(threads) : walk_smem_bytes<float>(threads);
    const int64_t W1 = ceil_div(P.Wmax, 32);
    size_t need = 0;
    for (int b = 0; b < kNumWarpBins; ++b)
        if (P.host.hist[BIN_WARP0 + b])
            need = std::max(need, al16((size_t)threads * 2 * warp_bin_R(b) * 4) +
                                      (size_t)threads * 2 * warp_bin_R(b) * 8);
    bool cta = false;
    int64_t maxop = 0, maxnnz = 0;
    for (int c = 0; c < kNumCtaBins; ++c)
        if (P.host.hist[BIN_CTA0 + c]) {
            cta = true;
            maxop = std::max<int64_t>(maxop, (int64_t)P.host.maxop[BIN_CTA0 + c]);
            maxnnz = std::max<int64_t>(maxnnz, (int64_t)P.host.maxnnz[BIN_CTA0 + c]);
        }
    const bool wd = warp_dense(P, phase);
    const bool dense = P.host.hist[BIN_DENSE] != 0 && !wd;
    if (wd) need = std::max(need, (size_t)(threads / 32) * al16((size_t)P.Wmax * (phase == 0 ? 4 : 8)));
    cap_sym = cta ? global_sym_slots(maxop, P.mmax) : 0;
    cap_cta = cta ? num_slots(maxnnz, P.cfg.table_slots_pct) : 0;
    if (phase == 0) {
        if (cta) need = std::max(need, walk_smem_bytes<float>(threads) + (size_t)cap_sym * 4);
        if (dense) need = std::max(need, walk_smem_bytes<float>(threads) + (size_t)P.Wmax * 4);
        cap_dense = 0;
        return need;
    }
    const size_t fixed = walk + (phase == 2 ? al16((size_t)threads * 4) : 0) + al16((size_t)P.Wmax * 8);
    const size_t room = P.smem_optin > fixed ? P.smem_optin - fixed : 0;
    cap_dense = std::min<int64_t>((int64_t)(room / w), (int64_t)P.host.maxnnz[BIN_DENSE]);
    if (phase == 2) {
        // CTA-level columns of the backward all use the dense lookup
        int64_t mx = (int64_t)P.host.maxnnz[BIN_DENSE];
        for (int c = 0; c < kNumCtaBins; ++c) mx = std::max<int64_t>(mx, (int64_t)P.host.maxnnz[BIN_CTA0 + c]);
        cap_dense = std::min<int64_t>((int64_t)(room / w), mx);
        if (cta || dense) need = std::max(need, fixed + (size_t)cap_dense * w);
        return need;
    }
    if (dense) need = std::max(need, fixed + (size_t)cap_dense * w);
    if (cta)
        need = std::max(need, walk + (P.any_f64 ? cta_table_bytes<double>(cap_cta) : cta_table_bytes<float>(cap_cta)) +
                                  al16((size_t)P.Wmax * 4) + al16((size_t)W1 * 4));
    return need;
}

const void *batched_kernel(int phase) {
    return phase == 0 ? reinterpret_cast<const void *>(k_batched<0>)
                      : phase == 1 ? reinterpret_cast<const void *>(k_batched<1>)
                                   : reinterpret_cast<const void *>(k_batched<2>);
}

// Launch shape of a phase; the function attribute is set here, outside any
// stream capture.
struct PhaseLaunch {
    BTask b;
    BItems it;
    size_t smem = 0;
    int grid = 0;
};

spg_status prepare_phase(spg_bplan &P, int phase, PhaseLaunch &L) {
    int64_t cap_cta = 0, cap_dense = 0, cap_sym = 0;
    const int threads = P.threads;
    L.smem = phase_smem(P, phase, threads, cap_cta, cap_dense, cap_sym);
    if (L.smem > P.smem_optin) return SPG_ERR_UNSUPPORTED;
    L.b = P.task();
    L.b.cap_cta = cap_cta;
    L.b.cap_dense = cap_dense;
    L.b.cap_sym = cap_sym;
    L.it = make_items(P, threads, phase);
    const void *kfn = batched_kernel(phase);
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(L.smem, 1)) != cudaSuccess)
        return SPG_ERR_CUDA;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, threads, L.smem) != cudaSuccess || occ < 1)
        occ = 1;
    L.grid = (int)std::min<int64_t>(std::max<int64_t>(L.it.nitems, 1), (int64_t)occ * P.sms);
    return SPG_OK;
}

// Work counter reset + the persistent launch (both captured when capturing).
spg_status enqueue_phase(const spg_bplan &P, int phase, const PhaseLaunch &L, cudaStream_t s) {
    if (cudaMemsetAsync(L.b.counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return SPG_ERR_CUDA;
    if (L.it.nitems == 0) return SPG_OK;
    if (phase == 0) k_batched<0><<<L.grid, P.threads, L.smem, s>>>(L.b, L.it);
    else if (phase == 1) k_batched<1><<<L.grid, P.threads, L.smem, s>>>(L.b, L.it);
    else k_batched<2><<<L.grid, P.threads, L.smem, s>>>(L.b, L.it);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

spg_status launch_phase(spg_bplan &P, int phase, cudaStream_t s) {
    PhaseLaunch L;
    spg_status st = prepare_phase(P, phase, L);
    if (st != SPG_OK) return st;
    return enqueue_phase(P, phase, L, s);
}

spg_status check_batch(int32_t nb, const spg_csc *A, const spg_csc *B) {
    if (nb < 0 || (nb > 0 && (!A || !B))) return SPG_ERR_INVALID;
    for (int i = 0; i < nb; ++i) {
        const spg_csc &a = A[i], &b = B[i];
        if (a.nrows < 0 || a.ncols < 0 || a.nnz < 0 || b.nrows < 0 || b.ncols < 0 || b.nnz < 0) return SPG_ERR_INVALID;
        if (a.nrows > INT32_MAX || a.ncols > INT32_MAX || b.ncols > INT32_MAX) return SPG_ERR_INDEX_OVERFLOW;
        if (a.ncols != b.nrows || a.dtype != b.dtype || (a.dtype != SPG_F64 && a.dtype != SPG_F32)) return SPG_ERR_INVALID;
        if (!a.colptr || !b.colptr || (a.nnz > 0 && !a.rowidx) || (b.nnz > 0 && !b.rowidx)) return SPG_ERR_INVALID;
        if ((a.ncols == 0 && a.nnz != 0) || (b.ncols == 0 && b.nnz != 0)) return SPG_ERR_INVALID;
    }
    return SPG_OK;
}

}  // namespace

extern "C" {

spg_status spgemm_batched_workspace_size(int32_t nb, const spg_csc *A, const spg_csc *B, const spg_config *cfg,
                                         size_t *bytes) {
    if (!bytes) return SPG_ERR_INVALID;
    spg_status st = check_batch(nb, A, B);
    if (st != SPG_OK) return st;
    spg_config c;
    spg_config_default(&c);
    if (cfg) c = *cfg;
    int64_t ntot = 0, ntotA = 0, ncp = 0;
    for (int i = 0; i < nb; ++i) {
        ntot += B[i].ncols;
        ntotA += A[i].ncols;
        ncp += B[i].ncols + 1;
    }
    *bytes = blayout(nb, ntot, ntotA, ncp, batch_cache_bytes(nb, A, B, c)).total;
    return SPG_OK;
}

spg_status spgemm_batched_symbolic(spg_handle *handle, int32_t nb, const spg_csc *A, const spg_csc *B,
                                   const spg_config *cfg, void *workspace, size_t ws_bytes, int64_t *C_colptr,
                                   int64_t *nnzC, spg_bplan **plan_out, spg_stream stream) {
    if (plan_out) *plan_out = nullptr;
    if (!plan_out || (nb > 0 && (!C_colptr || !nnzC))) return SPG_ERR_INVALID;
    spg_status st = check_batch(nb, A, B);
    if (st != SPG_OK) return st;
    spg_config c;
    spg_config_default(&c);
    if (cfg) c = *cfg;
    if (c.cta_threads < 128 || c.cta_threads > 1024 || c.cta_threads % 32) return SPG_ERR_INVALID;
    if (!(c.hash_cta_max == 256 || c.hash_cta_max == 512 || c.hash_cta_max == 1024 || c.hash_cta_max == 2048 ||
          c.hash_cta_max == 4096 || c.hash_cta_max == 8192))
        return SPG_ERR_INVALID;
    if (c.table_slots_pct < 125 || c.table_slots_pct > 400 || c.group_promote < 0 || c.group_promote > 2)
        return SPG_ERR_INVALID;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return SPG_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return SPG_ERR_CUDA;
    if (handle && handle->device != cur) return SPG_ERR_INVALID;
    spg_bplan *P = new (std::nothrow) spg_bplan();
    if (!P) return SPG_ERR_INVALID;
    P->h = handle;
    P->nb = nb;
    P->cfg = c;
    // the persistent kernel is built for at most 512 threads (register budget)
    P->threads = c.cta_threads > 512 ? 512 : c.cta_threads;
    cudaGetDevice(&P->device);
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
    P->sms = sms;
    P->smem_optin = (size_t)optin > 4096 ? (size_t)optin - 1024 : (size_t)optin;
    std::vector<int64_t> col0s(nb + 1), segs(nb + 1), aoff(nb + 1), boffe(nb + 1), acol0(nb + 1);
    std::vector<VMat> vA(nb), vB(nb);
    P->prob.resize(nb);
    int64_t ntot = 0, ncp = 0, na = 0, nbe = 0, ntotA = 0;
    for (int i = 0; i < nb; ++i) {
        col0s[i] = ntot;
        segs[i] = ncp;
        aoff[i] = na;
        boffe[i] = nbe;
        acol0[i] = ntotA;
        BProb &q = P->prob[i];
        std::memset(&q, 0, sizeof(q));
        q.Acp = A[i].colptr; q.Arow = A[i].rowidx; q.Aval = A[i].values;
        q.Bcp = B[i].colptr; q.Brow = B[i].rowidx; q.Bval = B[i].values;
        q.Ccp = C_colptr + ncp;
        q.m = A[i].nrows; q.n = B[i].ncols; q.col0 = ntot;
        q.t = prob_t(c, A[i].nrows);
        q.dtype = A[i].dtype;
        vA[i] = VMat{A[i].colptr, A[i].rowidx, A[i].nrows, A[i].ncols, A[i].nnz, ntotA};
        vB[i] = VMat{B[i].colptr, B[i].rowidx, B[i].nrows, B[i].ncols, B[i].nnz, ntot};
        if (A[i].dtype == SPG_F64) P->any_f64 = true;
        P->mmax = std::max<int64_t>(P->mmax, A[i].nrows);
        ntot += B[i].ncols;
        ntotA += A[i].ncols;
        ncp += B[i].ncols + 1;
        na += A[i].nnz;
        nbe += B[i].nnz;
    }
    col0s[nb] = ntot; segs[nb] = ncp; aoff[nb] = na; boffe[nb] = nbe; acol0[nb] = ntotA;
    P->ntot = ntot; P->ncp = ncp; P->na = na; P->nbe = nbe;
    P->Wmax = ceil_div(P->mmax, 32);
    if (c.dense_cache_bytes < 0) { delete P; return SPG_ERR_INVALID; }
    const size_t cache_bytes = batch_cache_bytes(nb, A, B, c);
    P->L = blayout(nb, ntot, ntotA, ncp, cache_bytes);
    if (ws_bytes < P->L.total) { delete P; return SPG_ERR_WORKSPACE; }
    P->ws = static_cast<unsigned char *>(workspace);
    P->nnz.assign(nb, 0);
    if (nb == 0) { *plan_out = P; return SPG_OK; }
    unsigned char *ws = P->ws;
#define CK(expr)                                                  \
    do {                                                          \
        if ((expr) != cudaSuccess) { delete P; return SPG_ERR_CUDA; } \
    } while (0)
    CK(cudaMemsetAsync(P->ctrl(), 0, sizeof(Ctrl), s));
    CK(cudaMemcpyAsync(ws + P->L.prob, P->prob.data(), (size_t)nb * sizeof(BProb), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.col0s, col0s.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.segs, segs.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.aoff, aoff.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.boffe, boffe.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.vA, vA.data(), (size_t)nb * sizeof(VMat), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.vB, vB.data(), (size_t)nb * sizeof(VMat), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ws + P->L.acol0, acol0.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(C_colptr, 0, (size_t)ncp * 8, s));
    const int vg = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(std::max(ntot, ntotA), 256)), 16 * (int64_t)sms);
    if (c.validate) {
        if (ntotA > 0)
            k_bvalidate<<<vg, 256, 0, s>>>(reinterpret_cast<const VMat *>(ws + P->L.vA), nb,
                                           reinterpret_cast<const int64_t *>(ws + P->L.acol0), ntotA, 0, P->ctrl());
        if (ntot > 0)
            k_bvalidate<<<vg, 256, 0, s>>>(reinterpret_cast<const VMat *>(ws + P->L.vB), nb,
                                           reinterpret_cast<const int64_t *>(ws + P->L.col0s), ntot, 1, P->ctrl());
        CK(handle_readback(P->h, &P->host, P->ctrl(), sizeof(Ctrl), nullptr, nullptr, 0, s));
        if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    }
    BTask b = P->task();
    int64_t *op = reinterpret_cast<int64_t *>(ws + P->L.op);
    if (ntot > 0) k_bcount<<<vg, 256, 0, s>>>(b, ntot, op);
    CK(cudaGetLastError());
    CK(handle_readback(P->h, &P->host, P->ctrl(), sizeof(Ctrl), nullptr, nullptr, 0, s));
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    for (int k = 0; k < NBINS; ++k)
        if (P->host.maxop[k] >= (1ULL << 31)) { delete P; return SPG_ERR_UNSUPPORTED; }
    P->off.v[0] = 0;
    for (int k = 0; k < NBINS; ++k) P->off.v[k + 1] = P->off.v[k] + (k == BIN_EMPTY ? 0 : (int64_t)P->host.hist[k]);
    b = P->task();
    if (ntot > 0) k_bscatter<<<(unsigned)ceil_div(ntot, 256), 256, 0, s>>>(b, ntot, op, reinterpret_cast<int32_t *>(ws + P->L.cols));
    CK(cudaGetLastError());
    // places of the dense columns' kept flags (per-warp dense columns only)
    const int64_t ndense = (int64_t)P->host.hist[BIN_DENSE];
    if (cache_bytes > 0 && ndense > 0) {
        int64_t *coff = reinterpret_cast<int64_t *>(ws + P->L.coff);
        k_bcache_words<<<(unsigned)std::min<int64_t>(ceil_div(ndense, 256), 16 * (int64_t)sms), 256, 0, s>>>(
            b, ndense, coff);
        CK(cudaGetLastError());
        CK(launch_inclusive_scan(coff, ndense + 1, reinterpret_cast<int64_t *>(ws + P->L.tiles), s));
        P->cache_words = (int64_t)(cache_bytes / 4);
        P->launches_sym += 4;
    }
    st = launch_phase(*P, 0, s);
    if (st != SPG_OK) { delete P; return st; }
    int64_t *ccp = C_colptr;
    CK(launch_inclusive_scan(ccp, ncp, reinterpret_cast<int64_t *>(ws + P->L.tiles), s));
    k_bbase<<<(unsigned)ceil_div(nb, 256), 256, 0, s>>>(b, ccp, reinterpret_cast<int64_t *>(ws + P->L.base));
    k_bfix<<<(unsigned)std::min<int64_t>(ceil_div(ncp, 256), 16 * (int64_t)sms), 256, 0, s>>>(
        b, ccp, ncp, reinterpret_cast<const int64_t *>(ws + P->L.base), reinterpret_cast<const int64_t *>(ws + P->L.segs),
        reinterpret_cast<int64_t *>(ws + P->L.nnz));
    CK(cudaGetLastError());
    CK(handle_readback(P->h, P->nnz.data(), ws + P->L.nnz, (size_t)nb * 8, &P->host, P->ctrl(), sizeof(Ctrl), s));
#undef CK
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    for (int i = 0; i < nb; ++i) nnzC[i] = P->nnz[i];
    P->launches_sym += (c.validate ? 2 : 0) + 2 + 1 + 3 + 2;
    *plan_out = P;
    return SPG_OK;
}

static spg_status batch_matches(const spg_bplan *P, const spg_csc *A, const spg_csc *B) {
    if (!P) return SPG_ERR_INVALID;
    if (P->nb > 0 && (!A || !B)) return SPG_ERR_INVALID;
    for (int i = 0; i < P->nb; ++i) {
        const BProb &q = P->prob[i];
        if (A[i].nrows != q.m || B[i].ncols != q.n || A[i].dtype != q.dtype || B[i].dtype != q.dtype) return SPG_ERR_INVALID;
        if ((A[i].nnz > 0 && !A[i].values) || (B[i].nnz > 0 && !B[i].values)) return SPG_ERR_INVALID;
    }
    return SPG_OK;
}

spg_status spgemm_batched_numeric(spg_bplan *P, const spg_csc *A, const spg_csc *B, const int64_t *C_colptr,
                                  int32_t *const *C_rowidx, void *const *C_values, int32_t use_graph,
                                  spg_stream stream) {
    spg_status st = batch_matches(P, A, B);
    if (st != SPG_OK) return st;
    if (P->nb == 0) return SPG_OK;
    if (!C_colptr || !C_rowidx || !C_values) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < P->nb; ++i) {
        BProb &q = P->prob[i];
        if (P->nnz[i] > 0 && (!C_rowidx[i] || !C_values[i])) return SPG_ERR_INVALID;
        q.Aval = A[i].values; q.Bval = B[i].values;
        q.Acp = A[i].colptr; q.Arow = A[i].rowidx; q.Bcp = B[i].colptr; q.Brow = B[i].rowidx;
        q.Crow = C_rowidx[i]; q.Cval = C_values[i];
    }
    const bool same = P->gexec && P->graph_prob.size() == P->prob.size() &&
                      std::memcmp(P->graph_prob.data(), P->prob.data(), P->prob.size() * sizeof(BProb)) == 0;
    if (!(use_graph && same)) {
        if (cudaMemcpyAsync(P->ws + P->L.prob, P->prob.data(), P->prob.size() * sizeof(BProb),
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SPG_ERR_CUDA;
    }
    // the legacy default stream cannot be captured: launch directly there
    if (!use_graph || s == nullptr || s == cudaStreamLegacy) return launch_phase(*P, 1, s);
    if (!same) {
        // (re)capture: counter reset + the persistent launch
        if (P->gexec) { cudaGraphExecDestroy(P->gexec); P->gexec = nullptr; }
        if (P->graph) { cudaGraphDestroy(P->graph); P->graph = nullptr; }
        PhaseLaunch L;
        st = prepare_phase(*P, 1, L);
        if (st != SPG_OK) return st;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SPG_ERR_CUDA;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPG_ERR_CUDA;
        st = enqueue_phase(*P, 1, L, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (st != SPG_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st != SPG_OK ? st : SPG_ERR_CUDA;
        }
        if (cudaGraphInstantiate(&P->gexec, g, 0) != cudaSuccess) {
            cudaGraphDestroy(g);
            return SPG_ERR_CUDA;
        }
        P->graph = g;
        P->graph_prob = P->prob;
    }
    return cudaGraphLaunch(P->gexec, s) == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

spg_status spgemm_batched_backward(spg_bplan *P, const spg_csc *A, const spg_csc *B, const int64_t *C_colptr,
                                   const int32_t *const *C_rowidx, const void *const *dC_values,
                                   void *const *dA_values, void *const *dB_values, spg_stream stream) {
    spg_status st = batch_matches(P, A, B);
    if (st != SPG_OK) return st;
    if (P->nb == 0) return SPG_OK;
    if (!C_colptr || !C_rowidx || !dC_values) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < P->nb; ++i) {
        BProb &q = P->prob[i];
        if (P->nnz[i] > 0 && (!C_rowidx[i] || !dC_values[i])) return SPG_ERR_INVALID;
        q.Aval = A[i].values; q.Bval = B[i].values;
        q.Crow = const_cast<int32_t *>(C_rowidx[i]);
        q.dC = dC_values[i];
        q.dA = dA_values ? dA_values[i] : nullptr;
        q.dB = dB_values ? dB_values[i] : nullptr;
    }
    if (cudaMemcpyAsync(P->ws + P->L.prob, P->prob.data(), P->prob.size() * sizeof(BProb), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return SPG_ERR_CUDA;
    P->graph_prob.clear();  // the device table changed
    BTask b = P->task();
    if (P->na + P->nbe > 0)
        k_bzero<<<(unsigned)std::min<int64_t>(ceil_div(P->na + P->nbe, 256), 16 * (int64_t)P->sms), 256, 0, s>>>(
            b, reinterpret_cast<const int64_t *>(P->ws + P->L.aoff), reinterpret_cast<const int64_t *>(P->ws + P->L.boffe),
            P->na, P->nbe);
    if (cudaGetLastError() != cudaSuccess) return SPG_ERR_CUDA;
    return launch_phase(*P, 2, s);
}

spg_status spg_bplan_check(spg_bplan *P, spg_stream stream) {
    if (!P) return SPG_ERR_INVALID;
    if (P->nb == 0) return SPG_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t err = 0;
    if (handle_readback(P->h, &err, &P->ctrl()->err, sizeof(err), nullptr, nullptr, 0, s) != cudaSuccess) return SPG_ERR_CUDA;
    return (spg_status)err;
}

spg_status spg_bplan_info(const spg_bplan *P, int64_t *bin_counts, int64_t *products, int64_t *launches) {
    if (!P) return SPG_ERR_INVALID;
    if (bin_counts)
        for (int k = 0; k < NBINS; ++k) bin_counts[k] = (int64_t)P->host.hist[k];
    if (products) *products = (int64_t)P->host.products;
    if (launches) {
        launches[0] = P->launches_sym;
        launches[1] = 1;
        launches[2] = 2;
    }
    return SPG_OK;
}

spg_status spg_bplan_destroy(spg_bplan *P) {
    delete P;
    return SPG_OK;
}

}  // extern "C"
