// Backward of C = A x B with respect to the stored values of A and B:
//   dA_ik = sum_{j: B_kj stored} dC_ij B_kj  on pattern(A),
//   dB_kj = sum_i A_ik dC_ij                 on pattern(B).
// The paper has no backward; these are the derivatives of C_ij = sum_k A_ik
// B_kj, computed as masked products over exactly the products the forward
// walks, with the forward's bins: per column j, dC[:, j] is loaded into the
// bin's lookup structure (a group hash table, a CTA hash table, or the dense
// SPA's flag bitmap whose prefix counts give each row its position in the
// sorted column), and every product A_ik B_kj looks up g = dC_ij.  dA_ik
// receives B_kj g by an atomic add at A's position q (many columns j reach
// the same A entry); dB_kj receives A_ik g summed over its A column: the
// products of one B entry are consecutive in the walk, so a segmented warp
// reduction leaves one atomic add per entry and window.
#include "kernels.cuh"

namespace spg {

constexpr int kGroupThreads = 256;

template <typename K>
static void allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename K>
static int occupancy(K kernel, int threads, size_t smem) {
    int n = 0;
    allow_smem(kernel, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) n = 1;
    return n < 1 ? 1 : n;
}

__host__ __device__ inline size_t al16b(size_t v) { return (v + 15) & ~size_t(15); }

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

// ------------------------------------------------------- group walk (bwd)
// Lanes of a group of G cover the column's products like group_products;
// every lane of the group calls step(row, a, b, qa, p) once per round from a
// single call site (p = -1 when the lane is idle).
template <int G, typename VT, typename S>
__device__ __forceinline__ void group_walk_bwd(unsigned mask, const int64_t *__restrict__ Acp,
                                               const int32_t *__restrict__ Arow, const VT *__restrict__ Aval,
                                               const int32_t *__restrict__ Brow, const VT *__restrict__ Bval,
                                               int64_t p0, int64_t p1, S &&step) {
    const int gl = threadIdx.x & (G - 1);
    for (int64_t base = p0; base < p1; base += G) {
        const int64_t p = base + gl;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = Brow[p];
            a0 = Acp[k];
            z = static_cast<int>(Acp[k + 1] - a0);
            bv = Bval[p];
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
            const int32_t row = on ? Arow[qa] : 0;
            const VT av = on ? Aval[qa] : VT(0);
            step(row, av, bvs, qa, on ? base + s : (int64_t)-1);
        }
    }
}

template <int G, int R, typename VT>
__global__ void __launch_bounds__(kGroupThreads) k_bwd_group(BinTask t, Operands o, const int64_t *Ccp,
                                                             const int32_t *Crow, const VT *dC, VT *dA, VT *dB) {
    constexpr int H = 2 * G * R;
    constexpr int NG = kGroupThreads / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const int grp = threadIdx.x / G;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * H;
    VT *vals = reinterpret_cast<VT *>(smem + (size_t)NG * H * 4) + grp * H;
    const unsigned mask = group_mask(G);
    const int gl = threadIdx.x & (G - 1);
    const int64_t gidx = (int64_t)blockIdx.x * NG + grp;
    if (gidx >= t.count) return;
    const int32_t j = t.cols[gidx];
    for (int i = gl; i < H; i += G) keys[i] = kEmptyKey;
    __syncwarp(mask);
    // dC[:, j] into the group's table (rows are distinct)
    const int64_t c0 = Ccp[j], c1 = Ccp[j + 1];
    for (int64_t e = c0 + gl; e < c1; e += G) {
        bool fresh;
        const int32_t slot = hash_insert(keys, (uint32_t)H, Crow[e], fresh);
        if (slot >= 0) vals[slot] = dC[e];
        else set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
    }
    __syncwarp(mask);
    auto lookup = [&](int32_t row) -> VT {
        const int32_t slot = hash_find(keys, (uint32_t)H, row);
        return slot >= 0 ? vals[slot] : VT(0);
    };
    group_walk_bwd<G, VT>(mask, o.Acp, o.Arow, static_cast<const VT *>(o.Aval), o.Brow,
                          static_cast<const VT *>(o.Bval), o.Bcp[j], o.Bcp[j + 1],
                          [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
                              bwd_product<G, VT>(mask, row, a, b, qa, p, dA, dB, lookup);
                          });
}

// ------------------------------------------------------ CTA walk (bwd)
// Same chunking and window split as cta_walk (one list of non-empty entries);
// every lane of a warp calls step(...) once per window from a single call
// site (p = -1 when idle), so the segmented reduction is warp-wide.
// Contains barriers: every thread of the CTA calls it.
template <typename VT, typename S>
__device__ __forceinline__ void cta_walk_bwd(const int64_t *__restrict__ Acp, const int32_t *__restrict__ Arow,
                                             const VT *__restrict__ Aval, const int32_t *__restrict__ Brow,
                                             const VT *__restrict__ Bval, int64_t p0, int64_t p1,
                                             const WalkSmem<VT> &w, int32_t *pidx, S &&step) {
    const int T = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    for (int64_t base = p0; base < p1; base += T) {
        const int64_t p = base + threadIdx.x;
        int z = 0;
        int64_t a0 = 0;
        VT bv = VT(0);
        if (p < p1) {
            const int32_t k = Brow[p];
            a0 = Acp[k];
            z = (int)(Acp[k + 1] - a0);
            bv = Bval[p];
        }
        // one list: every non-empty entry, in order
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
                const int32_t row = on ? Arow[qa] : 0;
                const VT av = on ? Aval[qa] : VT(0);
                step(row, av, on ? w.bv[own] : VT(0), qa, on ? base + pidx[own] : (int64_t)-1);
                s += __popc(bits) + (__ballot_sync(0xffffffffu, pos == 32) ? 1 : 0);
            }
        }
        __syncthreads();
    }
}

template <typename VT, bool TSM>
__global__ void __launch_bounds__(1024) k_bwd_cta(BinTask t, Operands o, const int64_t *Ccp, const int32_t *Crow,
                                                  const VT *dC, VT *dA, VT *dB, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    int32_t *pidx = reinterpret_cast<int32_t *>(smem + o_walk);
    const size_t o_tab = o_walk + al16b((size_t)blockDim.x * 4);
    unsigned char *tb = TSM ? smem + o_tab : t.scratch + (size_t)blockIdx.x * t.scratch_stride;
    int32_t *keys = reinterpret_cast<int32_t *>(tb);
    VT *vals = reinterpret_cast<VT *>(tb + al16b((size_t)cap * 4));
    const VT *Aval = static_cast<const VT *>(o.Aval);
    const VT *Bval = static_cast<const VT *>(o.Bval);
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j], nn = Ccp[j + 1] - c0;
        int64_t want = num_slots(nn);
        if (want > cap) want = cap;
        const uint32_t H = (uint32_t)want;
        for (uint32_t s = threadIdx.x; s < H; s += blockDim.x) keys[s] = kEmptyKey;
        __syncthreads();
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
            bool fresh;
            const int32_t slot = hash_insert(keys, H, Crow[c0 + e], fresh);
            if (slot >= 0) vals[slot] = dC[c0 + e];
            else set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
        }
        __syncthreads();
        auto lookup = [&](int32_t row) -> VT {
            const int32_t slot = hash_find(keys, H, row);
            return slot >= 0 ? vals[slot] : VT(0);
        };
        cta_walk_bwd<VT>(o.Acp, o.Arow, Aval, o.Brow, Bval, o.Bcp[j], o.Bcp[j + 1], w, pidx,
                         [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
                             bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
                         });
    }
}

template <typename VT, bool BSM>
__global__ void __launch_bounds__(1024) k_bwd_dense(BinTask t, Operands o, const int64_t *Ccp, const int32_t *Crow,
                                                    const VT *dC, VT *dA, VT *dB, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ int64_t s_warp[32];
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    int32_t *pidx = reinterpret_cast<int32_t *>(smem + o_walk);
    const size_t o_bm = o_walk + al16b((size_t)blockDim.x * 4);
    uint2 *bm = BSM ? reinterpret_cast<uint2 *>(smem + o_bm)
                    : reinterpret_cast<uint2 *>(t.scratch + (size_t)blockIdx.x * t.scratch_stride);
    VT *s_dc = reinterpret_cast<VT *>(smem + o_bm + (BSM ? (size_t)t.W * 8 : 0));
    for (int64_t i = threadIdx.x; i < t.W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
    const VT *Aval = static_cast<const VT *>(o.Aval);
    const VT *Bval = static_cast<const VT *>(o.Bval);
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j], nn = Ccp[j + 1] - c0;
        // flags of C's column; rank(row) is then the row's position in it
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
            const int32_t r = Crow[c0 + e];
            atomicOr(&bm[r >> 5].x, 1u << (r & 31));
        }
        __syncthreads();
        cta_bitmap_prefix(bm, t.W, s_warp);
        const bool in_smem = nn <= cap;
        if (in_smem)
            for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) s_dc[e] = dC[c0 + e];
        __syncthreads();
        if (in_smem) {
            auto lookup = [&](int32_t row) -> VT { return s_dc[bitmap_rank(bm, row)]; };
            cta_walk_bwd<VT>(o.Acp, o.Arow, Aval, o.Brow, Bval, o.Bcp[j], o.Bcp[j + 1], w, pidx,
                             [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
                                 bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
                             });
        } else {
            const VT *gdc = dC + c0;
            auto lookup = [&](int32_t row) -> VT { return gdc[bitmap_rank(bm, row)]; };
            cta_walk_bwd<VT>(o.Acp, o.Arow, Aval, o.Brow, Bval, o.Bcp[j], o.Bcp[j + 1], w, pidx,
                             [&](int32_t row, VT a, VT b, int64_t qa, int64_t p) {
                                 bwd_product<32, VT>(0xffffffffu, row, a, b, qa, p, dA, dB, lookup);
                             });
        }
        for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) bm[Crow[c0 + e] >> 5].x = 0u;
        __syncthreads();
    }
}

// ------------------------------------------------------------- launches
constexpr size_t kBitmapSmemMax = 96 * 1024;

static inline int bwd_cta_threads(int bin, int cfg_threads) {
    if (bin == BIN_CTA0 || bin == BIN_CTA0 + 1) return 256;
    if (bin == BIN_CTA0 + 2 || bin == BIN_CTA0 + 3) return 512;
    return cfg_threads;
}

template <typename VT>
static Geo backward_geometry_t(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                               int64_t maxnnz, int64_t scratch_ctas) {
    Geo g;
    const int64_t W = ceil_div(m, 32);
    if (bin >= BIN_WARP0 && bin < BIN_CTA0) {
        const int b = bin - BIN_WARP0;
        const int G = warp_bin_G(b), R = warp_bin_R(b);
        g.threads = kGroupThreads;
        g.smem = (size_t)(kGroupThreads / G) * 2 * G * R * (4 + sizeof(VT));
        g.grid = (int)ceil_div(count, kGroupThreads / G);
        return g;
    }
    g.threads = bwd_cta_threads(bin, threads);
    const size_t fixed = walk_smem_bytes<VT>(g.threads) + al16b((size_t)g.threads * 4);
    if (bin >= BIN_CTA0 && bin <= BIN_GLOBAL) {
        g.slots = num_slots(maxnnz);
        const size_t tab = al16b((size_t)g.slots * 4) + al16b((size_t)g.slots * sizeof(VT));
        const bool table_global = bin == BIN_GLOBAL || fixed + tab > smem_optin;
        g.cap = table_global ? 1 : 0;
        g.smem = fixed + (table_global ? 0 : tab);
        int occ = occupancy(k_bwd_cta<VT, true>, g.threads, g.smem);
        int64_t grid = std::min<int64_t>(count, (int64_t)occ * sms);
        if (table_global) grid = std::min<int64_t>(grid, scratch_ctas);
        g.grid = (int)std::max<int64_t>(1, grid);
        return g;
    }
    const size_t bmb = (size_t)W * 8;
    g.bm_global = bmb > kBitmapSmemMax || fixed + bmb > smem_optin;
    const size_t base = fixed + (g.bm_global ? 0 : bmb);
    const size_t room = smem_optin > base ? smem_optin - base : 0;
    int64_t cap = (int64_t)(room / sizeof(VT));
    if (cap > maxnnz) cap = maxnnz;
    g.cap = cap;
    g.smem = base + (size_t)cap * sizeof(VT);
    int occ = occupancy(k_bwd_dense<VT, true>, g.threads, g.smem);
    int64_t grid = std::min<int64_t>(count, (int64_t)occ * sms);
    if (g.bm_global) grid = std::min<int64_t>(grid, scratch_ctas);
    g.grid = (int)std::max<int64_t>(1, grid);
    return g;
}

Geo backward_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin, int64_t maxnnz,
                      int dtype, int shrink, int64_t scratch_ctas) {
    (void)shrink;
    return dtype == SPG_F64 ? backward_geometry_t<double>(bin, count, m, threads, sms, smem_optin, maxnnz, scratch_ctas)
                            : backward_geometry_t<float>(bin, count, m, threads, sms, smem_optin, maxnnz, scratch_ctas);
}

template <typename VT>
static cudaError_t launch_backward_t(const BinTask &t, const Operands &o, const int64_t *Ccp, const int32_t *Crow,
                                     const VT *dC, VT *dA, VT *dB, const Geo &g, cudaStream_t s) {
    if (t.count <= 0) return cudaSuccess;
    if (t.bin >= BIN_WARP0 && t.bin < BIN_CTA0) {
        switch (t.bin - BIN_WARP0) {
#define BWD_CASE(b)                                                                        \
    case b: {                                                                              \
        auto k = k_bwd_group<warp_bin_G(b), warp_bin_R(b), VT>;                            \
        allow_smem(k, g.smem);                                                             \
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, dC, dA, dB);                  \
        break;                                                                             \
    }
            BWD_CASE(0) BWD_CASE(1) BWD_CASE(2) BWD_CASE(3) BWD_CASE(4) BWD_CASE(5)
#undef BWD_CASE
        }
    } else if (t.bin <= BIN_GLOBAL) {
        auto k = g.cap ? k_bwd_cta<VT, false> : k_bwd_cta<VT, true>;
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, dC, dA, dB, g.slots);
    } else {
        auto k = g.bm_global ? k_bwd_dense<VT, false> : k_bwd_dense<VT, true>;
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, dC, dA, dB, g.cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_backward_bin(const BinTask &t, const Operands &o, const int64_t *Ccp, const int32_t *Crow,
                                const void *dC, void *dA, void *dB, int dtype, const Geo &g, cudaStream_t s) {
    if (dtype == SPG_F64)
        return launch_backward_t<double>(t, o, Ccp, Crow, static_cast<const double *>(dC), static_cast<double *>(dA),
                                         static_cast<double *>(dB), g, s);
    return launch_backward_t<float>(t, o, Ccp, Crow, static_cast<const float *>(dC), static_cast<float *>(dA),
                                    static_cast<float *>(dB), g, s);
}

}  // namespace spg
