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
#include "columns.cuh"

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

template <int G, int R, typename VT>
__global__ void __launch_bounds__(kGroupThreads, 1) k_bwd_group(BinTask t, Operands o, const int64_t *Ccp,
                                                             const int32_t *Crow, const VT *dC, VT *dA, VT *dB) {
    constexpr int H = 2 * G * R;
    constexpr int NG = kGroupThreads / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const int grp = threadIdx.x / G;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * H;
    VT *vals = reinterpret_cast<VT *>(smem + (size_t)NG * H * 4) + grp * H;
    const int64_t gidx = (int64_t)blockIdx.x * NG + grp;
    if (gidx >= t.count) return;
    const int32_t j = t.cols[gidx];
    if (!bwd_group_column<G, VT>(group_mask(G), typed<VT>(o), j, Ccp[j], Ccp[j + 1], Crow, dC, keys, vals,
                                 (uint32_t)H, dA, dB))
        set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
}

template <typename VT, bool TSM>
__global__ void __launch_bounds__(1024, 1) k_bwd_cta(BinTask t, Operands o, const int64_t *Ccp, const int32_t *Crow,
                                                  const VT *dC, VT *dA, VT *dB, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    int32_t *pidx = reinterpret_cast<int32_t *>(smem + o_walk);
    const size_t o_tab = o_walk + al16((size_t)blockDim.x * 4);
    unsigned char *tb = TSM ? smem + o_tab : t.scratch + (size_t)blockIdx.x * t.scratch_stride;
    int32_t *keys = reinterpret_cast<int32_t *>(tb);
    VT *vals = reinterpret_cast<VT *>(tb + al16((size_t)cap * 4));
    const TOps<VT> ops = typed<VT>(o);
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j], nn = Ccp[j + 1] - c0;
        int64_t want = num_slots(nn, t.slots_pct);
        if (want > cap) want = cap;
        if (!bwd_cta_column<VT>(ops, j, c0, nn, Crow, dC, keys, vals, (uint32_t)want, w, pidx, dA, dB))
            set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
    }
}

template <typename VT, bool BSM>
__global__ void __launch_bounds__(1024, 1) k_bwd_dense(BinTask t, Operands o, const int64_t *Ccp, const int32_t *Crow,
                                                    const VT *dC, VT *dA, VT *dB, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ int64_t s_warp[32];
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    int32_t *pidx = reinterpret_cast<int32_t *>(smem + o_walk);
    const size_t o_bm = o_walk + al16((size_t)blockDim.x * 4);
    uint2 *bm = BSM ? reinterpret_cast<uint2 *>(smem + o_bm)
                    : reinterpret_cast<uint2 *>(t.scratch + (size_t)blockIdx.x * t.scratch_stride);
    VT *s_dc = reinterpret_cast<VT *>(smem + o_bm + (BSM ? (size_t)t.W * 8 : 0));
    for (int64_t i = threadIdx.x; i < t.W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
    const TOps<VT> ops = typed<VT>(o);
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j], nn = Ccp[j + 1] - c0;
        bwd_dense_column<VT>(ops, j, c0, nn, Crow, dC, bm, t.W, s_dc, cap, w, pidx, s_warp, dA, dB);
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
                               int64_t maxnnz, int slots_pct, int64_t scratch_ctas) {
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
    const size_t fixed = walk_smem_bytes<VT>(g.threads) + al16((size_t)g.threads * 4);
    if (bin >= BIN_CTA0 && bin <= BIN_GLOBAL) {
        g.slots = num_slots(maxnnz, slots_pct);
        const size_t tab = al16((size_t)g.slots * 4) + al16((size_t)g.slots * sizeof(VT));
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
                      int dtype, int slots_pct, int64_t scratch_ctas) {
    return dtype == SPG_F64
               ? backward_geometry_t<double>(bin, count, m, threads, sms, smem_optin, maxnnz, slots_pct, scratch_ctas)
               : backward_geometry_t<float>(bin, count, m, threads, sms, smem_optin, maxnnz, slots_pct, scratch_ctas);
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
