// Numeric phase: values and ascending rows of every column of C = A x B.
//
// Per bin (Section 3.3's H-HASH(t)):
//   * warp-group hash bins (Op_j <= 256): a group of G lanes per column
//     accumulates into an open-addressing table (Section 3.2) in shared
//     memory, compacts it and sorts it with a register bitonic network;
//   * CTA hash bins (Op_j <= hash_cta_max) and the global hash bin: one CTA
//     per column, table of ~1.5 nnz(C_j) slots (shared or global memory);
//     the touched rows are then marked in a bitmap whose prefix counts give
//     every row its sorted position, and the column is written in row order
//     with one table lookup per entry;
//   * dense bin (Op_j >= t): the SPA of Algorithm 1 -- flags as a bitmap
//     (kept from the symbolic phase and staged one column ahead by a bulk
//     copy, or set again by a first walk), prefix counts turn each row into
//     its position in the sorted column, a walk adds every product at that
//     position (double sums in place in C, float sums in shared memory), and
//     a pass over the flags writes the rows in order.
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

// ------------------------------------------------- warp-group hash bins
template <int G, int R, typename VT>
__global__ void __launch_bounds__(kGroupThreads, 4) k_num_group(BinTask t, Operands o, const int64_t *Ccp,
                                                             int32_t *Crow, VT *Cval) {
    constexpr int H = 2 * G * R;
    constexpr int NG = kGroupThreads / G;
    extern __shared__ __align__(16) unsigned char smem[];
    const int grp = threadIdx.x / G;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + grp * H;
    VT *vals = reinterpret_cast<VT *>(smem + (size_t)NG * H * 4) + grp * H;
    const int64_t gidx = (int64_t)blockIdx.x * NG + grp;
    if (gidx >= t.count) return;
    uint32_t Hj = (uint32_t)H >> t.shrink;
    if (Hj < 1) Hj = 1;
    const int32_t j = t.cols[gidx];
    const int64_t c0 = Ccp[j];
    bool ovf = false;
    const bool ok = num_group_column<G, R, VT>(group_mask(G), typed<VT>(o), j, c0, Ccp[j + 1] - c0, keys, vals,
                                               Hj, Crow, Cval, ovf, t.cnt_out);
    if (ovf) set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
    if (!ok) set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
}

// ------------------------------------------------------- CTA hash bins
// Placement of the table (TSM) and of the row bitmap (BSM) is a template
// parameter: pointers derived straight from the shared-memory array let the
// compiler use shared-space loads and atomics instead of generic ones.
template <typename VT, bool TSM, bool BSM>
__global__ void __launch_bounds__(1024, 1) k_num_cta(BinTask t, Operands o, const int64_t *Ccp, int32_t *Crow,
                                                  VT *Cval, int64_t cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ unsigned s_occ;
    __shared__ int64_t s_warp[32];
    const int64_t W1 = (t.W + 31) / 32;
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    const size_t tab = cta_table_bytes<VT>(cap);
    unsigned char *gp = t.scratch + (size_t)blockIdx.x * t.scratch_stride;
    // the table and the word list scale with the table size: both live in
    // shared memory, or both in the CTA's global scratch
    unsigned char *tb = TSM ? smem + o_walk : gp;
    int32_t *keys = reinterpret_cast<int32_t *>(tb);
    VT *vals = reinterpret_cast<VT *>(tb + al16((size_t)cap * 4));
    int32_t *wlist = reinterpret_cast<int32_t *>(tb + al16((size_t)cap * 4) + al16((size_t)cap * sizeof(VT)));
    const size_t o_l0 = o_walk + (TSM ? tab : 0);
    uint32_t *L0 = BSM ? reinterpret_cast<uint32_t *>(smem + o_l0) : reinterpret_cast<uint32_t *>(gp + (TSM ? 0 : tab));
    uint32_t *L1 = reinterpret_cast<uint32_t *>(smem + o_l0 + (BSM ? al16((size_t)t.W * 4) : 0));
    for (int64_t i = threadIdx.x; i < t.W; i += blockDim.x) L0[i] = 0u;
    for (int64_t i = threadIdx.x; i < W1; i += blockDim.x) L1[i] = 0u;
    const TOps<VT> ops = typed<VT>(o);
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j];
        const int64_t nn = Ccp[j + 1] - c0;
        int64_t want = num_slots(nn, t.slots_pct);
        if (want > cap) want = cap;
        uint32_t H = (uint32_t)(want >> t.shrink);
        if (H < 1) H = 1;
        bool ovf = false;
        const bool ok = num_cta_column<VT>(ops, j, c0, nn, keys, vals, wlist, H, L0, L1, t.W, w, &s_occ, s_warp,
                                           Crow, Cval, ovf, t.cnt_out);
        if (ovf) set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
        if (!ok && threadIdx.x == 0) set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
    }
}

// ------------------------------------------------------------ dense bin
// With `prefetch`, the flags the symbolic phase kept for the next column are
// brought into shared memory by a bulk copy issued as soon as the current
// column's prefix pass has consumed the staging buffer, so the copy overlaps
// the current column's walk and extraction.
template <typename VT, bool BSM>
__global__ void __launch_bounds__(1024, 1) k_num_dense(BinTask t, Operands o, const int64_t *Ccp, int32_t *Crow,
                                                    VT *Cval, int64_t cap, int prefetch) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ int64_t s_warp[32];
    __shared__ unsigned s_chunk;
    __shared__ __align__(8) uint64_t s_bar;
    const WalkSmem<VT> w = carve_walk<VT>(smem);
    const size_t o_walk = walk_smem_bytes<VT>(blockDim.x);
    uint2 *bm = BSM ? reinterpret_cast<uint2 *>(smem + o_walk)
                    : reinterpret_cast<uint2 *>(t.scratch + (size_t)blockIdx.x * t.scratch_stride);
    VT *s_acc = reinterpret_cast<VT *>(smem + o_walk + (BSM ? (size_t)t.W * 8 : 0));
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + o_walk + (BSM ? (size_t)t.W * 8 : 0) +
                                                   al16((size_t)cap * sizeof(VT)));
    const int64_t n_cached = t.cache_cols < t.count ? t.cache_cols : t.count;
    const unsigned stage_bytes = (unsigned)(t.W * 4);
    for (int64_t i = threadIdx.x; i < t.W; i += blockDim.x) bm[i] = make_uint2(0u, 0u);
    if (threadIdx.x == 0) {
        if (prefetch) mbar_init(&s_bar, 1);
        s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        if (prefetch && s_col < n_cached) bulk_load(stage, t.flag_cache + (size_t)s_col * t.W, stage_bytes, &s_bar);
    }
    __syncthreads();
    const TOps<VT> ops = typed<VT>(o);
    unsigned phase = 0;
    bool timed_out = false;
    for (;;) {
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        const int64_t c0 = Ccp[j];
        const int64_t nn = Ccp[j + 1] - c0;
        const uint32_t *keep = ci < t.cache_cols ? t.flag_cache + (size_t)ci * t.W : nullptr;
        if (prefetch && keep) {
            const bool arrived = mbar_wait(&s_bar, phase, t.wait_cycles);
            if (__syncthreads_or(!arrived)) {
                if (threadIdx.x == 0) set_error(t.ctrl, SPG_ERR_TIMEOUT, t.bin, j);
                timed_out = true;
                break;
            }
            phase ^= 1u;
            keep = stage;
        }
        // after the prefix pass: take the next column and start its copy
        // (no thread reads s_col again before the column's last barrier)
        auto next = [&]() {
            if (threadIdx.x == 0) {
                s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
                if (prefetch && s_col < n_cached)
                    bulk_load(stage, t.flag_cache + (size_t)s_col * t.W, stage_bytes, &s_bar);
            }
        };
        const bool ok = num_dense_column<VT>(ops, j, c0, nn, bm, t.W, keep, s_acc, cap, w, s_warp, &s_chunk, Crow,
                                             Cval, next, t.cnt_out);
        if (!ok && threadIdx.x == 0) set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
    }
    // a copy is in flight only after a time-out: wait for it (bounded, at
    // full length whatever the first wait's limit) before the CTA's shared
    // memory goes away
    if (timed_out) mbar_wait(&s_bar, phase, kBulkWaitCycles);
}

// ------------------------------------------------------------- launches
constexpr size_t kBitmapSmemMax = 96 * 1024;

// Threads per CTA of the CTA-level bins: small columns share an SM among
// several CTAs, the largest get a whole SM.
inline int cta_bin_threads(int bin, int cfg_threads) {
    if (bin == BIN_CTA0 || bin == BIN_CTA0 + 1) return 256;
    if (bin == BIN_CTA0 + 2 || bin == BIN_CTA0 + 3) return 512;
    return cfg_threads;
}

template <typename VT>
static Geo numeric_geometry_t(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                              int64_t maxnnz, int slots_pct, int64_t scratch_ctas) {
    Geo g;
    const int64_t W = ceil_div(m, 32);
    const int64_t W1 = ceil_div(W, 32);
    if (bin >= BIN_WARP0 && bin < BIN_CTA0) {
        const int b = bin - BIN_WARP0;
        const int G = warp_bin_G(b), R = warp_bin_R(b);
        g.threads = kGroupThreads;
        g.smem = (size_t)(kGroupThreads / G) * 2 * G * R * (4 + sizeof(VT));
        g.grid = (int)ceil_div(count, kGroupThreads / G);
        return g;
    }
    g.threads = cta_bin_threads(bin, threads);
    if (bin >= BIN_CTA0 && bin <= BIN_GLOBAL) {
        g.slots = num_slots(maxnnz, slots_pct);
        // table (keys, values) and word list; L1 always in shared memory
        const size_t tab = al16((size_t)g.slots * 4) + al16((size_t)g.slots * sizeof(VT)) +
                           al16((size_t)g.slots * 4);
        const size_t fixed = al16((size_t)W1 * 4) + walk_smem_bytes<VT>(g.threads);
        const size_t l0 = al16((size_t)W * 4);
        const bool table_global = bin == BIN_GLOBAL || fixed + tab > smem_optin;
        g.bm_global = l0 > kBitmapSmemMax || fixed + (table_global ? 0 : tab) + l0 > smem_optin;
        g.cap = table_global ? 1 : 0;  // reused as "table in global" flag
        g.smem = fixed + (table_global ? 0 : tab) + (g.bm_global ? 0 : l0);
        int occ = occupancy(k_num_cta<VT, true, true>, g.threads, g.smem);
        int64_t grid = std::min<int64_t>(count, (int64_t)occ * sms);
        if (table_global || g.bm_global) grid = std::min<int64_t>(grid, scratch_ctas);
        g.grid = (int)std::max<int64_t>(1, grid);
        return g;
    }
    // dense
    const size_t bmb = (size_t)W * 8;
    // shape of one CTA with t threads: its cap (values kept in shared
    // memory), dynamic shared memory, staging of the next column's flags,
    // and CTAs per SM
    auto shape = [&](int tt, Geo &o) {
        o = g;
        o.threads = tt;
        const size_t walk = walk_smem_bytes<VT>(tt);
        o.bm_global = bmb > kBitmapSmemMax || walk + bmb > smem_optin;
        const size_t base = walk + (o.bm_global ? 0 : bmb);
        const size_t room = smem_optin > base ? (smem_optin - base) & ~size_t(15) : 0;
        int64_t cap = (int64_t)(room / sizeof(VT));
        if (cap > maxnnz) cap = maxnnz;
        // Double sums go to C in place: on GB300 a walk that adds with
        // RED.F64 into L2-resident C takes about 1.3x the products per
        // SM-second of one that adds with shared-memory f64 atomics (also
        // when the first positions of a column stay in shared memory), and
        // the extraction then copies no values.  Float sums stay in shared
        // memory (native f32 atomics).
        if (sizeof(VT) == 8) cap = 0;
        o.cap = cap;
        o.smem = base + al16((size_t)cap * sizeof(VT));
        int occ = occupancy(k_num_dense<VT, true>, tt, o.smem);
        // staging buffer for the next column's kept flags: bulk copies need
        // 16-byte aligned columns (W a multiple of 4); only if it costs no CTA
        o.prefetch = false;
        if (!o.bm_global && W % 4 == 0) {
            const size_t with = o.smem + (size_t)W * 4;
            if (with <= smem_optin && occupancy(k_num_dense<VT, true>, tt, with) >= occ) {
                o.smem = with;
                o.prefetch = true;
            }
        }
        return occ;
    };
    // With the double sums in C a CTA holds only the walk scratch and the
    // flags: where four 256-thread CTAs fit an SM they beat two of 512 (more
    // CTAs overlap one another's per-column barriers; measured), else two of
    // 512, else the configured size.
    Geo g256, g512;
    int occ = 0;
    if (sizeof(VT) == 8 && threads >= 256) {
        const int o256 = shape(256, g256);
        const int o512 = threads >= 512 ? shape(512, g512) : 0;
        if (o256 * 256 >= o512 * 512) { g = g256; occ = o256; }
        else { g = g512; occ = o512; }
    } else {
        Geo gc;
        occ = shape(threads, gc);
        g = gc;
    }
    int64_t grid = std::min<int64_t>(count, (int64_t)occ * sms);
    if (g.bm_global) grid = std::min<int64_t>(grid, scratch_ctas);
    g.grid = (int)std::max<int64_t>(1, grid);
    return g;
}

Geo numeric_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                     int64_t maxnnz, int dtype, int slots_pct, int64_t scratch_ctas) {
    return dtype == SPG_F64
               ? numeric_geometry_t<double>(bin, count, m, threads, sms, smem_optin, maxnnz, slots_pct, scratch_ctas)
               : numeric_geometry_t<float>(bin, count, m, threads, sms, smem_optin, maxnnz, slots_pct, scratch_ctas);
}

template <typename VT>
static cudaError_t launch_numeric_t(const BinTask &t, const Operands &o, const int64_t *Ccp, int32_t *Crow,
                                    VT *Cval, const Geo &g, cudaStream_t s) {
    if (t.count <= 0) return cudaSuccess;
    if (t.bin >= BIN_WARP0 && t.bin < BIN_CTA0) {
        switch (t.bin - BIN_WARP0) {
#define NUM_CASE(b)                                                                        \
    case b: {                                                                              \
        auto k = k_num_group<warp_bin_G(b), warp_bin_R(b), VT>;                            \
        allow_smem(k, g.smem);                                                             \
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, Cval);                        \
        break;                                                                             \
    }
            NUM_CASE(0) NUM_CASE(1) NUM_CASE(2) NUM_CASE(3) NUM_CASE(4) NUM_CASE(5)
#undef NUM_CASE
        }
    } else if (t.bin <= BIN_GLOBAL) {
        const bool tsm = g.cap == 0, bsm = !g.bm_global;
        auto k = tsm ? (bsm ? k_num_cta<VT, true, true> : k_num_cta<VT, true, false>)
                     : (bsm ? k_num_cta<VT, false, true> : k_num_cta<VT, false, false>);
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, Cval, g.slots);
    } else {
        auto k = g.bm_global ? k_num_dense<VT, false> : k_num_dense<VT, true>;
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, Crow, Cval, g.cap, g.prefetch ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_numeric_bin(const BinTask &t, const Operands &o, const int64_t *Ccp, int32_t *Crow,
                               void *Cval, int dtype, const Geo &g, cudaStream_t s) {
    return dtype == SPG_F64 ? launch_numeric_t<double>(t, o, Ccp, Crow, static_cast<double *>(Cval), g, s)
                            : launch_numeric_t<float>(t, o, Ccp, Crow, static_cast<float *>(Cval), g, s);
}

}  // namespace spg
