// Symbolic phase: nnz of every column of C = A x B, per bin.
//
// Hash bins count the distinct rows a column's products touch with an
// open-addressing key table sized from Op_j (Section 3.2: the table is
// larger than the column's product count); the dense bin (Op_j >= t,
// Section 3.3) sets one bit per touched row, the SPA flags of Algorithm 1,
// and counts the bits (Algorithm 1's counter).
#include "columns.cuh"

namespace spg {

constexpr int kGroupThreads = 256;

// ------------------------------------------------- warp-group hash bins
// One group of G lanes per column; the group's table has 2 G R slots for
// Op_j <= G R, so it is at most half full.
template <int G, int R>
__global__ void __launch_bounds__(kGroupThreads, 1) k_sym_group(BinTask t, Operands o, int64_t *Ccp) {
    constexpr int H = 2 * G * R;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_max, s_sum;
    int32_t *keys = reinterpret_cast<int32_t *>(smem) + (threadIdx.x / G) * H;
    if (threadIdx.x == 0) s_max = s_sum = 0;
    __syncthreads();
    const unsigned mask = group_mask(G);
    const int gl = threadIdx.x & (G - 1);
    const int64_t gidx = (int64_t)blockIdx.x * (kGroupThreads / G) + threadIdx.x / G;
    uint32_t Hj = (uint32_t)H >> t.shrink;
    if (Hj < 1) Hj = 1;
    if (gidx < t.count) {
        const int32_t j = t.cols[gidx];
        bool ovf = false;
        const int cnt = sym_group_column<G, R>(mask, typed<float>(o), j, keys, Hj, ovf);
        if (ovf) set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
        if (gl == 0) {
            Ccp[j + 1] = cnt;
            atomicMax(&s_max, (unsigned long long)cnt);
            atomicAdd(&s_sum, (unsigned long long)cnt);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_max) {
        atomicMax(&t.ctrl->maxnnz[t.bin], s_max);
        atomicAdd(&t.ctrl->binnnz[t.bin], s_sum);
    }
}

// ------------------------------------------------------- CTA hash bins
// One CTA per column (dynamic work counter); table of pow2 >= 2 Op_j keys in
// shared memory (KSM), or in the CTA's global scratch for the global bin.
template <bool KSM>
__global__ void __launch_bounds__(1024, 1) k_sym_cta(BinTask t, Operands o, int64_t *Ccp, int64_t cap_slots) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ unsigned long long s_cnt, s_max, s_sum;
    const WalkSmem<float> w = carve_walk<float>(smem);
    int32_t *keys = KSM ? reinterpret_cast<int32_t *>(smem + walk_smem_bytes<float>(blockDim.x))
                        : reinterpret_cast<int32_t *>(t.scratch + (size_t)blockIdx.x * t.scratch_stride);
    const TOps<float> ops = typed<float>(o);
    if (threadIdx.x == 0) s_max = s_sum = 0;
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        int64_t want = global_sym_slots(t.op[j], t.m);
        if (want > cap_slots) want = cap_slots;
        uint32_t H = (uint32_t)(want >> t.shrink);
        if (H < 1) H = 1;
        bool ovf = false;
        const int64_t cnt = sym_cta_column(ops, j, keys, H, w, &s_cnt, ovf);
        if (ovf) set_error(t.ctrl, SPG_ERR_TABLE_OVERFLOW, t.bin, j);
        if (threadIdx.x == 0) {
            Ccp[j + 1] = cnt;
            if ((unsigned long long)cnt > s_max) s_max = cnt;
            s_sum += cnt;
        }
    }
    if (threadIdx.x == 0 && s_max) {
        atomicMax(&t.ctrl->maxnnz[t.bin], s_max);
        atomicAdd(&t.ctrl->binnnz[t.bin], s_sum);
    }
}

// ------------------------------------------------------------ dense bin
// SPA flags as a bitmap of m bits (shared memory when BSM, else global
// scratch); nnz(C_j) is the number of set bits.  Columns with a cache slot
// keep their flags for the numeric phase.
template <bool BSM>
// launched with at most kSymCtaThreads threads (the host caps them); the
// walk issues an instruction on most cycles, so the kernel is built for a
// full SM of warps (eight CTAs of 256 threads, 32 registers, no spills)
__global__ void __launch_bounds__(kSymCtaThreads, 8) k_sym_dense(BinTask t, Operands o, int64_t *Ccp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t s_col;
    __shared__ unsigned long long s_cnt, s_max, s_sum;
    const WalkSmem<float> w = carve_walk<float>(smem);
    uint32_t *bm = BSM ? reinterpret_cast<uint32_t *>(smem + walk_smem_bytes<float>(blockDim.x))
                       : reinterpret_cast<uint32_t *>(t.scratch + (size_t)blockIdx.x * t.scratch_stride);
    const TOps<float> ops = typed<float>(o);
    for (int64_t i = threadIdx.x; i < t.W; i += blockDim.x) bm[i] = 0u;
    if (threadIdx.x == 0) s_max = s_sum = 0;
    for (;;) {
        if (threadIdx.x == 0) s_col = (int64_t)atomicAdd(&t.ctrl->work[t.bin], 1ULL);
        __syncthreads();
        const int64_t ci = s_col;
        if (ci >= t.count) break;
        const int32_t j = t.cols[ci];
        uint32_t *keep = ci < t.cache_cols ? t.flag_cache + (size_t)ci * t.W : nullptr;
        const int64_t cnt = sym_dense_column(ops, j, bm, t.W, keep, w, &s_cnt);
        if (threadIdx.x == 0) {
            Ccp[j + 1] = cnt;
            if ((unsigned long long)cnt > s_max) s_max = cnt;
            s_sum += cnt;
        }
    }
    if (threadIdx.x == 0 && s_max) {
        atomicMax(&t.ctrl->maxnnz[t.bin], s_max);
        atomicAdd(&t.ctrl->binnnz[t.bin], s_sum);
    }
}

// ------------------------------------------------------------- launches
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

// Shared-memory budget for the dense bitmap before it moves to global scratch.
constexpr size_t kBitmapSmemMax = 96 * 1024;

Geo symbolic_geometry(int bin, int64_t count, int64_t m, int threads, int sms, size_t smem_optin,
                      int64_t max_op, int shrink, int64_t scratch_ctas) {
    (void)shrink;
    Geo g;
    const int64_t W = ceil_div(m, 32);
    if (bin >= BIN_WARP0 && bin < BIN_CTA0) {
        const int b = bin - BIN_WARP0;
        const int G = warp_bin_G(b), R = warp_bin_R(b);
        g.threads = kGroupThreads;
        g.smem = (size_t)(kGroupThreads / G) * 2 * G * R * 4;
        g.grid = (int)ceil_div(count, kGroupThreads / G);
        return g;
    }
    g.threads = threads;
    const size_t walk = walk_smem_bytes<float>(threads);
    if (bin >= BIN_CTA0 && bin < BIN_GLOBAL) {
        g.slots = global_sym_slots(cta_bin_opmax(bin - BIN_CTA0), m);
        g.smem = walk + (size_t)g.slots * 4;
        int occ = occupancy(k_sym_cta<true>, threads, g.smem);
        g.grid = (int)std::min<int64_t>(count, (int64_t)occ * sms);
    } else if (bin == BIN_GLOBAL) {
        g.slots = global_sym_slots(max_op, m);
        g.smem = walk;
        int occ = occupancy(k_sym_cta<true>, threads, g.smem);
        g.grid = (int)std::min<int64_t>(std::min<int64_t>(count, (int64_t)occ * sms), scratch_ctas);
    } else {  // dense
        const size_t bmb = (size_t)W * 4;
        g.bm_global = bmb > kBitmapSmemMax || walk + bmb > smem_optin;
        g.smem = walk + (g.bm_global ? 0 : bmb);
        int occ = occupancy(k_sym_dense<true>, threads, g.smem);
        int64_t grid = std::min<int64_t>(count, (int64_t)occ * sms);
        if (g.bm_global) grid = std::min<int64_t>(grid, scratch_ctas);
        g.grid = (int)grid;
    }
    if (g.grid < 1) g.grid = 1;
    return g;
}

cudaError_t launch_symbolic_bin(const BinTask &t, const Operands &o, int64_t *Ccp, const Geo &g,
                                cudaStream_t s) {
    if (t.count <= 0) return cudaSuccess;
    if (t.bin >= BIN_WARP0 && t.bin < BIN_CTA0) {
        switch (t.bin - BIN_WARP0) {
#define SYM_CASE(b)                                                                        \
    case b: {                                                                              \
        auto k = k_sym_group<warp_bin_G(b), warp_bin_R(b)>;                                \
        allow_smem(k, g.smem);                                                             \
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp);                                    \
        break;                                                                             \
    }
            SYM_CASE(0) SYM_CASE(1) SYM_CASE(2) SYM_CASE(3) SYM_CASE(4) SYM_CASE(5)
#undef SYM_CASE
        }
    } else if (t.bin < BIN_DENSE) {
        auto k = t.bin == BIN_GLOBAL ? k_sym_cta<false> : k_sym_cta<true>;
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp, g.slots);
    } else {
        auto k = g.bm_global ? k_sym_dense<false> : k_sym_dense<true>;
        allow_smem(k, g.smem);
        k<<<g.grid, g.threads, g.smem, s>>>(t, o, Ccp);
    }
    return cudaGetLastError();
}

}  // namespace spg
