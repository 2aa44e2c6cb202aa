// Internal definitions shared by the kernels and the host orchestration of
// the column-wise SpGEMM C = A x B (arXiv 2303.02471).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/spgemm.h"

namespace spg {

// ------------------------------------------------------------------ bins
// Columns of B are grouped by Op_j (Section 3.1) instead of being sorted by
// decreasing Op_j: every bin runs one kernel whose launch shape and table
// size fit the bin's largest Op_j (Section 3.2's adaptive table size, taken
// per bin and per column).
constexpr int kNumWarpBins = 6;  // warp-group hash bins, Op_j <= 8 .. 256
constexpr int kNumCtaBins = 5;   // CTA shared-memory hash bins, Op_j <= 512 .. 8192
constexpr int BIN_EMPTY = 0;
constexpr int BIN_WARP0 = 1;
constexpr int BIN_CTA0 = BIN_WARP0 + kNumWarpBins;   // 7
constexpr int BIN_GLOBAL = BIN_CTA0 + kNumCtaBins;   // 12
constexpr int BIN_DENSE = BIN_GLOBAL + 1;            // 13
constexpr int NBINS = BIN_DENSE + 1;                 // 14

// Group width G (lanes per column) and entries per lane R of each warp bin;
// a bin holds columns with Op_j <= G * R.
__host__ __device__ constexpr int warp_bin_G(int b) {
    return b == 0 ? 8 : b == 1 ? 8 : b == 2 ? 16 : 32;
}
__host__ __device__ constexpr int warp_bin_R(int b) {
    return b == 0 ? 1 : b == 1 ? 2 : b == 2 ? 2 : b == 3 ? 2 : b == 4 ? 4 : 8;
}
__host__ __device__ constexpr int warp_bin_opmax(int b) { return warp_bin_G(b) * warp_bin_R(b); }
__host__ __device__ constexpr int64_t cta_bin_opmax(int c) { return 512LL << c; }

// Bin of a column with Op_j = op under threshold t and CTA-hash limit; a
// column of a lane-group bin moves `promote` group bins up (more lanes and
// table slots per column), at most to the last group bin.
__host__ __device__ inline int bin_of(int64_t op, int64_t t, int64_t hash_cta_max, int promote = 0) {
    if (op <= 0) return BIN_EMPTY;
    if (op >= t) return BIN_DENSE;
    for (int b = 0; b < kNumWarpBins; ++b)
        if (op <= warp_bin_opmax(b))
            return BIN_WARP0 + (b + promote < kNumWarpBins ? b + promote : kNumWarpBins - 1);
    if (op <= hash_cta_max) {
        for (int c = 0; c < kNumCtaBins; ++c)
            if (op <= cta_bin_opmax(c)) return BIN_CTA0 + c;
    }
    return BIN_GLOBAL;
}

// ------------------------------------------------------- control block
// Small device block at the start of the workspace; copied to the host in
// one transfer.  Error codes are spg_status values; the first one wins.
struct Ctrl {
    int32_t err;
    int32_t err_detail;
    int64_t err_index;
    unsigned long long hist[NBINS];     // columns per bin
    unsigned long long fill[NBINS];     // scatter cursors
    unsigned long long maxnnz[NBINS];   // largest nnz(C_j) per bin
    unsigned long long work[NBINS];     // dynamic work counters (CTA kernels)
    unsigned long long maxop[NBINS];    // largest Op_j per bin
    unsigned long long binprod[NBINS];  // sum of Op_j per bin
    unsigned long long binnnz[NBINS];   // sum of nnz(C_j) per bin
    unsigned long long binnnzb[NBINS];  // sum of nnz(B_j) per bin
    unsigned long long products;        // sum_j Op_j
    unsigned long long capsum;          // sum_j min(Op_j, rows): the single pass's slots
    unsigned long long pad[2];
};

// Code for a column whose numeric count disagrees with the symbolic one
// (the pattern changed between the phases).
constexpr int kDetailCountMismatch = 100;
// Code for an entry of A whose row held no entry when the plan was made.
constexpr int kDetailRowMap = 200;

__device__ inline void set_error(Ctrl *ctrl, int code, int detail, int64_t index) {
    if (atomicCAS(&ctrl->err, 0, code) == 0) {
        ctrl->err_detail = detail;
        ctrl->err_index = index;
    }
}

// Per-bin launch description passed by value to the kernels.
struct BinArgs {
    const int32_t *cols;  // column ids of this bin
    int64_t count;        // number of columns
    int bin;              // bin id
};

// CSC operand views passed by value.
template <typename VT>
struct Csc {
    const int64_t *cp;
    const int32_t *row;
    const VT *val;
    int64_t nrows, ncols;
};

// ------------------------------------------------------------- hashing
// Multiplicative hashing (Knuth, TAOCP vol. 3, 6.4) with the golden-ratio
// constant; the slot is the high part of (x * c mod 2^32) * H / 2^32, which
// equals the top log2(H) bits when H is a power of two and also serves
// tables of any size.  Section 3.2 writes h(i) = (i * c) mod H; with H a
// power of two that keeps only the low bits of i, which collide on the
// regular strides of stencil matrices, so the high bits are used instead.
__device__ __forceinline__ uint32_t hash_slot(int32_t row, uint32_t H) {
    uint32_t x = static_cast<uint32_t>(row) * 2654435761u;
    return static_cast<uint32_t>((static_cast<uint64_t>(x) * H) >> 32);
}

constexpr int32_t kEmptyKey = -1;

// Insert `row` into an open-addressing key table of H slots with linear
// probing (wrap-around, Section 3.2).  Returns the slot, sets `fresh` when
// this call created the key; returns -1 after H probes (table full).
__device__ __forceinline__ int32_t hash_insert(int32_t *keys, uint32_t H, int32_t row, bool &fresh) {
    uint32_t h = hash_slot(row, H);
    fresh = false;
    for (uint32_t probe = 0; probe < H; ++probe) {
        int32_t cur = *((volatile int32_t *)&keys[h]);
        if (cur == row) return static_cast<int32_t>(h);
        if (cur == kEmptyKey) {
            int32_t old = atomicCAS(&keys[h], kEmptyKey, row);
            if (old == kEmptyKey) { fresh = true; return static_cast<int32_t>(h); }
            if (old == row) return static_cast<int32_t>(h);
        }
        h = (h + 1 == H) ? 0u : h + 1;
    }
    return -1;
}

// Look a row up without inserting; -1 when absent.
__device__ __forceinline__ int32_t hash_find(const int32_t *keys, uint32_t H, int32_t row) {
    uint32_t h = hash_slot(row, H);
    for (uint32_t probe = 0; probe < H; ++probe) {
        int32_t cur = keys[h];
        if (cur == row) return static_cast<int32_t>(h);
        if (cur == kEmptyKey) return -1;
        h = (h + 1 == H) ? 0u : h + 1;
    }
    return -1;
}

// ------------------------------------------------------- small helpers
__device__ __forceinline__ unsigned group_mask(int G) {
    if (G == 32) return 0xffffffffu;
    unsigned lane = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lane & ~(G - 1));
}

template <int G>
__device__ __forceinline__ int group_incl_scan(unsigned mask, int v) {
    const int gl = threadIdx.x & (G - 1);
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        int o = __shfl_up_sync(mask, v, d, G);
        if (gl >= d) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T shfl_idx(unsigned mask, T v, int src, int width) {
    return __shfl_sync(mask, v, src, width);
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline uint32_t next_pow2_u32(uint32_t v) {
    uint32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Compare-exchange used by the bitonic networks: after the call the pair
// (a at the lower index, b at the higher) is ordered ascending if `up`.
template <typename VT>
__device__ __forceinline__ void cas_pair(int32_t &ka, VT &va, int32_t &kb, VT &vb, bool up) {
    bool swap = up ? (ka > kb) : (ka < kb);
    if (swap) {
        int32_t tk = ka; ka = kb; kb = tk;
        VT tv = va; va = vb; vb = tv;
    }
}

// Bitonic sort of N = G * R (key, value) pairs held by a lane group: element
// e = r * G + gl sits in register r of group lane gl.  Keys ascend; padding
// keys are INT32_MAX.  Partners closer than G are exchanged by shuffles,
// farther ones are registers of the same lane.
template <int G, int R, typename VT>
__device__ __forceinline__ void group_bitonic_sort(unsigned mask, int32_t (&key)[R], VT (&val)[R]) {
    const int gl = threadIdx.x & (G - 1);
    constexpr int N = G * R;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= G) {
                const int jr = j / G;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((r & jr) == 0) {
                        const int e = r * G + gl;
                        const bool up = (e & k) == 0;
                        cas_pair(key[r], val[r], key[r | jr], val[r | jr], up);
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int e = r * G + gl;
                    int32_t ok = __shfl_xor_sync(mask, key[r], j, G);
                    VT ov = __shfl_xor_sync(mask, val[r], j, G);
                    const bool up = (e & k) == 0;
                    const bool lower = (e & j) == 0;
                    // lower element keeps the min when ascending, else max
                    bool take_other = lower ? (up ? ok < key[r] : ok > key[r])
                                            : (up ? ok > key[r] : ok < key[r]);
                    if (take_other) { key[r] = ok; val[r] = ov; }
                }
            }
        }
    }
}

}  // namespace spg
