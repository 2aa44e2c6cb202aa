// ESC accumulator (Expand, Sort, Compress; Section 4) for the light columns
// of C = A x B: the lane-group bins, Op_j <= 256.
//
// A warp works a tile of kEscTile = 256 product slots: the columns of a bin
// list are cut into tiles of 256 / S columns, S = the bin's largest Op_j (a
// power of two, 8 .. 256), and column c of the tile owns the aligned slots
// [c S, (c + 1) S).  Per tile:
//   Expand    every product A_ik * B_kj of the tile's columns is gathered:
//             its value into the warp's shared memory at its slot, its key
//             (i << 8) | slot into the slot's key (unused slots hold a key
//             above every row);
//   Sort      the 256 keys sit in eight registers per lane (slot e in
//             register e / 32 of lane e % 32) and a bitonic network over the
//             slots, cut off at S, sorts every column's segment by row: the
//             stages exchange partners by shuffles (distance < 32) or within
//             a lane's registers, and the eight registers are independent;
//   Compress  equal rows are neighbours: the first of each run sums the run
//             in sorted order (values looked up through the slot in the key)
//             and writes one entry of C at its column's pointer plus its rank
//             among the column's runs.
// The sums do not depend on timing (no atomics on values).  The paper's ESC
// sorts with a radix sort tuned to its vector unit; a warp-level radix sort
// (8-bit digits, ranks from __match_any_sync) was measured here first and
// spent its time in chains of dependent shared-memory steps, which the
// register network does not have.
//
// Modes: with values and no count output it is the numeric phase (C's
// column pointers come from the symbolic phase; a column whose run count
// differs is reported); without values it counts the runs of each column
// into cnt_out[j + 1] (the symbolic phase); with values and a count output it
// writes each column at base[j] and its count into cnt_out[j + 1] (the
// single-pass form, where base holds slots sized by Op_j).
//
// Keys are 32-bit: the forward passes' rows must be below 2^24 - 1; the host
// keeps hash tables otherwise.
#include "columns.cuh"
#include "esc.cuh"

namespace spg {

constexpr uint32_t kEscPad = 0xffffffffu;

// Shared memory of one warp: the slots' keys (expansion, then the sorted
// keys), the run count of each of the tile's columns, and the values.
template <bool VALS, typename VT>
struct EscWarp {
    uint32_t key[kEscTile];
    int32_t cnt[32];
};
template <typename VT>
struct EscWarp<true, VT> {
    uint32_t key[kEscTile];
    int32_t cnt[32];
    VT val[kEscTile];
};

template <bool VALS, typename VT>
__host__ __device__ constexpr size_t esc_warp_bytes() {
    return (sizeof(EscWarp<VALS, VT>) + 15) & ~size_t(15);
}

// CTAs per SM the kernels are built for (registers).
template <bool VALS>
constexpr int esc_min_blocks() { return VALS ? 4 : 4; }

// Lane holding the owner of position q among 32 lanes with non-decreasing
// exclusive offsets `excl` (the last lane whose offset is <= q).
__device__ __forceinline__ int esc_owner(int excl, int q) {
    int s = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int ex = __shfl_sync(0xffffffffu, excl, s + step);
        if (ex <= q) s += step;
    }
    return s;
}

// Bitonic network over the 256 slots (slot e = r * 32 + lane in register r),
// stages kk = 2 .. S: every aligned segment of S slots ends up ascending.
template <int S>
__device__ __forceinline__ void esc_segment_sort(uint32_t (&k)[kEscTile / 32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= S; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jr = j / 32;
#pragma unroll
                for (int r = 0; r < kEscTile / 32; ++r) {
                    if ((r & jr) == 0) {
                        const int e = r * 32 + lane;
                        // direction from the slot's place in its segment: every
                        // segment ends ascending (the last stage has kk = S)
                        const bool up = ((e & (S - 1)) & kk) == 0;
                        const uint32_t a = k[r], b = k[r | jr];
                        const bool swap = up ? a > b : a < b;
                        k[r] = swap ? b : a;
                        k[r | jr] = swap ? a : b;
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < kEscTile / 32; ++r) {
                    const int e = r * 32 + lane;
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, k[r], j);
                    const bool up = ((e & (S - 1)) & kk) == 0;
                    const bool lower = (e & j) == 0;
                    // the lower slot keeps the minimum when ascending
                    const bool take = lower ? (up ? o < k[r] : o > k[r]) : (up ? o > k[r] : o < k[r]);
                    if (take) k[r] = o;
                }
            }
        }
    }
}

template <bool VALS, typename VT, int S>
__global__ void __launch_bounds__(kEscWarps * 32, esc_min_blocks<VALS>())
    k_esc(BinTask t, Operands o, const int64_t *base, int64_t *cnt_out, int32_t *Crow, VT *Cval) {
    constexpr int CT = kEscTile / S;   // columns per tile (<= 32)
    constexpr int NR = kEscTile / 32;  // key registers per lane
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_max, s_sum;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    EscWarp<VALS, VT> &W = *reinterpret_cast<EscWarp<VALS, VT> *>(smem + (size_t)warp * esc_warp_bytes<VALS, VT>());
    if (threadIdx.x == 0) s_max = s_sum = 0;
    __syncthreads();
    const TOps<VT> ops = typed<VT>(o);
    const uint64_t pol = keep_policy();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t ntiles = ceil_div(t.count, (int64_t)CT);
    unsigned long long my_max = 0, my_sum = 0;
    const int64_t tstride = (int64_t)gridDim.x * kEscWarps;
    int64_t tile = (int64_t)blockIdx.x * kEscWarps + warp;
    // the next tile's column ids, B column pointers and Op_j are loaded
    // while the current tile is sorted
    int32_t nj = 0;
    int64_t np0 = 0, np1 = 0, nop = 0;
    auto fetch = [&](int64_t tl) {
        const int64_t f = tl * CT;
        if (tl < ntiles && lane < CT && f + lane < t.count) {
            nj = t.cols[f + lane];
            np0 = ops.Bcp[nj];
            np1 = ops.Bcp[nj + 1];
            nop = t.op[nj];
        }
    };
    fetch(tile);
    for (; tile < ntiles; tile += tstride) {
        const int64_t first = tile * CT;
        const int nc = (int)(t.count - first < CT ? t.count - first : CT);
        // ---- the tile's columns, one per lane: B entries and their offsets
        const bool col = lane < nc;
        const int32_t j = col ? nj : 0;
        const int64_t p0 = col ? np0 : 0;
        const int nb = col ? (int)(np1 - np0) : 0;
        // products of the column (Op_j of the plan; products beyond it mean
        // the pattern changed: reported, never written past the segment)
        const int opc = col ? (int)nop : 0;
        int64_t cb = 0, ccap = 0;
        if (col) {
            cb = base[j];
            ccap = base[j + 1] - cb;  // entries the column's place holds
        }
        fetch(tile + tstride);
        int eincl = nb;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, eincl, d);
            if (lane >= d) eincl += v;
        }
        const int eexcl = eincl - nb;
        const int E = __shfl_sync(0xffffffffu, eincl, 31);
        // first flat product of each column (the expansion runs column by column)
        int pincl = opc;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, pincl, d);
            if (lane >= d) pincl += v;
        }
        const int pexcl = pincl - opc;
        // ---- expand: every slot starts as padding, products take their slots
#pragma unroll
        for (int r = 0; r < NR; ++r) W.key[r * 32 + lane] = kEscPad;
        __syncwarp();
        int n = 0;  // flat products so far
        bool bad = false;
        for (int e0 = 0; e0 < E; e0 += 32) {
            const int en = e0 + lane;
            const int c = esc_owner(eexcl, en < E ? en : E - 1);
            const int64_t p0c = __shfl_sync(0xffffffffu, p0, c);
            const int exc = __shfl_sync(0xffffffffu, eexcl, c);
            int z = 0;
            int64_t a0 = 0;
            VT bv = VT(0);
            if (en < E) {
                const int64_t p = p0c + (en - exc);
                const int32_t k = ops.Brow[p];
                a0 = ops.Acp[k];
                z = (int)(ops.Acp[k + 1] - a0);
                if (VALS) bv = ops.Bval[p];
            }
            int zincl = z;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, zincl, d);
                if (lane >= d) zincl += v;
            }
            const int zexcl = zincl - z;
            const int total = __shfl_sync(0xffffffffu, zincl, 31);
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                const int s = esc_owner(zexcl, q < total ? q : total - 1);
                const int64_t a0s = __shfl_sync(0xffffffffu, a0, s);
                const int exs = __shfl_sync(0xffffffffu, zexcl, s);
                const int cs = __shfl_sync(0xffffffffu, c, s);
                const int ps = __shfl_sync(0xffffffffu, pexcl, cs);
                const int os = __shfl_sync(0xffffffffu, opc, cs);
                VT bs = VT(0);
                if (VALS) bs = __shfl_sync(0xffffffffu, bv, s);
                if (q < total) {
                    const int within = n + q - ps;  // the product's place in its column
                    if (within >= 0 && within < os && within < S) {
                        const int slot = cs * S + within;
                        const int64_t qa = a0s + (q - exs);
                        const int32_t row = ld_keep(ops.Arow + qa, pol);
                        W.key[slot] = ((uint32_t)row << 8) | (uint32_t)slot;
                        if constexpr (VALS) W.val[slot] = ld_keep(ops.Aval + qa, pol) * bs;
                    } else {
                        bad = true;  // Op_j differs from the plan's
                    }
                }
            }
            n += total;
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
            continue;
        }
        __syncwarp();
        // ---- sort every column's segment by row
        uint32_t k[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) k[r] = W.key[r * 32 + lane];
        esc_segment_sort<S>(k);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < NR; ++r) W.key[r * 32 + lane] = k[r];
        __syncwarp();
        // ---- compress: the first slot of each run of equal rows writes the
        // run's sum; heads are ranked inside their column's segment
        int runs = 0;  // S >= 32: heads of the current column in earlier registers
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int e = r * 32 + lane;
            const int c = e / S;  // column of the slot (< CT <= 32)
            const int q = e % S;  // place in the column's sorted segment
            const int oc = __shfl_sync(0xffffffffu, opc, c);
            const bool valid = q < oc;
            const uint32_t kv = k[r];
            const uint32_t row = kv >> 8;
            const bool head = valid && (q == 0 || (W.key[e - 1] >> 8) != row);
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            int rank;
            if constexpr (S >= 32) {
                // every lane of the register is in the same column
                if ((r * 32) % S == 0) runs = 0;
                rank = runs + __popc(hm & lt);
                runs += __popc(hm);
                if ((r * 32) % S == S - 32 && lane == 0) W.cnt[c] = runs;
            } else {
                const unsigned seg = ((1u << S) - 1u) << (lane & ~(S - 1));
                rank = __popc(hm & seg & lt);
                if (q == 0) W.cnt[c] = __popc(hm & seg);
            }
            if constexpr (VALS) {
                const int64_t cbase = __shfl_sync(0xffffffffu, cb, c);
                const int64_t cc = __shfl_sync(0xffffffffu, ccap, c);
                if (head) {
                    VT sum = W.val[kv & 0xffu];
                    for (int m2 = e + 1; (m2 % S) != 0 && (m2 % S) < oc && (W.key[m2] >> 8) == row; ++m2)
                        sum += W.val[W.key[m2] & 0xffu];
                    // a column with more runs than its place holds is reported
                    // below and not written past its place
                    if (rank < cc) {
                        Crow[cbase + rank] = ops.crow((int32_t)row);
                        Cval[cbase + rank] = sum;
                    }
                }
            }
        }
        __syncwarp();
        // ---- per-column run counts: written (symbolic, single pass) or checked
        if (col) {
            const int64_t cnt = W.cnt[lane];
            if (cnt_out) {
                cnt_out[j + 1] = cnt;
                if ((unsigned long long)cnt > my_max) my_max = (unsigned long long)cnt;
                my_sum += (unsigned long long)cnt;
            } else if (ccap != cnt) {
                set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
            }
        }
        __syncwarp();
    }
    if (cnt_out) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            my_sum += __shfl_xor_sync(0xffffffffu, my_sum, d);
            const unsigned long long om = __shfl_xor_sync(0xffffffffu, my_max, d);
            if (om > my_max) my_max = om;
        }
        if (lane == 0 && my_sum) {
            atomicMax(&s_max, my_max);
            atomicAdd(&s_sum, my_sum);
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_max) {
            atomicMax(&t.ctrl->maxnnz[t.bin], s_max);
            atomicAdd(&t.ctrl->binnnz[t.bin], s_sum);
        }
    }
}

// ------------------------------------------------------------- launches
template <typename K>
static void esc_allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

bool esc_shape(int bin, int64_t m, EscShape &e) {
    if (bin < BIN_WARP0 || bin >= BIN_CTA0) return false;
    const int opmax = warp_bin_opmax(bin - BIN_WARP0);
    e.ct = kEscTile / opmax;
    if (e.ct < 1 || e.ct > 32) return false;
    // keys (row << 8) | slot stay below the padding key
    if (m >= ((int64_t)1 << 24) - 1) return false;
    int rb = 1;
    while (rb < 32 && ((int64_t)1 << rb) < m) ++rb;
    e.rb = rb;
    return true;
}

template <bool VALS, typename VT, int S>
static cudaError_t launch_esc_s(const BinTask &t, const Operands &o, const int64_t *base, int64_t *cnt_out,
                                int32_t *Crow, VT *Cval, int sms, cudaStream_t s) {
    auto k = k_esc<VALS, VT, S>;
    const size_t smem = (size_t)kEscWarps * esc_warp_bytes<VALS, VT>();
    esc_allow_smem(k, smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kEscWarps * 32, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t ntiles = ceil_div(t.count, (int64_t)(kEscTile / S));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(ntiles, kEscWarps), (int64_t)occ * sms));
    k<<<(unsigned)grid, kEscWarps * 32, smem, s>>>(t, o, base, cnt_out, Crow, Cval);
    return cudaGetLastError();
}

template <bool VALS, typename VT>
static cudaError_t launch_esc_t(const BinTask &t, const Operands &o, const int64_t *base, int64_t *cnt_out,
                                int32_t *Crow, VT *Cval, const EscShape &e, int sms, cudaStream_t s) {
    if (t.count <= 0) return cudaSuccess;
    switch (kEscTile / e.ct) {
        case 8: return launch_esc_s<VALS, VT, 8>(t, o, base, cnt_out, Crow, Cval, sms, s);
        case 16: return launch_esc_s<VALS, VT, 16>(t, o, base, cnt_out, Crow, Cval, sms, s);
        case 32: return launch_esc_s<VALS, VT, 32>(t, o, base, cnt_out, Crow, Cval, sms, s);
        case 64: return launch_esc_s<VALS, VT, 64>(t, o, base, cnt_out, Crow, Cval, sms, s);
        case 128: return launch_esc_s<VALS, VT, 128>(t, o, base, cnt_out, Crow, Cval, sms, s);
        case 256: return launch_esc_s<VALS, VT, 256>(t, o, base, cnt_out, Crow, Cval, sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_esc_bin(const BinTask &t, const Operands &o, const int64_t *base, int64_t *cnt_out,
                           int32_t *Crow, void *Cval, bool values, int dtype, const EscShape &e, int sms,
                           cudaStream_t s) {
    if (!values)
        return launch_esc_t<false, float>(t, o, base, cnt_out, nullptr, nullptr, e, sms, s);
    return dtype == SPG_F64
               ? launch_esc_t<true, double>(t, o, base, cnt_out, Crow, static_cast<double *>(Cval), e, sms, s)
               : launch_esc_t<true, float>(t, o, base, cnt_out, Crow, static_cast<float *>(Cval), e, sms, s);
}

}  // namespace spg
