// ESC accumulator (Expand, Sort, Compress; Section 4) for the light columns
// of C = A x B: the lane-group bins, Op_j <= 256.
//
// A warp works a tile of kEscTile products: the columns of a bin list are cut
// into tiles of kEscTile / opmax columns (opmax = the bin's largest Op_j, so
// every tile fits), one column per lane.  Per tile:
//   Expand    every product A_ik * B_kj of the tile's columns is gathered
//             into the warp's shared memory as the key (c << rb) | i (c the
//             column's place in the tile, i the row, rb the row bits) and
//             its value;
//   Sort      a stable LSD radix sort of the keys (digits of kEscRadixBits
//             bits; a lane's place among the lanes with the same digit comes
//             from one ballot per digit bit), which orders the products by
//             column and, inside a column, by row.  In bins of short columns
//             (Op_j <= kEscRankOpMax) each product instead counts the
//             products of its own column that precede it in (row, position
//             of expansion) order: the products are expanded column after
//             column, so that count plus the column's first position is the
//             product's place in the sorted tile, the same place the stable
//             radix sort gives it.  Where (column, row, position) fits 32
//             bits the count runs over 16-byte words of an aligned window
//             around the column, else over the column's (row, position)
//             pairs alone;
//   Compress  equal keys are neighbours: the first of each run sums the run
//             in sorted order and writes one entry of C at its column's
//             pointer plus its rank among the column's runs.
// The sums do not depend on timing (no atomics on values).
//
// Modes: with values and no count output it is the numeric phase (C's
// column pointers come from the symbolic phase; a column whose run count
// differs is reported); without values it counts the runs of each column
// into cnt_out[j + 1] (the symbolic phase); with values and a count output it
// writes each column at base[j] and its count into cnt_out[j + 1] (the
// single-pass form, where base holds slots sized by Op_j).  Counting with a
// rank form needs no order: a product opens a run unless an earlier product
// of its column has its row, so the same comparisons count the runs.
//
// Keys are 32-bit: the forward passes' rows and the tile's column places must
// fit (rb + log2(columns per tile) <= 32); the host keeps hash tables
// otherwise.
#include "columns.cuh"
#include "esc.cuh"

namespace spg {

// Shared memory of one warp.  The radix sort and the exact rank form move
// (key, index) pairs, the values staying where the expansion put them and
// read through the index; the window rank form moves each value with its key
// (into the bucket counters' space, free once the column bounds are read).
template <bool VALS, typename VT>
struct EscWarp {
    uint32_t key[2][kEscTile];
    uint32_t cnt[2][1 << kEscRadixBits];
    int32_t hstart[32];
};
template <typename VT>
struct EscWarp<true, VT> {
    uint32_t key[2][kEscTile];
    VT val[kEscTile];
    uint32_t cnt[2][1 << kEscRadixBits];
    int32_t hstart[32];
    uint8_t idx[2][kEscTile];
};

// the exact-form rank sort keeps the sorted keys in cnt[1], the window form
// the sorted values in cnt[0..1]
static_assert((1 << kEscRadixBits) >= kEscTile, "radix count space holds a tile's keys");
static_assert(sizeof(uint32_t) * 2 * (1 << kEscRadixBits) >= sizeof(double) * kEscTile,
              "radix count space holds a tile's values");

template <typename VT, typename W>
__device__ __forceinline__ VT *wval(W &S) {
    return reinterpret_cast<VT *>(&S.cnt[0][0]);
}

template <bool VALS, typename VT>
__host__ __device__ constexpr size_t esc_warp_bytes() {
    return (sizeof(EscWarp<VALS, VT>) + 15) & ~size_t(15);
}

// CTAs per SM the kernels are built for (registers): the value-carrying
// form holds more shared memory per warp.
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

template <bool VALS, typename VT, int FORM>
__global__ void __launch_bounds__(kEscWarps * 32, esc_min_blocks<VALS>())
    k_esc(BinTask t, Operands o, const int64_t *base, int64_t *cnt_out, int32_t *Crow, VT *Cval, EscShape e) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_max, s_sum;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    EscWarp<VALS, VT> &S = *reinterpret_cast<EscWarp<VALS, VT> *>(smem + (size_t)warp * esc_warp_bytes<VALS, VT>());
    if (threadIdx.x == 0) s_max = s_sum = 0;
    __syncthreads();
    const TOps<VT> ops = typed<VT>(o);
    const uint64_t pol = keep_policy();
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t rowmask = e.rb >= 32 ? 0xffffffffu : ((1u << e.rb) - 1u);
    const int64_t ntiles = ceil_div(t.count, (int64_t)e.ct);
    unsigned long long my_max = 0, my_sum = 0;
    const int64_t tstride = (int64_t)gridDim.x * kEscWarps;
    int64_t tile = (int64_t)blockIdx.x * kEscWarps + warp;
    // the next tile's column ids and B column pointers are loaded while the
    // current tile is sorted
    int32_t nj = 0;
    int64_t np0 = 0, np1 = 0;
    auto fetch = [&](int64_t tl) {
        const int64_t f = tl * e.ct;
        if (tl < ntiles && lane < e.ct && f + lane < t.count) {
            nj = t.cols[f + lane];
            np0 = ops.Bcp[nj];
            np1 = ops.Bcp[nj + 1];
        }
    };
    fetch(tile);
    for (; tile < ntiles; tile += tstride) {
        const int64_t first = tile * e.ct;
        const int nc = (int)(t.count - first < e.ct ? t.count - first : e.ct);
        // ---- the tile's columns, one per lane: B entries and their offsets
        const int32_t j = lane < nc ? nj : 0;
        const int64_t p0 = lane < nc ? np0 : 0;
        const int nb = lane < nc ? (int)(np1 - np0) : 0;
        int64_t cb = 0, ccap = 0;
        if (lane < nc) {
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
        // ---- expand: 32 B entries per round, then their products; the
        // first pass's digits are counted as the keys are written
        constexpr uint32_t DM = (1u << kEscRadixBits) - 1u;
#pragma unroll
        for (int b = lane; b < (1 << kEscRadixBits); b += 32) S.cnt[0][b] = 0u;
        __syncwarp();
        int n = 0;
        bool over = false;
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
            if (n + total > kEscTile) {  // only if the pattern changed since planning
                over = true;
                break;
            }
            // products per column place (the rank sort's column bounds)
            if (FORM != kEscRadix && en < E && z > 0) atomicAdd(&S.cnt[0][c], (uint32_t)z);
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                const int s = esc_owner(zexcl, q < total ? q : total - 1);
                const int64_t a0s = __shfl_sync(0xffffffffu, a0, s);
                const int exs = __shfl_sync(0xffffffffu, zexcl, s);
                const int cs = __shfl_sync(0xffffffffu, c, s);
                VT bs = VT(0);
                if (VALS) bs = __shfl_sync(0xffffffffu, bv, s);
                if (q < total) {
                    const int64_t qa = a0s + (q - exs);
                    const int32_t row = ld_keep(ops.Arow + qa, pol);
                    const uint32_t key = ((uint32_t)cs << e.rb) | ((uint32_t)row & rowmask);
                    // rank sort: the key (window form) or the row (exact
                    // form) with the position of expansion below it: distinct,
                    // and ordered as the stable radix sort orders the keys
                    if constexpr (FORM == kEscRankWindow) {
                        S.key[1][n + q] = (key << 8) | (uint32_t)(n + q);
                    } else if constexpr (FORM == kEscRankExact) {
                        S.key[0][n + q] = key;
                        S.key[1][n + q] = (((uint32_t)row & rowmask) << 8) | (uint32_t)(n + q);
                    } else {
                        S.key[0][n + q] = key;
                        atomicAdd(&S.cnt[0][key & DM], 1u);
                        if constexpr (VALS) S.idx[0][n + q] = (uint8_t)(n + q);
                    }
                    if constexpr (VALS) S.val[n + q] = ld_keep(ops.Aval + qa, pol) * bs;
                }
            }
            n += total;
        }
        if (over) {
            if (lane == 0) set_error(t.ctrl, SPG_ERR_INVALID, kDetailCountMismatch + t.bin, j);
            continue;
        }
        __syncwarp();
        // ---- sort: ranks counted within columns, or a stable LSD radix sort
        // over the key bits (the counts of pass p + 1's digits are taken while
        // pass p scatters the keys)
        int cur = 0;
        if constexpr (FORM != kEscRadix) {
            // column place l's products are positions [beg, end) of lane l
            const int pc = lane < nc ? (int)S.cnt[0][lane] : 0;
            int pincl = pc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, pincl, d);
                if (lane >= d) pincl += v;
            }
            const int pbeg = pincl - pc;
            if constexpr (FORM == kEscRankWindow) {
                // composite keys above every other up to the next multiple of 4
                const int n4 = (n + 3) & ~3;
                if (n + lane < n4) S.key[1][n + lane] = 0xffffffffu;
            }
            // counting only: no order is needed; a product repeats a row when
            // an earlier product of its column has it (the same key above a
            // smaller position), and a column's runs are its products less
            // its repeats
            if constexpr (!VALS) S.hstart[lane] = 0;
            __syncwarp();
            for (int i0 = 0; i0 < n; i0 += 32) {
                const int i = i0 + lane;
                const bool valid = i < n;
                const uint32_t me = valid ? S.key[1][i] : 0u;
                if constexpr (FORM == kEscRankWindow) {
                    const int c = (int)(me >> (e.rb + 8)) & 31;
                    const int b = __shfl_sync(0xffffffffu, pbeg, c);
                    const int en = __shfl_sync(0xffffffffu, pincl, c);
                    if (valid) {
                        // every position before lo holds an earlier column
                        // (a smaller composite key) and every one from hi on
                        // a later column or a pad: counting the smaller keys
                        // in [lo, hi) completes the place
                        const int lo = b & ~3, hi = (en + 3) & ~3;
                        if constexpr (VALS) {
                            int at = lo;
                            for (int q = lo; q < hi; q += 4) {
                                const uint4 k4 = *reinterpret_cast<const uint4 *>(&S.key[1][q]);
                                at += (int)(k4.x < me) + (int)(k4.y < me) + (int)(k4.z < me) + (int)(k4.w < me);
                            }
                            S.key[0][at] = me >> 8;
                            // the value moves with its key, into the radix
                            // counts' space (read above, free from here on)
                            wval<VT>(S)[at] = S.val[me & 0xffu];
                        } else {
                            // x in [me - pos, me): the same key, earlier
                            const uint32_t base = me & ~0xffu, pm = me & 0xffu;
                            bool dup = false;
                            for (int q = lo; q < hi; q += 4) {
                                const uint4 k4 = *reinterpret_cast<const uint4 *>(&S.key[1][q]);
                                dup |= (k4.x - base < pm) | (k4.y - base < pm) | (k4.z - base < pm) |
                                       (k4.w - base < pm);
                            }
                            if (dup) atomicAdd(&S.hstart[c], 1);
                        }
                    }
                } else {
                    const uint32_t k = valid ? S.key[0][i] : 0u;
                    const int c = (int)(k >> e.rb) & 31;
                    const int b = __shfl_sync(0xffffffffu, pbeg, c);
                    const int en = __shfl_sync(0xffffffffu, pincl, c);
                    if (valid && VALS) {
                        // the row composites of the column alone
                        int at = b, q = b;
                        for (; q + 4 <= en; q += 4) {
                            const uint32_t x0 = S.key[1][q], x1 = S.key[1][q + 1];
                            const uint32_t x2 = S.key[1][q + 2], x3 = S.key[1][q + 3];
                            at += (int)(x0 < me) + (int)(x1 < me) + (int)(x2 < me) + (int)(x3 < me);
                        }
                        for (; q < en; ++q) at += (int)(S.key[1][q] < me);
                        // key[0] is still being read: the sorted keys go to the
                        // radix counts' space, free here
                        S.cnt[1][at] = k;
                        if constexpr (VALS) S.idx[1][at] = (uint8_t)i;
                    } else if (valid) {
                        const uint32_t base = me & ~0xffu, pm = me & 0xffu;
                        bool dup = false;
                        for (int q = b; q < en; ++q) dup |= S.key[1][q] - base < pm;
                        if (dup) atomicAdd(&S.hstart[c], 1);
                    }
                }
            }
            __syncwarp();
        }
        const unsigned vm_all = 0xffffffffu;
        for (int pass = 0; FORM == kEscRadix && pass < e.passes; ++pass) {
            const int sh = pass * kEscRadixBits;
            uint32_t *cnt = S.cnt[pass & 1];
            uint32_t *ncnt = S.cnt[(pass + 1) & 1];
            const bool more = pass + 1 < e.passes;
            {  // exclusive scan of the buckets: lane l owns the 8 buckets from 8 l
                constexpr int PER = (1 << kEscRadixBits) / 32;
                uint32_t v[PER];
                uint32_t run = 0;
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    v[u] = cnt[lane * PER + u];
                    const uint32_t x = v[u];
                    v[u] = run;
                    run += x;
                }
                uint32_t incl = run;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += y;
                }
                const uint32_t off = incl - run;
#pragma unroll
                for (int u = 0; u < PER; ++u) cnt[lane * PER + u] = v[u] + off;
                if (more)
#pragma unroll
                    for (int u = 0; u < PER; ++u) ncnt[lane * PER + u] = 0u;
            }
            __syncwarp();
            for (int i0 = 0; i0 < n; i0 += 32) {
                const int i = i0 + lane;
                const bool valid = i < n;
                const uint32_t k = valid ? S.key[cur][i] : 0u;
                uint8_t ix = 0;
                if constexpr (VALS) ix = valid ? S.idx[cur][i] : (uint8_t)0;
                const uint32_t dg = (k >> sh) & DM;
                // the lanes holding the same digit: one ballot per digit bit
                unsigned same = __ballot_sync(vm_all, valid);
#pragma unroll
                for (int b = 0; b < kEscRadixBits; ++b) {
                    const bool bit = (dg >> b) & 1u;
                    const unsigned bb = __ballot_sync(vm_all, bit);
                    same &= bit ? bb : ~bb;
                }
                const int leader = __ffs(same | (1u << lane)) - 1;
                uint32_t at = 0;
                if (valid && lane == leader) {
                    at = cnt[dg];
                    cnt[dg] = at + (uint32_t)__popc(same);
                }
                at = __shfl_sync(0xffffffffu, at, leader) + (uint32_t)__popc(same & lt);
                if (valid) {
                    S.key[cur ^ 1][at] = k;
                    if constexpr (VALS) S.idx[cur ^ 1][at] = ix;
                    if (more) atomicAdd(&ncnt[(k >> (sh + kEscRadixBits)) & DM], 1u);
                }
                __syncwarp();
            }
            cur ^= 1;
        }
        // ---- compress: the first key of each run writes the run's sum (not
        // needed when the ranks only counted runs)
        constexpr bool ranked_counts = !VALS && FORM != kEscRadix;
        int64_t cnt = 0;
        if constexpr (ranked_counts) {
            cnt = lane < nc ? (int64_t)S.cnt[0][lane] - S.hstart[lane] : 0;
        } else {
            constexpr bool moved = FORM == kEscRankExact;
            const uint32_t *skey = moved ? S.cnt[1] : S.key[cur];
            const uint8_t *sidx = nullptr;
            if constexpr (VALS && FORM != kEscRankWindow) sidx = moved ? S.idx[1] : S.idx[cur];
            if (lane < 32) S.hstart[lane] = 0x7fffffff;  // columns without runs stay unset
            __syncwarp();
            int hbase = 0;
            for (int i0 = 0; i0 < n; i0 += 32) {
                const int i = i0 + lane;
                const bool valid = i < n;
                const uint32_t k = valid ? skey[i] : 0u;
                const uint32_t kp = valid && i > 0 ? skey[i - 1] : 0u;
                const bool head = valid && (i == 0 || kp != k);
                const unsigned hm = __ballot_sync(0xffffffffu, head);
                const int hr = hbase + __popc(hm & lt);
                hbase += __popc(hm);
                const int c = (int)(k >> e.rb);
                if (head && (i == 0 || (int)(kp >> e.rb) != c)) S.hstart[c] = hr;
                __syncwarp();
                if constexpr (VALS) {
                    const int64_t cbase = __shfl_sync(0xffffffffu, cb, c & 31);
                    const int64_t cc = __shfl_sync(0xffffffffu, ccap, c & 31);
                    if (head) {
                        VT sum;
                        if constexpr (FORM == kEscRankWindow) {  // values in sorted order
                            const VT *sv = wval<VT>(S);
                            sum = sv[i];
                            for (int m2 = i + 1; m2 < n && skey[m2] == k; ++m2) sum += sv[m2];
                        } else {
                            sum = S.val[sidx[i]];
                            for (int m2 = i + 1; m2 < n && skey[m2] == k; ++m2) sum += S.val[sidx[m2]];
                        }
                        const int64_t r = hr - S.hstart[c];
                        // a column with more runs than its place holds is reported
                        // below and not written past its place
                        if (r < cc) {
                            Crow[cbase + r] = ops.crow((int32_t)(k & rowmask));
                            Cval[cbase + r] = sum;
                        }
                    }
                }
            }
            __syncwarp();
            // ---- per-column run counts: written (symbolic, single pass) or checked.
            // A column's runs end where the next column with runs starts.
            const int st = lane < nc ? S.hstart[lane] : 0x7fffffff;
            int nxt = st;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_down_sync(0xffffffffu, nxt, d);
                if (lane + d < 32 && v < nxt) nxt = v;
            }
            nxt = __shfl_down_sync(0xffffffffu, nxt, 1);
            if (lane == 31 || nxt > hbase) nxt = hbase;
            cnt = st == 0x7fffffff ? 0 : (int64_t)(nxt - st);
        }
        if (lane < nc) {
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
    if (e.ct > 32) e.ct = 32;
    if (e.ct < 1) return false;
    int cb = 0;
    while ((1 << cb) < e.ct) ++cb;
    int rb = 1;
    while (rb < 32 && ((int64_t)1 << rb) < m) ++rb;
    e.rb = rb;
    const int bits = rb + cb;
    if (bits > 32) return false;
    // the rank sort's composite keys carry 8 bits of position (kEscTile)
    e.rank = opmax > kEscRankOpMax ? kEscRadix
             : bits + 8 <= 32      ? kEscRankWindow
             : rb + 8 <= 32        ? kEscRankExact
                                   : kEscRadix;
    e.passes = e.rank ? 0 : (bits + kEscRadixBits - 1) / kEscRadixBits;
    return true;
}

template <bool VALS, typename VT>
static cudaError_t launch_esc_t(const BinTask &t, const Operands &o, const int64_t *base, int64_t *cnt_out,
                                int32_t *Crow, VT *Cval, const EscShape &e, int sms, cudaStream_t s) {
    if (t.count <= 0) return cudaSuccess;
    auto k = e.rank == kEscRankWindow ? k_esc<VALS, VT, kEscRankWindow>
             : e.rank == kEscRankExact ? k_esc<VALS, VT, kEscRankExact>
                                       : k_esc<VALS, VT, kEscRadix>;
    const size_t smem = (size_t)kEscWarps * esc_warp_bytes<VALS, VT>();
    esc_allow_smem(k, smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kEscWarps * 32, smem) != cudaSuccess || occ < 1)
        occ = 1;
    const int64_t ntiles = ceil_div(t.count, (int64_t)e.ct);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(ntiles, kEscWarps), (int64_t)occ * sms));
    k<<<(unsigned)grid, kEscWarps * 32, smem, s>>>(t, o, base, cnt_out, Crow, Cval, e);
    return cudaGetLastError();
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
