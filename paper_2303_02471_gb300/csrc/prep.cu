// Preprocessing kernels of the column-wise SpGEMM (arXiv 2303.02471):
// input validation, the operation count Op_j with binning (Section 3.1's
// "Sorting" pre-pass, done as a bucket pass), per-bin column lists, and the
// int64 scan that turns per-column counts into C's column pointers.
#include <cstring>

#include "kernels.cuh"

namespace spg {

// CSC well-formedness (Section 2.1): colptr[0] = 0, colptr[n] = nnz,
// colptr non-decreasing, rows in [0, nrows).
__global__ void k_validate(const int64_t *__restrict__ cp, const int32_t *__restrict__ row,
                           int64_t nrows, int64_t ncols, int64_t nnz, int which, Ctrl *ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = tid; j <= ncols; j += stride) {
        int64_t c = cp[j];
        if ((j == 0 && c != 0) || (j == ncols && c != nnz) || (j < ncols && cp[j + 1] < c) || c < 0)
            set_error(ctrl, SPG_ERR_INVALID, which * 2 + 0, j);
    }
    for (int64_t e = tid; e < nnz; e += stride) {
        int32_t r = row[e];
        if (r < 0 || (int64_t)r >= nrows) set_error(ctrl, SPG_ERR_INVALID, which * 2 + 1, e);
    }
}

// Op_j = sum over stored B_kj of Z^A_k (Section 3.1), its bin, the bin
// histogram and the total product count.  Empty columns get nnz 0 here.
//
// A warp takes 32 columns, one per lane.  The columns are dealt through a
// permutation (index times `mult` modulo nB, mult coprime to nB) so that the
// heavy columns of a skewed matrix, which sit together (or, in R-MAT, at
// indices with few one bits), spread over the warps.  Columns with more than
// 32 B entries are walked by the whole warp one after another, its loads
// strided over the lanes; the others' entries are walked 32 at a time as one
// flattened sequence (the owner of an entry is found by a search over the
// lanes' entry offsets) and the Z^A_k of an owner's lanes are summed by a
// segmented warp scan.  Per-bin statistics are summed over the warp before
// one shared atomic per bin present.
constexpr int kCountLong = 32;

__global__ void k_count_bin(const int64_t *__restrict__ Bcp, const int32_t *__restrict__ Brow,
                            const int64_t *__restrict__ Acp, int64_t nB, int64_t t, int64_t hmax, int promote,
                            int64_t mrows,
                            int64_t mult, int64_t *__restrict__ op, int64_t *__restrict__ Ccp, Ctrl *ctrl) {
    __shared__ unsigned long long s_hist[NBINS];
    __shared__ unsigned long long s_max[NBINS];
    __shared__ unsigned long long s_binprod[NBINS];
    __shared__ unsigned long long s_binb[NBINS];
    __shared__ unsigned long long s_prod, s_cap;
    __shared__ int64_t s_op[32 * 32];  // per warp: the Op of its 32 columns (blockDim <= 1024)
    if (threadIdx.x < NBINS) {
        s_hist[threadIdx.x] = 0;
        s_max[threadIdx.x] = 0;
        s_binprod[threadIdx.x] = 0;
        s_binb[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) s_prod = s_cap = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int64_t *wop = s_op + (threadIdx.x & ~31);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mine = 0, cap = 0;
    for (int64_t g0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; g0 < nB; g0 += nwarps * 32) {
        const int64_t g = g0 + lane;
        const bool on = g < nB;
        // mult < nB < 2^31 and g < nB: the product fits 63 bits
        const int64_t j = on ? (int64_t)(((unsigned long long)g * (unsigned long long)mult) % (unsigned long long)nB)
                             : 0;
        int64_t p0 = 0, nb = 0;
        if (on) {
            p0 = Bcp[j];
            nb = Bcp[j + 1] - p0;
        }
        wop[lane] = 0;
        // long columns: the whole warp, one column at a time
        unsigned longs = __ballot_sync(0xffffffffu, nb > kCountLong);
        while (longs) {
            const int c = __ffs(longs) - 1;
            longs &= longs - 1u;
            const int64_t pc = __shfl_sync(0xffffffffu, p0, c);
            const int64_t nc = __shfl_sync(0xffffffffu, nb, c);
            int64_t sz = 0;
            for (int64_t p = pc + lane; p < pc + nc; p += 32) {
                const int32_t k = Brow[p];
                sz += Acp[k + 1] - Acp[k];
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sz += __shfl_xor_sync(0xffffffffu, sz, d);
            if (lane == c) wop[c] = sz;
        }
        // short columns: their entries as one flattened sequence
        const int64_t ns = nb > kCountLong ? 0 : nb;
        int64_t eincl = ns;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, eincl, d);
            if (lane >= d) eincl += v;
        }
        const int64_t eexcl = eincl - ns;
        const int64_t E = __shfl_sync(0xffffffffu, eincl, 31);
        __syncwarp();
        for (int64_t e0 = 0; e0 < E; e0 += 32) {
            const int64_t e = e0 + lane;
            const int64_t q = e < E ? e : E - 1;
            int c = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int64_t ex = __shfl_sync(0xffffffffu, eexcl, c + step);
                if (ex <= q) c += step;
            }
            const int64_t pc = __shfl_sync(0xffffffffu, p0, c);
            const int64_t xc = __shfl_sync(0xffffffffu, eexcl, c);
            int64_t z = 0;
            if (e < E) {
                const int32_t k = Brow[pc + (e - xc)];
                z = Acp[k + 1] - Acp[k];
            }
            // owners are non-decreasing over the lanes: segmented inclusive sum
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t v = __shfl_up_sync(0xffffffffu, z, d);
                const int oc = __shfl_up_sync(0xffffffffu, c, d);
                if (lane >= d && oc == c) z += v;
            }
            const int cn = __shfl_down_sync(0xffffffffu, c, 1);
            if (e < E && (lane == 31 || e + 1 >= E || cn != c)) wop[c] += z;
            __syncwarp();
        }
        __syncwarp();
        const int64_t s = wop[lane];
    int b = -1;
        if (on) {
            op[j] = s;
            mine += (unsigned long long)s;
            cap += (unsigned long long)(s < mrows ? s : mrows);
            b = bin_of(s, t, hmax, promote);
            if (b == BIN_EMPTY) Ccp[j + 1] = 0;
        }
        // per-bin statistics, one group of lanes per bin present
        unsigned pending = __ballot_sync(0xffffffffu, on);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const int bb = __shfl_sync(0xffffffffu, b, leader);
            const unsigned m = __ballot_sync(0xffffffffu, on && b == bb);
            unsigned long long sm = (m >> lane) & 1u ? (unsigned long long)s : 0ull;
            unsigned long long mx = sm;
            unsigned long long nbs = (m >> lane) & 1u ? (unsigned long long)nb : 0ull;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                sm += __shfl_xor_sync(0xffffffffu, sm, d);
                nbs += __shfl_xor_sync(0xffffffffu, nbs, d);
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, mx, d);
                if (o > mx) mx = o;
            }
            if (lane == leader) {
                atomicAdd(&s_hist[bb], (unsigned long long)__popc(m));
                atomicMax(&s_max[bb], mx);
                if (sm) atomicAdd(&s_binprod[bb], sm);
                if (nbs) atomicAdd(&s_binb[bb], nbs);
            }
            pending &= ~m;
        }
        __syncwarp();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) Ccp[0] = 0;
    for (int d = 16; d > 0; d >>= 1) {
        mine += __shfl_xor_sync(0xffffffffu, mine, d);
        cap += __shfl_xor_sync(0xffffffffu, cap, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_prod, mine);
        atomicAdd(&s_cap, cap);
    }
    __syncthreads();
    if (threadIdx.x < NBINS && s_hist[threadIdx.x]) {
        atomicAdd(&ctrl->hist[threadIdx.x], s_hist[threadIdx.x]);
        atomicMax(&ctrl->maxop[threadIdx.x], s_max[threadIdx.x]);
        atomicAdd(&ctrl->binprod[threadIdx.x], s_binprod[threadIdx.x]);
        atomicAdd(&ctrl->binnnzb[threadIdx.x], s_binb[threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&ctrl->products, s_prod);
        atomicAdd(&ctrl->capsum, s_cap);
    }
}

int64_t column_deal_mult(int64_t n) {
    if (n <= 2) return 1;
    auto gcd = [](int64_t a, int64_t b) {
        while (b) {
            const int64_t r = a % b;
            a = b;
            b = r;
        }
        return a;
    };
    int64_t m = (int64_t)((double)n * 0.6180339887498949);
    if (m < 1) m = 1;
    while (gcd(m, n) != 1) ++m;
    return m % n == 0 ? 1 : m;
}

// Single pass: slot capacity min(Op_j, rows) of every column, written to
// caps[j] (caps = the slot offsets + 1, scanned afterwards).
__global__ void k_slot_caps(const int64_t *__restrict__ op, int64_t nB, int64_t mrows, int64_t *__restrict__ caps) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nB; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = op[j];
        caps[j] = v < mrows ? v : mrows;
    }
}

// Single pass: every entry of C from its column's slot to its place in C.
// The positions of C are cut into tiles of kCopyTile entries, each copied by
// one CTA with coalesced stores, so a column of any length is spread over
// as many CTAs as its tiles (a warp per column left the longest columns of
// a power-law matrix to single warps).  k_tile_cols records the column
// holding each tile's first position; k_tile_copy then takes the tile's
// columns 256 at a time (their first positions and slot offsets staged in
// shared memory), and every thread finds its positions' columns by a binary
// search there.
constexpr int64_t kCopyTile = 4096;
constexpr int kCopyThreads = 256;

__global__ void k_tile_cols(int64_t nB, const int64_t *__restrict__ Ccp, int32_t *__restrict__ tile_col) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nB; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c0 = Ccp[j], c1 = Ccp[j + 1];
        for (int64_t k = (c0 + kCopyTile - 1) / kCopyTile; k * kCopyTile < c1; ++k) tile_col[k] = (int32_t)j;
    }
}

template <typename W>
__global__ void __launch_bounds__(kCopyThreads) k_tile_copy(int64_t nB, int64_t nnzC, const int64_t *__restrict__ Ccp,
                                                           const int64_t *__restrict__ soff,
                                                           const int32_t *__restrict__ tile_col,
                                                           const int32_t *__restrict__ srow,
                                                           const W *__restrict__ sval, int32_t *__restrict__ Crow,
                                                           W *__restrict__ Cval) {
    __shared__ int64_t s_c[kCopyThreads + 1];  // first positions in C of the group's columns, then its end
    __shared__ int64_t s_s[kCopyThreads + 1];  // their slot offsets (slot of column i: [s_s[i], s_s[i + 1]))
    for (int64_t k = blockIdx.x; k * kCopyTile < nnzC; k += gridDim.x) {
        const int64_t p_lo = k * kCopyTile;
        const int64_t p_hi = p_lo + kCopyTile < nnzC ? p_lo + kCopyTile : nnzC;
        int64_t jg = tile_col[k];
        for (;;) {
            const int G = (int)(nB - jg < kCopyThreads ? nB - jg : kCopyThreads);
            if (threadIdx.x < G) {
                s_c[threadIdx.x] = Ccp[jg + threadIdx.x];
                s_s[threadIdx.x] = soff[jg + threadIdx.x];
            }
            if (threadIdx.x == 0) {  // the group's end (jg + G <= nB)
                s_c[G] = Ccp[jg + G];
                s_s[G] = soff[jg + G];
            }
            __syncthreads();
            const int64_t g_lo = p_lo > s_c[0] ? p_lo : s_c[0];
            const int64_t g_hi = p_hi < s_c[G] ? p_hi : s_c[G];
            // every position of the tile in the group's first column (a long
            // column): no search
            const bool one = G == 1 || s_c[1] >= g_hi;
            for (int64_t p0 = g_lo; p0 < g_hi; p0 += 4 * kCopyThreads) {
                int32_t r[4];
                W v[4];
                int64_t dst[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t p = p0 + u * kCopyThreads + threadIdx.x;
                    dst[u] = -1;
                    if (p < g_hi) {
                        // the last column starting at or before p (s_c[0] <= p < s_c[G]): it holds p
                        int lo = 0, hi = one ? 0 : G - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_c[mid] <= p) lo = mid; else hi = mid - 1;
                        }
                        const int64_t off = p - s_c[lo];
                        // a count never exceeds its slot; reads stay inside the slots
                        if (off < s_s[lo + 1] - s_s[lo]) {
                            r[u] = srow[s_s[lo] + off];
                            v[u] = sval[s_s[lo] + off];
                            dst[u] = p;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (dst[u] >= 0) {
                        Crow[dst[u]] = r[u];
                        Cval[dst[u]] = v[u];
                    }
            }
            const bool more = s_c[G] < p_hi;  // uniform over the CTA
            __syncthreads();
            if (!more) break;
            jg += G;
        }
    }
}

cudaError_t launch_slot_copy(int64_t nB, int64_t nnzC, const int64_t *Ccp, const int64_t *soff, int32_t *tile_col,
                             const int32_t *srow, const void *sval, int32_t *Crow, void *Cval, int w, int sms,
                             cudaStream_t s) {
    if (nB <= 0 || nnzC <= 0) return cudaSuccess;
    const int gc = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nB, 256), 8 * (int64_t)sms));
    k_tile_cols<<<gc, 256, 0, s>>>(nB, Ccp, tile_col);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nnzC, kCopyTile), 8 * (int64_t)sms));
    if (w == 8)
        k_tile_copy<uint64_t><<<g, kCopyThreads, 0, s>>>(nB, nnzC, Ccp, soff, tile_col, srow,
                                                         static_cast<const uint64_t *>(sval), Crow,
                                                         static_cast<uint64_t *>(Cval));
    else
        k_tile_copy<uint32_t><<<g, kCopyThreads, 0, s>>>(nB, nnzC, Ccp, soff, tile_col, srow,
                                                         static_cast<const uint32_t *>(sval), Crow,
                                                         static_cast<uint32_t *>(Cval));
    return cudaGetLastError();
}

int64_t copy_tile_count(int64_t n) { return n / kCopyTile + 2; }

// Column ids into per-bin lists at off[bin] (each block reserves its slots
// with one global atomic per bin, so columns of a bin stay roughly in
// ascending order within a block's tile).
__global__ void k_bin_scatter(const int64_t *__restrict__ op, int64_t nB, int64_t t, int64_t hmax, int promote,
                              BinOffsets off, int32_t *__restrict__ bin_cols, Ctrl *ctrl) {
    __shared__ unsigned int s_cnt[NBINS];
    __shared__ unsigned long long s_base[NBINS];
    if (threadIdx.x < NBINS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    unsigned r = 0;
    if (j < nB) {
        b = bin_of(op[j], t, hmax, promote);
        if (b != BIN_EMPTY) r = atomicAdd(&s_cnt[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NBINS && s_cnt[threadIdx.x])
        s_base[threadIdx.x] = atomicAdd(&ctrl->fill[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
    __syncthreads();
    if (b > BIN_EMPTY) bin_cols[off.v[b] + (int64_t)s_base[b] + r] = (int32_t)j;
}

// ----------------------------------------------------------- int64 scan
// Inclusive scan of x[0..n) in place, in three passes over tiles of
// kScanTile elements: tile sums, a scan of the tile sums, the tiles.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_incl_scan_i64(int64_t v, int64_t *s_warp, int64_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[nw - 1];
    int64_t r = v + (warp > 0 ? s_warp[warp - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const int64_t *__restrict__ x, int64_t n, int64_t *__restrict__ sums) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t e = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (e < n) s += x[e];
    }
    int64_t total;
    block_incl_scan_i64(s, s_warp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int64_t *sums, int64_t ntiles) {
    __shared__ int64_t s_warp[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t e = base + threadIdx.x;
        int64_t v = e < ntiles ? sums[e] : 0;
        int64_t total;
        int64_t incl = block_incl_scan_i64(v, s_warp, total);
        if (e < ntiles) sums[e] = carry + incl - v;  // exclusive
        carry += total;
    }
}

__global__ void k_scan_apply(int64_t *__restrict__ x, int64_t n, const int64_t *__restrict__ sums) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t e = base + i;
        v[i] = e < n ? x[e] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t incl = block_incl_scan_i64(s, s_warp, total);
    int64_t run = sums[blockIdx.x] + incl - s;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t e = base + i;
        run += v[i];
        if (e < n) x[e] = run;
    }
}

cudaError_t launch_inclusive_scan(int64_t *x, int64_t n, int64_t *tile_sums, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t ntiles = ceil_div(n, kScanTile);
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(x, n, tile_sums);
    k_scan_sums<<<1, 1024, 0, s>>>(tile_sums, ntiles);
    k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, s>>>(x, n, tile_sums);
    return cudaGetLastError();
}

int64_t scan_tile_count(int64_t n) { return n <= 0 ? 1 : ceil_div(n, kScanTile); }



// ------------------------------------------------------- row compaction
__global__ void k_row_mark(const int32_t *Arow, int64_t nnz, int64_t m, int64_t *mark) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = Arow[i];
        if (r >= 0 && r < m) mark[r] = 1;
    }
}

__global__ void k_row_map(const int64_t *incl, int64_t m, int32_t *map, int32_t *inv) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t before = r > 0 ? incl[r - 1] : 0;
        if (incl[r] != before) {
            map[r] = (int32_t)before;
            inv[before] = (int32_t)r;
        } else {
            map[r] = -1;
        }
    }
}

__global__ void k_row_remap(const int32_t *Arow, int64_t nnz, const int32_t *map, int64_t m, int32_t *out,
                            Ctrl *ctrl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = Arow[i];
        int32_t c = r >= 0 && r < m ? map[r] : -1;
        if (c < 0) {
            set_error(ctrl, SPG_ERR_INVALID, kDetailRowMap, i);
            c = 0;
        }
        out[i] = c;
    }
}

// ------------------------------------------------------------ readback
namespace {

__global__ void k_readback(const unsigned char *s0, size_t n0, const unsigned char *s1, size_t n1,
                           unsigned char *dst, size_t off1) {
    for (size_t i = threadIdx.x; i < n0; i += blockDim.x) dst[i] = s0[i];
    for (size_t i = threadIdx.x; i < n1; i += blockDim.x) dst[off1 + i] = s1[i];
}

constexpr int kMaxDevices = 64;
thread_local Mirror t_mirror[kMaxDevices];

}  // namespace

Mirror::~Mirror() {
    if (host) cudaFreeHost(host);
}

cudaError_t Mirror::reserve(size_t need) {
    if (cap >= need) return cudaSuccess;
    if (host) cudaFreeHost(host);
    host = dev = nullptr;
    cap = 0;
    const size_t want = need > (size_t(64) << 10) ? need : (size_t(64) << 10);
    cudaError_t e = cudaHostAlloc(&host, want, cudaHostAllocMapped);
    if (e != cudaSuccess) {
        host = nullptr;
        return e;
    }
    if ((e = cudaHostGetDevicePointer(&dev, host, 0)) != cudaSuccess) return e;
    cap = want;
    return cudaSuccess;
}

cudaError_t readback(Mirror *mp, void *dst0, const void *src0, size_t n0, void *dst1, const void *src1, size_t n1,
                     cudaStream_t s) {
    cudaError_t e;
    if (!mp) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        mp = &t_mirror[dev];
    }
    Mirror &m = *mp;
    const size_t off1 = (n0 + 15) & ~size_t(15);
    if ((e = m.reserve(off1 + n1)) != cudaSuccess) return e;
    k_readback<<<1, 256, 0, s>>>(static_cast<const unsigned char *>(src0), n0,
                                 static_cast<const unsigned char *>(src1), n1,
                                 static_cast<unsigned char *>(m.dev), off1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (n0) std::memcpy(dst0, m.host, n0);
    if (n1) std::memcpy(dst1, static_cast<unsigned char *>(m.host) + off1, n1);
    return cudaSuccess;
}

}  // namespace spg
