// CSC transpose: row k of M (m x n) becomes column k of M^T (n x m).  Data
// movement only; the Galerkin product P^T (A P) needs P^T as a CSC operand.
//
// Steps: count the entries of every row (atomics), scan into T's column
// pointers, scatter every entry (e, row r, column j) to a slot of column r
// claimed with an atomic cursor, then sort each output column by j so the
// result is deterministic (warp register sort up to 256 entries, CTA bitonic
// sort in shared memory up to 16384, in place in global memory beyond), and
// finally gather the values through the permutation.
#include "kernels.cuh"

namespace spg {

namespace {

constexpr int kTrSmemSort = 16384;

// Rows outside [0, m) are skipped by both the count and the scatter.
__global__ void k_tr_count(const int32_t *__restrict__ row, int64_t nnz, int64_t m, unsigned long long *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t r = row[e];
        if (r >= 0 && r < m) atomicAdd(&cnt[r], 1ULL);
    }
}

__global__ void k_tr_scatter(const int64_t *__restrict__ cp, const int32_t *__restrict__ row, int64_t ncols,
                             int64_t m, unsigned long long *cursor, int32_t *__restrict__ Trow,
                             int64_t *__restrict__ Tperm) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ncols; j += stride) {
        for (int64_t e = cp[j]; e < cp[j + 1]; ++e) {
            const int32_t r = row[e];
            if (r < 0 || r >= m) continue;
            const int64_t pos = (int64_t)atomicAdd(&cursor[r], 1ULL);
            Trow[pos] = (int32_t)j;
            Tperm[pos] = e;
        }
    }
}

// One warp per output column of at most 256 entries.
__global__ void k_tr_sort_warp(const int64_t *__restrict__ Tcp, int64_t ncolsT, int32_t *Trow, int64_t *Tperm) {
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= ncolsT) return;
    const int64_t b = Tcp[c], L = Tcp[c + 1] - b;
    if (L <= 1 || L > 256) return;
    int32_t key[8];
    int64_t val[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int e = r * 32 + lane;
        key[r] = e < L ? Trow[b + e] : 0x7fffffff;
        val[r] = e < L ? Tperm[b + e] : 0;
    }
    group_bitonic_sort<32, 8, int64_t>(0xffffffffu, key, val);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int e = r * 32 + lane;
        if (e < L) {
            Trow[b + e] = key[r];
            Tperm[b + e] = val[r];
        }
    }
}

// One CTA per output column of more than 256 entries: bitonic sort over the
// next power of two, in shared memory when it fits, else in place in `tmp`.
__global__ void k_tr_sort_cta(const int64_t *__restrict__ Tcp, int64_t ncolsT, int32_t *Trow, int64_t *Tperm,
                              int32_t *gkey, int64_t *gval) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int64_t c = blockIdx.x; c < ncolsT; c += gridDim.x) {
        const int64_t b = Tcp[c], L = Tcp[c + 1] - b;
        if (L <= 256) continue;
        int64_t N = 1;
        while (N < L) N <<= 1;
        const bool in_smem = N <= kTrSmemSort;
        // beyond shared memory, sort a padded copy in the scratch: column c
        // owns [2 b, 2 b + N) there, inside [2 b, 2 (b + L)) since N < 2 L
        int32_t *key = in_smem ? reinterpret_cast<int32_t *>(smem) : gkey + 2 * b;
        int64_t *val = in_smem ? reinterpret_cast<int64_t *>(smem + (size_t)kTrSmemSort * 4) : gval + 2 * b;
        for (int64_t e = threadIdx.x; e < N; e += blockDim.x) {
            key[e] = e < L ? Trow[b + e] : 0x7fffffff;
            val[e] = e < L ? Tperm[b + e] : 0;
        }
        __syncthreads();
        for (int64_t k = 2; k <= N; k <<= 1) {
            for (int64_t jj = k >> 1; jj > 0; jj >>= 1) {
                for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
                    const int64_t l = i ^ jj;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const int32_t ki = key[i], kl = key[l];
                        if (up ? ki > kl : ki < kl) {
                            key[i] = kl;
                            key[l] = ki;
                            const int64_t t = val[i];
                            val[i] = val[l];
                            val[l] = t;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int64_t e = threadIdx.x; e < L; e += blockDim.x) {
            Trow[b + e] = key[e];
            Tperm[b + e] = val[e];
        }
        __syncthreads();
    }
}

// T's values through the permutation, for the entries T actually holds.
template <typename VT>
__global__ void k_tr_gather(const int64_t *__restrict__ perm, const int64_t *__restrict__ Tcp, int64_t m,
                            const VT *__restrict__ src, VT *__restrict__ dst) {
    const int64_t n = Tcp[m];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) dst[e] = src[perm[e]];
}

// dst[i] = src[idx[i]] (gather) or dst[idx[i]] = src[i] (scatter).
template <typename VT>
__global__ void k_permute(const VT *__restrict__ src, const int64_t *__restrict__ idx, VT *__restrict__ dst,
                          int64_t n, int scatter) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (scatter) dst[idx[i]] = src[i];
        else dst[i] = src[idx[i]];
    }
}

struct TrLayout {
    size_t cnt = 0, tiles = 0, perm = 0, key = 0, val = 0, total = 0;
};

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

TrLayout tr_layout(const spg_csc *M) {
    TrLayout L;
    size_t off = 0;
    L.cnt = off; off = al256(off + (size_t)(M->nrows + 1) * 8);
    L.tiles = off; off = al256(off + (size_t)scan_tile_count(M->nrows) * 8);
    L.perm = off; off = al256(off + (size_t)M->nnz * 8);       // permutation when the caller passes none
    L.key = off; off = al256(off + (size_t)M->nnz * 2 * 4 + 64);  // padded sort copies of long columns
    L.val = off; off = al256(off + (size_t)M->nnz * 2 * 8 + 64);
    L.total = off;
    return L;
}

}  // namespace

}  // namespace spg

using namespace spg;

extern "C" {

spg_status spg_transpose_workspace_size(const spg_csc *M, size_t *bytes) {
    if (!M || !bytes || M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPG_ERR_INVALID;
    *bytes = tr_layout(M).total;
    return SPG_OK;
}

spg_status spg_csc_transpose(const spg_csc *M, int64_t *T_colptr, int32_t *T_rowidx, void *T_values, int64_t *perm,
                             void *workspace, size_t ws_bytes, spg_stream stream) {
    if (!M || !T_colptr || M->nrows < 0 || M->ncols < 0 || M->nnz < 0 || !M->colptr) return SPG_ERR_INVALID;
    if (M->nrows > INT32_MAX || M->ncols > INT32_MAX) return SPG_ERR_INDEX_OVERFLOW;
    if (M->nnz > 0 && (!M->rowidx || !T_rowidx || (T_values && !M->values))) return SPG_ERR_INVALID;
    if (M->dtype != SPG_F64 && M->dtype != SPG_F32) return SPG_ERR_INVALID;
    const TrLayout L = tr_layout(M);
    if (!workspace || ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return SPG_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(ws + L.cnt);
    int64_t *pm = perm ? perm : reinterpret_cast<int64_t *>(ws + L.perm);
    const int64_t m = M->nrows, nnz = M->nnz;
    if (cudaMemsetAsync(cnt, 0, (size_t)(m + 1) * 8, s) != cudaSuccess) return SPG_ERR_CUDA;
    if (cudaMemsetAsync(T_colptr, 0, sizeof(int64_t), s) != cudaSuccess) return SPG_ERR_CUDA;
    if (nnz > 0) {
        const int g = (int)std::min<int64_t>(ceil_div(nnz, 256), 4096);
        k_tr_count<<<g, 256, 0, s>>>(M->rowidx, nnz, m, cnt);
    }
    if (m > 0) {
        if (cudaMemcpyAsync(T_colptr + 1, cnt, (size_t)m * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SPG_ERR_CUDA;
        if (launch_inclusive_scan(T_colptr + 1, m, reinterpret_cast<int64_t *>(ws + L.tiles), s) != cudaSuccess)
            return SPG_ERR_CUDA;
        // cursors start at the column starts
        if (cudaMemcpyAsync(cnt, T_colptr, (size_t)m * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return SPG_ERR_CUDA;
    }
    if (nnz > 0) {
        const int gc = (int)std::min<int64_t>(ceil_div(M->ncols, 256), 4096);
        k_tr_scatter<<<gc, 256, 0, s>>>(M->colptr, M->rowidx, M->ncols, m, cnt, T_rowidx, pm);
        k_tr_sort_warp<<<(unsigned)ceil_div(m * 32, 256), 256, 0, s>>>(T_colptr, m, T_rowidx, pm);
        const size_t smem = (size_t)kTrSmemSort * 12;
        cudaFuncSetAttribute(k_tr_sort_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tr_sort_cta<<<(unsigned)std::min<int64_t>(std::max<int64_t>(m, 1), 1024), 512, smem, s>>>(
            T_colptr, m, T_rowidx, pm, reinterpret_cast<int32_t *>(ws + L.key),
            reinterpret_cast<int64_t *>(ws + L.val));
        if (T_values) {
            const int gg = (int)std::min<int64_t>(ceil_div(nnz, 256), 4096);
            if (M->dtype == SPG_F64)
                k_tr_gather<double><<<gg, 256, 0, s>>>(pm, T_colptr, m, static_cast<const double *>(M->values),
                                                       static_cast<double *>(T_values));
            else
                k_tr_gather<float><<<gg, 256, 0, s>>>(pm, T_colptr, m, static_cast<const float *>(M->values),
                                                      static_cast<float *>(T_values));
        }
    }
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

spg_status spg_permute_values(const void *src, const int64_t *idx, void *dst, int64_t n, int32_t dtype,
                              int32_t scatter, spg_stream stream) {
    if (n < 0 || (dtype != SPG_F64 && dtype != SPG_F32)) return SPG_ERR_INVALID;
    if (n == 0) return SPG_OK;
    if (!src || !idx || !dst) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int g = (int)std::min<int64_t>(ceil_div(n, 256), 8192);
    if (dtype == SPG_F64)
        k_permute<double><<<g, 256, 0, s>>>(static_cast<const double *>(src), idx, static_cast<double *>(dst), n,
                                            scatter);
    else
        k_permute<float><<<g, 256, 0, s>>>(static_cast<const float *>(src), idx, static_cast<float *>(dst), n,
                                           scatter);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

}  // extern "C"
