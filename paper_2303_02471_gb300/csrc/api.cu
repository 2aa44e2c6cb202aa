// Host side of the C ABI (include/spgemm.h): argument checks, workspace
// layout, plan object, and the launch sequence of the symbolic, numeric and
// backward phases.  No device memory is allocated here: everything lives in
// the caller's workspace and output buffers.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "esc.cuh"
#include "handle.cuh"

using namespace spg;

namespace {

struct DeviceInfo {
    int sms = 0;
    size_t smem_optin = 0;
};

DeviceInfo device_info(int dev) {
    static std::mutex mu;
    static DeviceInfo cache[64];
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return DeviceInfo{};
    if (cache[dev].sms == 0) {
        int sms = 0, optin = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cache[dev].sms = sms > 0 ? sms : 1;
        // keep a little room for the kernels' static shared memory
        cache[dev].smem_optin = optin > 4096 ? (size_t)optin - 1024 : 48 * 1024;
    }
    return cache[dev];
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t ctrl = 0, op = 0, cols = 0, tiles = 0, scratch = 0, cache = 0, total = 0;
    size_t rmark = 0, rtiles = 0, rmap = 0, rinv = 0, arow = 0;
    size_t scratch_stride = 0;
    int64_t scratch_ctas = 0;
    int64_t cache_cols = 0;
    size_t cache_bytes = 0;
};

spg_config normalized(const spg_config *cfg) {
    spg_config c;
    spg_config_default(&c);
    if (cfg) c = *cfg;
    return c;
}

// Default threshold: the dense SPA pays O(m / 32) words per column (flag
// bitmap prefix and sorted extraction), so a column goes dense once its
// product count reaches m / 512 (the crossover measured on GB300), within
// [257, hash_cta_max + 1]; m counts the rows the forward passes number.
int64_t effective_t(const spg_config &c, int64_t m) {
    if (c.t >= 0) return c.t;
    int64_t t = (m + 511) / 512;
    if (t > (int64_t)c.hash_cta_max + 1) t = (int64_t)c.hash_cta_max + 1;
    if (t < 257) t = 257;
    return t;
}

bool valid_hash_max(int32_t h) {
    return h == 256 || h == 512 || h == 1024 || h == 2048 || h == 4096 || h == 8192;
}

Layout make_layout(int64_t m, int64_t nB, int64_t nnzA, int dtype, const spg_config &c, int sms) {
    Layout L;
    const size_t w = dtype == SPG_F64 ? 8 : 4;
    const int64_t W = ceil_div(m, 32);
    const int64_t hmax = c.hash_cta_max;
    size_t off = 0;
    L.ctrl = off; off = align256(off + sizeof(Ctrl));
    L.op = off; off = align256(off + (size_t)nB * 8);
    L.cols = off; off = align256(off + (size_t)nB * 4);
    L.tiles = off; off = align256(off + (size_t)scan_tile_count(nB) * 8);
    // row compaction: marks (scanned in place), the map to compact rows and
    // back, and A's rows renumbered
    L.rmark = off; off = align256(off + (size_t)m * 8);
    L.rtiles = off; off = align256(off + (size_t)scan_tile_count(m) * 8);
    L.rmap = off; off = align256(off + (size_t)m * 4);
    L.rinv = off; off = align256(off + (size_t)m * 4);
    L.arow = off; off = align256(off + (size_t)nnzA * 4);
    // per-CTA global scratch: a bitmap (uint2 per 32 rows) plus, for hash
    // tables that do not fit shared memory, keys and values
    const int64_t reach = std::min<int64_t>(std::max<int64_t>(nnzA, 1), std::max<int64_t>(m, 1));
    // hash table keys + values + word list of the extraction (numeric)
    size_t tab = (size_t)num_slots(std::min<int64_t>(hmax, reach), c.table_slots_pct) * (8 + w) + 64;
    if (effective_t(c, m) > hmax + 1) {
        const size_t sym = (size_t)global_sym_slots(reach, m) * 4;
        const size_t num = (size_t)num_slots(reach, c.table_slots_pct) * (8 + w) + 64;
        tab = std::max(tab, std::max(sym, num));
    }
    L.scratch_stride = align256((size_t)W * 8) + align256(tab);
    int64_t ctas = 2 * (int64_t)sms;
    if (c.scratch_cap_bytes > 0) {
        int64_t fit = c.scratch_cap_bytes / (int64_t)L.scratch_stride;
        if (fit < ctas) ctas = fit;
    }
    if (ctas < 1) ctas = 1;
    L.scratch_ctas = ctas;
    L.scratch = off;
    off = align256(off + (size_t)ctas * L.scratch_stride);
    // SPA flag bitmaps of dense columns, kept from the symbolic phase
    L.cache = off;
    if (c.dense_cache_bytes > 0 && W > 0) {
        L.cache_cols = std::min<int64_t>(nB, c.dense_cache_bytes / (W * 4));
        L.cache_bytes = (size_t)L.cache_cols * (size_t)W * 4;
        off = align256(off + L.cache_bytes);
    }
    L.total = off;
    return L;
}

spg_status check_csc(const spg_csc *M, bool need_values) {
    if (!M) return SPG_ERR_INVALID;
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPG_ERR_INVALID;
    if (M->nrows > INT32_MAX || M->ncols > INT32_MAX) return SPG_ERR_INDEX_OVERFLOW;
    if (M->dtype != SPG_F64 && M->dtype != SPG_F32) return SPG_ERR_INVALID;
    if (!M->colptr) return SPG_ERR_INVALID;
    if (M->nnz > 0 && (!M->rowidx || (need_values && !M->values))) return SPG_ERR_INVALID;
    return SPG_OK;
}

spg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SPG_OK : SPG_ERR_CUDA; }

}  // namespace

struct spg_plan {
    int device = 0;
    DeviceInfo dev;
    int64_t mA = 0, nA = 0, nB = 0, nnzA = 0, nnzB = 0;
    // rows of the forward pass: A's rows renumbered over the rows that hold
    // entries (mC of them) when that saves at least a tenth of the rows
    bool compact = false;
    int64_t mC = 0;
    int dtype = 0;
    spg_config cfg{};
    int64_t t_eff = 0;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    Layout L;
    Ctrl host{};
    BinOffsets off{};
    int64_t nnzC = 0;
    Geo num_geo[NBINS];
    bool num_geo_ready = false;
    Geo bwd_geo[NBINS];
    bool bwd_geo_ready = false;
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev0[NBINS] = {}, ev1[NBINS] = {};
    int64_t sym_launches = 0;
    // the lane-group bins run on side streams, forked from and joined back
    // to the caller's stream: the handle's, or (no handle) the plan's own,
    // created on first use
    spg_handle *h = nullptr;
    SideStreams own;
    // lane-group bins worked by the ESC accumulator (and their tile shapes)
    bool esc[NBINS] = {};
    EscShape esc_shape_of[NBINS];
    // single pass: the columns' slots (offsets, rows, values) after the
    // regular layout, sum of the slot sizes
    bool single = false;
    size_t soff_at = 0, srow_at = 0, sval_at = 0, tcol_at = 0, slots_total = 0;
    int64_t capsum = 0;

    ~spg_plan() {
        for (int b = 0; b < NBINS; ++b) {
            if (ev0[b]) cudaEventDestroy(ev0[b]);
            if (ev1[b]) cudaEventDestroy(ev1[b]);
        }
        own.release();
    }
    SideStreams &ss() { return h ? h->streams : own; }
    bool side_streams() { return ss().ready() || ss().create(); }
    cudaError_t read(void *dst0, const void *src0, size_t n0, void *dst1, const void *src1, size_t n1,
                     cudaStream_t s) {
        return handle_readback(h, dst0, src0, n0, dst1, src1, n1, s);
    }
    int64_t nonempty_bins() const {
        int64_t n = 0;
        for (int b = 1; b < NBINS; ++b) n += host.hist[b] ? 1 : 0;
        return n;
    }

    Ctrl *ctrl() const { return reinterpret_cast<Ctrl *>(ws + L.ctrl); }
    int64_t *op() const { return reinterpret_cast<int64_t *>(ws + L.op); }
    int32_t *cols() const { return reinterpret_cast<int32_t *>(ws + L.cols); }
    int64_t *tiles() const { return reinterpret_cast<int64_t *>(ws + L.tiles); }
    unsigned char *scratch() const { return ws + L.scratch; }
    int64_t *rmark() const { return reinterpret_cast<int64_t *>(ws + L.rmark); }
    int32_t *rmap() const { return reinterpret_cast<int32_t *>(ws + L.rmap); }
    int32_t *rinv() const { return reinterpret_cast<int32_t *>(ws + L.rinv); }
    int32_t *arow() const { return reinterpret_cast<int32_t *>(ws + L.arow); }

    // fwd: the symbolic and numeric passes (compact rows when `compact`);
    // otherwise the backward, which works on C's own rows
    BinTask task(int b, bool fwd = true) const {
        BinTask t;
        t.cols = cols() + off.v[b];
        t.count = (int64_t)host.hist[b];
        t.bin = b;
        t.shrink = cfg.table_shrink;
        t.slots_pct = cfg.table_slots_pct;
        t.m = fwd ? mC : mA;
        t.W = ceil_div(t.m, 32);
        t.op = op();
        t.scratch = scratch();
        t.scratch_stride = L.scratch_stride;
        t.ctrl = ctrl();
        t.flag_cache = b == BIN_DENSE ? reinterpret_cast<uint32_t *>(ws + L.cache) : nullptr;
        // the cache region holds more columns of the shorter compact flags
        t.cache_cols = b == BIN_DENSE && fwd && t.W > 0
                           ? std::min<int64_t>(nB, (int64_t)(L.cache_bytes / ((size_t)t.W * 4)))
                           : 0;
        t.wait_cycles = cfg.test_wait_timeout ? 0 : kBulkWaitCycles;
        return t;
    }

    // The bins write disjoint columns of C.  Next to a dense bin, the bins
    // that use no workspace scratch (the lane-group bins, and CTA hash bins
    // whose table and flags fit shared memory) run on side streams: the
    // dense kernel is launched first and keeps every SM, the others fill SMs
    // as its CTAs finish and overlap one another.
    bool side_rule(int b) const {
        if (b >= BIN_WARP0 && b < BIN_CTA0) return true;
        return b >= BIN_CTA0 && b < BIN_GLOBAL && num_geo[b].cap == 0 && !num_geo[b].bm_global;
    }
    bool numeric_fork() const {
        if (!cfg.side_streams || !host.hist[BIN_DENSE]) return false;
        for (int b = 1; b < BIN_DENSE; ++b)
            if (host.hist[b] && side_rule(b)) return true;
        return false;
    }
};

extern "C" {

spg_status spg_config_default(spg_config *cfg) {
    if (!cfg) return SPG_ERR_INVALID;
    cfg->t = -1;
    cfg->hash_cta_max = 8192;
    cfg->cta_threads = 1024;
    cfg->validate = 1;
    cfg->table_shrink = 0;
    cfg->scratch_cap_bytes = (int64_t)1 << 30;
    cfg->dense_cache_bytes = (int64_t)2 << 30;
    cfg->side_streams = 1;
    cfg->test_wait_timeout = 0;
    cfg->small_accumulator = SPG_ACC_AUTO;
    cfg->table_slots_pct = kDefaultSlotsPct;
    cfg->group_promote = 0;
    return SPG_OK;
}

const char *spg_status_string(spg_status s) {
    switch (s) {
        case SPG_OK: return "SPG_OK";
        case SPG_ERR_INVALID: return "SPG_ERR_INVALID: bad argument or malformed CSC input";
        case SPG_ERR_WORKSPACE: return "SPG_ERR_WORKSPACE: workspace missing or too small";
        case SPG_ERR_TABLE_OVERFLOW: return "SPG_ERR_TABLE_OVERFLOW: a hash table ran out of slots";
        case SPG_ERR_TIMEOUT: return "SPG_ERR_TIMEOUT: a bounded device loop hit its limit";
        case SPG_ERR_CUDA: return "SPG_ERR_CUDA: a CUDA runtime call failed";
        case SPG_ERR_UNSUPPORTED: return "SPG_ERR_UNSUPPORTED: shape or option not supported";
        case SPG_ERR_INDEX_OVERFLOW: return "SPG_ERR_INDEX_OVERFLOW: a size exceeds the index types";
    }
    return "SPG_ERR_UNKNOWN";
}

static spg_status check_pair(const spg_csc *A, const spg_csc *B, bool values) {
    spg_status s = check_csc(A, values);
    if (s != SPG_OK) return s;
    s = check_csc(B, values);
    if (s != SPG_OK) return s;
    if (A->ncols != B->nrows || A->dtype != B->dtype) return SPG_ERR_INVALID;
    return SPG_OK;
}

static spg_status check_config(const spg_config &c) {
    if (!valid_hash_max(c.hash_cta_max)) return SPG_ERR_INVALID;
    if (c.cta_threads < 128 || c.cta_threads > 1024 || c.cta_threads % 32) return SPG_ERR_INVALID;
    if (c.table_shrink < 0 || c.table_shrink > 30) return SPG_ERR_INVALID;
    if (c.dense_cache_bytes < 0 || c.scratch_cap_bytes < 0) return SPG_ERR_INVALID;
    if (c.small_accumulator != SPG_ACC_HASH && c.small_accumulator != SPG_ACC_ESC &&
        c.small_accumulator != SPG_ACC_AUTO)
        return SPG_ERR_INVALID;
    if (c.table_slots_pct < 125 || c.table_slots_pct > 400) return SPG_ERR_INVALID;
    if (c.group_promote < 0 || c.group_promote > 2) return SPG_ERR_INVALID;
    return SPG_OK;
}

spg_status spgemm_workspace_size(const spg_csc *A, const spg_csc *B, const spg_config *cfg, size_t *bytes) {
    if (!bytes) return SPG_ERR_INVALID;
    spg_status s = check_pair(A, B, false);
    if (s != SPG_OK) return s;
    spg_config c = normalized(cfg);
    if ((s = check_config(c)) != SPG_OK) return s;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPG_ERR_CUDA;
    DeviceInfo di = device_info(dev);
    *bytes = make_layout(A->nrows, B->ncols, A->nnz, A->dtype, c, di.sms).total;
    return SPG_OK;
}

spg_status spg_create(spg_handle **handle) {
    if (!handle) return SPG_ERR_INVALID;
    *handle = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPG_ERR_CUDA;
    spg_handle *h = new (std::nothrow) spg_handle();
    if (!h) return SPG_ERR_INVALID;
    h->device = dev;
    if (!h->streams.create() || h->mirror.reserve(0) != cudaSuccess) {
        delete h;
        return SPG_ERR_CUDA;
    }
    *handle = h;
    return SPG_OK;
}

spg_status spg_destroy(spg_handle *handle) {
    delete handle;
    return SPG_OK;
}

// Slots of the single pass after the regular layout: offsets int64[nB + 1],
// rows int32[capsum], values[capsum], and the copy's first column of every
// tile of C's positions (nnz(C) <= capsum).
static void slot_layout(spg_plan *P) {
    const size_t w = P->dtype == SPG_F64 ? 8 : 4;
    size_t off = align256(P->L.total);
    P->soff_at = off;
    off = align256(off + (size_t)(P->nB + 1) * 8);
    P->srow_at = off;
    off = align256(off + (size_t)P->capsum * 4);
    P->sval_at = off;
    off = align256(off + (size_t)P->capsum * w);
    P->tcol_at = off;
    off = align256(off + (size_t)copy_tile_count(P->capsum) * 4);
    P->slots_total = off;
}

// Everything before the accumulators, shared by the symbolic phase and the
// single pass: a new plan over `workspace`, input validation, row
// compaction, Op_j and bins (Sections 3.1-3.3) and, with `scatter`, the
// per-bin column lists.  On success *out holds the plan; on error it is
// deleted.
static spg_status prepare(spg_handle *handle, const spg_csc *A, const spg_csc *B, const spg_config &c,
                          void *workspace, size_t ws_bytes, int64_t *C_colptr, cudaStream_t s, bool scatter,
                          spg_plan **out) {
    *out = nullptr;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return SPG_ERR_WORKSPACE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPG_ERR_CUDA;
    if (handle && handle->device != dev) return SPG_ERR_INVALID;
    spg_plan *P = new (std::nothrow) spg_plan();
    if (!P) return SPG_ERR_INVALID;
    P->h = handle;
    P->device = dev;
    P->dev = device_info(dev);
    P->mA = A->nrows; P->nA = A->ncols; P->nB = B->ncols;
    P->nnzA = A->nnz; P->nnzB = B->nnz;
    P->dtype = A->dtype;
    P->cfg = c;
    P->L = make_layout(P->mA, P->nB, P->nnzA, P->dtype, c, P->dev.sms);
    if (ws_bytes < P->L.total) { delete P; return SPG_ERR_WORKSPACE; }
    P->ws = static_cast<unsigned char *>(workspace);
    P->ws_bytes = ws_bytes;
    const int64_t hmax = c.hash_cta_max;
    Ctrl *ctrl = P->ctrl();
    spg_status st;

#define CK(expr)                                                      \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) { delete P; return SPG_ERR_CUDA; }     \
    } while (0)

    CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s));
    if (c.validate) {
        const int vg = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max(A->nnz, A->ncols + 1), 256), 8 * P->dev.sms));
        k_validate<<<vg, 256, 0, s>>>(A->colptr, A->rowidx, A->nrows, A->ncols, A->nnz, 0, ctrl);
        const int vb = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max(B->nnz, B->ncols + 1), 256), 8 * P->dev.sms));
        k_validate<<<vb, 256, 0, s>>>(B->colptr, B->rowidx, B->nrows, B->ncols, B->nnz, 1, ctrl);
        CK(cudaGetLastError());
    }
    // Row compaction of the forward passes (bounds-checked, so it may run
    // before the validation outcome): a row of A without entries has none in
    // C, and the dense flags, their cache and the CTA bitmaps then span only
    // the rows that hold entries.
    int64_t mC = P->mA;
    const bool try_compact = P->mA > 0 && P->nnzA > 0;
    if (try_compact) {
        CK(cudaMemsetAsync(P->rmark(), 0, (size_t)P->mA * 8, s));
        const int ga = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(A->nnz, 256), 8 * P->dev.sms));
        k_row_mark<<<ga, 256, 0, s>>>(A->rowidx, A->nnz, P->mA, P->rmark());
        CK(cudaGetLastError());
        CK(launch_inclusive_scan(P->rmark(), P->mA, reinterpret_cast<int64_t *>(P->ws + P->L.rtiles), s));
    }
    // one read: the validation outcome (a malformed colptr would make the
    // walks read out of bounds: stop here) and the count of rows with entries
    CK(P->read(&P->host, ctrl, sizeof(Ctrl), try_compact ? &mC : nullptr,
               try_compact ? P->rmark() + (P->mA - 1) : nullptr, try_compact ? sizeof(int64_t) : 0, s));
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    P->compact = try_compact && mC > 0 && mC * 10 <= P->mA * 9;
    P->mC = P->compact ? mC : P->mA;
    if (P->compact) {
        // the map to compact rows and back, and A's rows renumbered (rows
        // out of range were rejected by the validation, or are reported here)
        const int ga = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(A->nnz, 256), 8 * P->dev.sms));
        const int gm = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(P->mA, 256), 8 * P->dev.sms));
        k_row_map<<<gm, 256, 0, s>>>(P->rmark(), P->mA, P->rmap(), P->rinv());
        k_row_remap<<<ga, 256, 0, s>>>(A->rowidx, A->nnz, P->rmap(), P->mA, P->arow(), ctrl);
        CK(cudaGetLastError());
    }
    P->t_eff = effective_t(c, P->mC);
    if (P->nB > 0) {
        // a warp per 32 columns, 8 warps per CTA
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(P->nB, 256), 16 * (int64_t)P->dev.sms));
        k_count_bin<<<g, 256, 0, s>>>(B->colptr, B->rowidx, A->colptr, P->nB, P->t_eff, hmax, c.group_promote, P->mC,
                                      column_deal_mult(P->nB), P->op(), C_colptr, ctrl);
        CK(cudaGetLastError());
    } else {
        CK(cudaMemsetAsync(C_colptr, 0, sizeof(int64_t), s));
    }
    CK(P->read(&P->host, ctrl, sizeof(Ctrl), nullptr, nullptr, 0, s));
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    // the walks index a column's products with 32-bit offsets
    for (int b = 0; b < NBINS; ++b)
        if (P->host.maxop[b] >= (1ULL << 31)) { delete P; return SPG_ERR_UNSUPPORTED; }
    P->capsum = (int64_t)P->host.capsum;
    P->off.v[0] = 0;
    for (int b = 0; b < NBINS; ++b) {
        // empty columns are not listed
        const int64_t n = b == BIN_EMPTY ? 0 : (int64_t)P->host.hist[b];
        P->off.v[b + 1] = P->off.v[b] + n;
    }
    if (scatter && P->nB > 0) {
        k_bin_scatter<<<(unsigned)ceil_div(P->nB, 256), 256, 0, s>>>(P->op(), P->nB, P->t_eff, hmax, c.group_promote,
                                                                     P->off, P->cols(), ctrl);
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(&ctrl->work, 0, sizeof(ctrl->work), s));
#undef CK
    // the numeric phase (and the single pass) take ESC unless hash tables
    // were asked for; the symbolic phase counts with ESC when asked, and by
    // default in the bins that ESC sorts by rank (sym_bin)
    if (c.small_accumulator != SPG_ACC_HASH)
        for (int b = BIN_WARP0; b < BIN_CTA0; ++b) P->esc[b] = esc_shape(b, P->mC, P->esc_shape_of[b]);
    // validation, row marks (mark, 3 scan kernels) and, when compacting,
    // map and remap, the two control reads, Op counting + scatter
    P->sym_launches = (c.validate ? 2 : 0) + (try_compact ? 4 : 0) + (P->compact ? 2 : 0) + 2 +
                      (P->nB > 0 ? 1 + (scatter ? 1 : 0) : 0);
    *out = P;
    return SPG_OK;
}

spg_status spgemm_symbolic(spg_handle *handle, const spg_csc *A, const spg_csc *B, const spg_config *cfg,
                           void *workspace, size_t ws_bytes, int64_t *C_colptr, int64_t *nnzC, spg_plan **plan_out,
                           spg_stream stream) {
    if (plan_out) *plan_out = nullptr;
    if (!C_colptr || !nnzC || !plan_out) return SPG_ERR_INVALID;
    spg_status st = check_pair(A, B, false);
    if (st != SPG_OK) return st;
    spg_config c = normalized(cfg);
    if ((st = check_config(c)) != SPG_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spg_plan *P = nullptr;
    if ((st = prepare(handle, A, B, c, workspace, ws_bytes, C_colptr, s, true, &P)) != SPG_OK) return st;
    Ctrl *ctrl = P->ctrl();

#define CK(expr)                                                      \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) { delete P; return SPG_ERR_CUDA; }     \
    } while (0)

    Operands o{A->colptr, P->compact ? P->arow() : A->rowidx, nullptr, B->colptr, B->rowidx, nullptr};
    // as in the numeric phase: beside a dense bin, the lane-group bins (shared
    // memory only) run on the side streams, launched after the dense kernel
    bool groups = false;
    for (int b = BIN_WARP0; b < BIN_CTA0; ++b) groups |= P->host.hist[b] != 0;
    const bool fork = groups && P->host.hist[BIN_DENSE] != 0 && c.side_streams;
    if (fork) {
        if (!P->side_streams()) { delete P; return SPG_ERR_CUDA; }
        CK(cudaEventRecord(P->ss().fork, s));
    }
    auto sym_bin = [&](int b, cudaStream_t sb) {
        // counting by rank (no sort, no compress) beat the hash tables on
        // GB300; counting through the radix sort did not
        const bool esc_counts = c.small_accumulator == SPG_ACC_ESC ||
                                (c.small_accumulator == SPG_ACC_AUTO && P->esc_shape_of[b].rank != kEscRadix);
        if (P->esc[b] && esc_counts)
            return launch_esc_bin(P->task(b), o, C_colptr, C_colptr, nullptr, nullptr, false, P->dtype,
                                  P->esc_shape_of[b], P->dev.sms, sb);
        // the symbolic CTA kernels carry no values: CTAs of up to 256 threads,
        // several per SM, overlap one another's barriers (measured faster)
        Geo g = symbolic_geometry(b, (int64_t)P->host.hist[b], P->mC, std::min(c.cta_threads, kSymCtaThreads),
                                  P->dev.sms, P->dev.smem_optin, (int64_t)P->host.maxop[b], c.table_shrink,
                                  P->L.scratch_ctas);
        return launch_symbolic_bin(P->task(b), o, C_colptr, g, sb);
    };
    {
        // once forked, the side streams are joined back to `stream` even when
        // a call fails, so a capture of `stream` is never left unjoined
        cudaError_t first = cudaSuccess;
        auto keep = [&](cudaError_t e) {
            if (first == cudaSuccess) first = e;
        };
        if (fork)
            for (int i = 0; i < kNumSideStreams; ++i) keep(cudaStreamWaitEvent(P->ss().side[i], P->ss().fork, 0));
        for (int b = 1; b < NBINS && first == cudaSuccess; ++b)
            if (P->host.hist[b] && !(fork && b >= BIN_WARP0 && b < BIN_CTA0)) keep(sym_bin(b, s));
        if (fork) {
            for (int b = BIN_CTA0 - 1, i = 0; b >= BIN_WARP0 && first == cudaSuccess; --b)
                if (P->host.hist[b]) keep(sym_bin(b, P->ss().side[i++ % kNumSideStreams]));
            for (int i = 0; i < kNumSideStreams; ++i) {
                keep(cudaEventRecord(P->ss().join[i], P->ss().side[i]));
                keep(cudaStreamWaitEvent(s, P->ss().join[i], 0));
            }
        }
        CK(first);
    }
    CK(launch_inclusive_scan(C_colptr + 1, P->nB, P->tiles(), s));
    CK(P->read(&P->nnzC, C_colptr + P->nB, sizeof(int64_t), &P->host, ctrl, sizeof(Ctrl), s));
#undef CK
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    for (int b = 1; b < NBINS; ++b) {
        if (!P->host.hist[b]) continue;
        P->num_geo[b] = numeric_geometry(b, (int64_t)P->host.hist[b], P->mC, c.cta_threads, P->dev.sms,
                                         P->dev.smem_optin, (int64_t)P->host.maxnnz[b], P->dtype, c.table_slots_pct,
                                         P->L.scratch_ctas);
    }
    P->num_geo_ready = true;
    // the preparation, 3 scan kernels, the control read, the bins
    P->sym_launches += 4 + P->nonempty_bins();
    *nnzC = P->nnzC;
    *plan_out = P;
    return SPG_OK;
}

static spg_status check_plan_operands(const spg_plan *P, const spg_csc *A, const spg_csc *B) {
    if (!P) return SPG_ERR_INVALID;
    spg_status st = check_pair(A, B, true);
    if (st != SPG_OK) return st;
    if (A->nrows != P->mA || A->ncols != P->nA || B->ncols != P->nB || A->nnz != P->nnzA || B->nnz != P->nnzB ||
        A->dtype != P->dtype)
        return SPG_ERR_INVALID;
    return SPG_OK;
}

// The accumulators of every bin on `s` (side streams forked and joined as
// the plan says): C's rows and values at base[j] + rank, the counts checked
// against base (two-pass) or written to cnt_out[j + 1] (single pass).
static spg_status run_numeric(spg_plan *P, const Operands &o, const int64_t *base, int64_t *cnt_out,
                              int32_t *rows, void *vals, cudaStream_t s) {
    auto on_side = [&](int b) { return P->side_rule(b); };
    const bool fork = P->numeric_fork();
    if (fork && !P->side_streams()) return SPG_ERR_CUDA;
    auto launch = [&](int b, cudaStream_t sb) -> spg_status {
        if (P->timing && cudaEventRecord(P->ev0[b], sb) != cudaSuccess) return SPG_ERR_CUDA;
        BinTask t = P->task(b);
        t.cnt_out = cnt_out;
        if (cnt_out) t.cache_cols = 0;  // no symbolic phase kept flags
        cudaError_t e = P->esc[b] ? launch_esc_bin(t, o, base, cnt_out, rows, vals, true, P->dtype,
                                                   P->esc_shape_of[b], P->dev.sms, sb)
                                  : launch_numeric_bin(t, o, base, rows, vals, P->dtype, P->num_geo[b], sb);
        if (e != cudaSuccess) return SPG_ERR_CUDA;
        if (P->timing && cudaEventRecord(P->ev1[b], sb) != cudaSuccess) return SPG_ERR_CUDA;
        return SPG_OK;
    };
    spg_status st;
    if (fork) {
        if (cudaEventRecord(P->ss().fork, s) != cudaSuccess) return SPG_ERR_CUDA;
        // from here on the side streams are joined back to `stream` whatever
        // fails, so a capture of `stream` is never left unjoined; the first
        // error is returned
        spg_status first = SPG_OK;
        auto keep = [&](spg_status x) {
            if (first == SPG_OK) first = x;
        };
        for (int i = 0; i < kNumSideStreams; ++i)
            if (cudaStreamWaitEvent(P->ss().side[i], P->ss().fork, 0) != cudaSuccess) keep(SPG_ERR_CUDA);
        for (int b = 1; b < NBINS && first == SPG_OK; ++b)
            if (P->host.hist[b] && !on_side(b)) keep(launch(b, s));
        // heaviest side bin first, bins dealt round-robin to the side streams
        for (int b = BIN_DENSE - 1, i = 0; b >= 1 && first == SPG_OK; --b)
            if (P->host.hist[b] && on_side(b)) keep(launch(b, P->ss().side[i++ % kNumSideStreams]));
        for (int i = 0; i < kNumSideStreams; ++i)
            if (cudaEventRecord(P->ss().join[i], P->ss().side[i]) != cudaSuccess ||
                cudaStreamWaitEvent(s, P->ss().join[i], 0) != cudaSuccess)
                keep(SPG_ERR_CUDA);
        if (first != SPG_OK) return first;
    } else {
        for (int b = 1; b < NBINS; ++b)
            if (P->host.hist[b] && (st = launch(b, s)) != SPG_OK) return st;
    }
    P->timed = P->timing;
    return SPG_OK;
}

spg_status spgemm_numeric(spg_plan *P, const spg_csc *A, const spg_csc *B, const int64_t *C_colptr,
                          int32_t *C_rowidx, void *C_values, spg_stream stream) {
    spg_status st = check_plan_operands(P, A, B);
    if (st != SPG_OK) return st;
    if (!C_colptr || (P->nnzC > 0 && (!C_rowidx || !C_values))) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ctrl *ctrl = P->ctrl();
    if (cudaMemsetAsync(&ctrl->work, 0, sizeof(ctrl->work), s) != cudaSuccess) return SPG_ERR_CUDA;
    if (P->compact && P->nnzA > 0) {
        // A's rows renumbered again from the A given here: an entry in a row
        // that held none at planning time is reported, not walked
        const int ga = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(A->nnz, 256), 8 * P->dev.sms));
        k_row_remap<<<ga, 256, 0, s>>>(A->rowidx, A->nnz, P->rmap(), P->mA, P->arow(), ctrl);
        if (cudaGetLastError() != cudaSuccess) return SPG_ERR_CUDA;
    }
    Operands o{A->colptr, P->compact ? P->arow() : A->rowidx, A->values, B->colptr, B->rowidx, B->values,
               P->compact ? P->rinv() : nullptr};
    return run_numeric(P, o, C_colptr, nullptr, C_rowidx, C_values, s);
}

spg_status spgemm_single_pass_size(spg_handle *handle, const spg_csc *A, const spg_csc *B, const spg_config *cfg,
                                   void *workspace, size_t ws_bytes, int64_t *C_colptr, size_t *bytes,
                                   spg_stream stream) {
    if (!bytes || !C_colptr) return SPG_ERR_INVALID;
    spg_status st = check_pair(A, B, false);
    if (st != SPG_OK) return st;
    spg_config c = normalized(cfg);
    if ((st = check_config(c)) != SPG_OK) return st;
    c.dense_cache_bytes = 0;  // nothing is kept between phases
    spg_plan *P = nullptr;
    if ((st = prepare(handle, A, B, c, workspace, ws_bytes, C_colptr, reinterpret_cast<cudaStream_t>(stream), false,
                      &P)) != SPG_OK)
        return st;
    slot_layout(P);
    *bytes = P->slots_total;
    delete P;
    return SPG_OK;
}

spg_status spgemm_single_pass(spg_handle *handle, const spg_csc *A, const spg_csc *B, const spg_config *cfg,
                              void *workspace, size_t ws_bytes, int64_t *C_colptr, int64_t *nnzC,
                              spg_plan **plan_out, spg_stream stream) {
    if (plan_out) *plan_out = nullptr;
    if (!C_colptr || !nnzC || !plan_out) return SPG_ERR_INVALID;
    spg_status st = check_pair(A, B, true);
    if (st != SPG_OK) return st;
    spg_config c = normalized(cfg);
    if ((st = check_config(c)) != SPG_OK) return st;
    c.dense_cache_bytes = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    spg_plan *P = nullptr;
    if ((st = prepare(handle, A, B, c, workspace, ws_bytes, C_colptr, s, true, &P)) != SPG_OK) return st;
    slot_layout(P);
    if (ws_bytes < P->slots_total) { delete P; return SPG_ERR_WORKSPACE; }
    P->single = true;
    Ctrl *ctrl = P->ctrl();
    int64_t *soff = reinterpret_cast<int64_t *>(P->ws + P->soff_at);

#define CK(expr)                                                      \
    do {                                                              \
        cudaError_t e_ = (expr);                                      \
        if (e_ != cudaSuccess) { delete P; return SPG_ERR_CUDA; }     \
    } while (0)

    // slot offsets: an exclusive scan of min(Op_j, rows)
    CK(cudaMemsetAsync(soff, 0, sizeof(int64_t), s));
    if (P->nB > 0) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(P->nB, 256), 16 * (int64_t)P->dev.sms));
        k_slot_caps<<<g, 256, 0, s>>>(P->op(), P->nB, P->mC, soff + 1);
        CK(cudaGetLastError());
        CK(launch_inclusive_scan(soff + 1, P->nB, P->tiles(), s));
    }
    // the tables and shared-memory shapes follow the slot sizes (no nnz(C_j) yet)
    for (int b = 1; b < NBINS; ++b) {
        if (!P->host.hist[b]) continue;
        const int64_t bound = std::min<int64_t>((int64_t)P->host.maxop[b], P->mC);
        P->num_geo[b] = numeric_geometry(b, (int64_t)P->host.hist[b], P->mC, c.cta_threads, P->dev.sms,
                                         P->dev.smem_optin, bound, P->dtype, c.table_slots_pct, P->L.scratch_ctas);
    }
    P->num_geo_ready = true;
    Operands o{A->colptr, P->compact ? P->arow() : A->rowidx, A->values, B->colptr, B->rowidx, B->values,
               P->compact ? P->rinv() : nullptr};
    st = run_numeric(P, o, soff, C_colptr, reinterpret_cast<int32_t *>(P->ws + P->srow_at), P->ws + P->sval_at, s);
    if (st != SPG_OK) { delete P; return st; }
    CK(launch_inclusive_scan(C_colptr + 1, P->nB, P->tiles(), s));
    CK(P->read(&P->nnzC, C_colptr + P->nB, sizeof(int64_t), &P->host, ctrl, sizeof(Ctrl), s));
#undef CK
    if (P->host.err) { st = (spg_status)P->host.err; delete P; return st; }
    // the preparation, slot caps and 3 scan kernels, the bins, 3 scan
    // kernels and the control read
    P->sym_launches += (P->nB > 0 ? 4 : 0) + P->nonempty_bins() + 4;
    *nnzC = P->nnzC;
    *plan_out = P;
    return SPG_OK;
}

spg_status spgemm_single_pass_copy(spg_plan *P, const int64_t *C_colptr, int32_t *C_rowidx, void *C_values,
                                   spg_stream stream) {
    if (!P || !P->single || !C_colptr || (P->nnzC > 0 && (!C_rowidx || !C_values))) return SPG_ERR_INVALID;
    const int w = P->dtype == SPG_F64 ? 8 : 4;
    return cuda_status(launch_slot_copy(P->nB, P->nnzC, C_colptr, reinterpret_cast<const int64_t *>(P->ws + P->soff_at),
                                        reinterpret_cast<int32_t *>(P->ws + P->tcol_at),
                                        reinterpret_cast<const int32_t *>(P->ws + P->srow_at),
                                        P->ws + P->sval_at, C_rowidx, C_values, w, P->dev.sms,
                                        reinterpret_cast<cudaStream_t>(stream)));
}

spg_status spgemm_backward(spg_plan *P, const spg_csc *A, const spg_csc *B, const int64_t *C_colptr,
                           const int32_t *C_rowidx, const void *dC_values, void *dA_values, void *dB_values,
                           spg_stream stream) {
    spg_status st = check_plan_operands(P, A, B);
    if (st != SPG_OK) return st;
    if (!C_colptr || (P->nnzC > 0 && (!C_rowidx || !dC_values))) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t w = P->dtype == SPG_F64 ? 8 : 4;
    if (dA_values && P->nnzA > 0 && cudaMemsetAsync(dA_values, 0, (size_t)P->nnzA * w, s) != cudaSuccess)
        return SPG_ERR_CUDA;
    if (dB_values && P->nnzB > 0 && cudaMemsetAsync(dB_values, 0, (size_t)P->nnzB * w, s) != cudaSuccess)
        return SPG_ERR_CUDA;
    if (!dA_values && !dB_values) return SPG_OK;
    Ctrl *ctrl = P->ctrl();
    if (cudaMemsetAsync(&ctrl->work, 0, sizeof(ctrl->work), s) != cudaSuccess) return SPG_ERR_CUDA;
    if (!P->bwd_geo_ready) {
        for (int b = 1; b < NBINS; ++b) {
            if (!P->host.hist[b]) continue;
            P->bwd_geo[b] = backward_geometry(b, (int64_t)P->host.hist[b], P->mA, P->cfg.cta_threads, P->dev.sms,
                                              P->dev.smem_optin, (int64_t)P->host.maxnnz[b], P->dtype,
                                              P->cfg.table_slots_pct, P->L.scratch_ctas);
        }
        P->bwd_geo_ready = true;
    }
    Operands o{A->colptr, A->rowidx, A->values, B->colptr, B->rowidx, B->values};
    for (int b = 1; b < NBINS; ++b) {
        if (!P->host.hist[b]) continue;
        cudaError_t e = launch_backward_bin(P->task(b, false), o, C_colptr, C_rowidx, dC_values, dA_values, dB_values,
                                            P->dtype, P->bwd_geo[b], s);
        if (e != cudaSuccess) return SPG_ERR_CUDA;
    }
    return SPG_OK;
}

// ------------------------------------------------------------ row-wise form
// The CSC view of M^T for a CSR matrix M: the same arrays.
static spg_csc csc_of_transpose(const spg_csr *M) {
    return spg_csc{M->ncols, M->nrows, M->nnz, M->rowptr, M->colidx, M->values, M->dtype};
}

spg_status spgemm_csr_workspace_size(const spg_csr *A, const spg_csr *B, const spg_config *cfg, size_t *bytes) {
    if (!A || !B) return SPG_ERR_INVALID;
    const spg_csc Bt = csc_of_transpose(B), At = csc_of_transpose(A);
    return spgemm_workspace_size(&Bt, &At, cfg, bytes);
}

spg_status spgemm_csr_symbolic(spg_handle *handle, const spg_csr *A, const spg_csr *B, const spg_config *cfg,
                               void *workspace, size_t ws_bytes, int64_t *C_rowptr, int64_t *nnzC,
                               spg_plan **plan, spg_stream stream) {
    if (plan) *plan = nullptr;
    if (!A || !B) return SPG_ERR_INVALID;
    const spg_csc Bt = csc_of_transpose(B), At = csc_of_transpose(A);
    return spgemm_symbolic(handle, &Bt, &At, cfg, workspace, ws_bytes, C_rowptr, nnzC, plan, stream);
}

spg_status spgemm_csr_numeric(spg_plan *plan, const spg_csr *A, const spg_csr *B, const int64_t *C_rowptr,
                              int32_t *C_colidx, void *C_values, spg_stream stream) {
    if (!A || !B) return SPG_ERR_INVALID;
    const spg_csc Bt = csc_of_transpose(B), At = csc_of_transpose(A);
    return spgemm_numeric(plan, &Bt, &At, C_rowptr, C_colidx, C_values, stream);
}

spg_status spgemm_csr_backward(spg_plan *plan, const spg_csr *A, const spg_csr *B, const int64_t *C_rowptr,
                               const int32_t *C_colidx, const void *dC_values, void *dA_values, void *dB_values,
                               spg_stream stream) {
    if (!A || !B) return SPG_ERR_INVALID;
    const spg_csc Bt = csc_of_transpose(B), At = csc_of_transpose(A);
    // the product runs as B^T A^T: its first operand's gradient is dB
    return spgemm_backward(plan, &Bt, &At, C_rowptr, C_colidx, dC_values, dB_values, dA_values, stream);
}

spg_status spg_plan_check(spg_plan *P, spg_stream stream) {
    if (!P) return SPG_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t err = 0;
    if (P->read(&err, &P->ctrl()->err, sizeof(err), nullptr, nullptr, 0, s) != cudaSuccess) return SPG_ERR_CUDA;
    return (spg_status)err;
}

spg_status spg_plan_destroy(spg_plan *P) {
    delete P;
    return SPG_OK;
}

spg_status spg_plan_info(const spg_plan *P, int32_t *nbins, int64_t *bin_counts, int64_t *products,
                         int64_t *t_effective) {
    if (!P) return SPG_ERR_INVALID;
    if (nbins) *nbins = NBINS;
    if (bin_counts)
        for (int b = 0; b < NBINS; ++b) bin_counts[b] = (int64_t)P->host.hist[b];
    if (products) *products = (int64_t)P->host.products;
    if (t_effective) *t_effective = P->t_eff;
    return SPG_OK;
}

spg_status spg_plan_bin_stats(const spg_plan *P, int64_t *bin_products, int64_t *bin_nnz, int64_t *bin_max_op,
                              int64_t *bin_max_nnz, int64_t *bin_nnz_b) {
    if (!P) return SPG_ERR_INVALID;
    for (int b = 0; b < NBINS; ++b) {
        if (bin_products) bin_products[b] = (int64_t)P->host.binprod[b];
        if (bin_nnz) bin_nnz[b] = (int64_t)P->host.binnnz[b];
        if (bin_max_op) bin_max_op[b] = (int64_t)P->host.maxop[b];
        if (bin_max_nnz) bin_max_nnz[b] = (int64_t)P->host.maxnnz[b];
        if (bin_nnz_b) bin_nnz_b[b] = (int64_t)P->host.binnnzb[b];
    }
    return SPG_OK;
}

spg_status spg_plan_launch_count(const spg_plan *P, int64_t *symbolic, int64_t *numeric, int64_t *backward) {
    if (!P) return SPG_ERR_INVALID;
    if (symbolic) *symbolic = P->sym_launches;
    if (numeric) *numeric = P->nonempty_bins() + (P->compact ? 1 : 0);
    if (backward) *backward = P->nonempty_bins();
    return SPG_OK;
}

spg_status spg_plan_bin_streams(const spg_plan *P, int32_t *side) {
    if (!P || !side) return SPG_ERR_INVALID;
    const bool fork = P->numeric_fork();
    for (int b = 0; b < NBINS; ++b) side[b] = fork && P->host.hist[b] && P->side_rule(b) ? 1 : 0;
    return SPG_OK;
}

spg_status spg_plan_set_timing(spg_plan *P, int32_t enable) {
    if (!P) return SPG_ERR_INVALID;
    if (enable) {
        for (int b = 0; b < NBINS; ++b) {
            if (!P->ev0[b] && cudaEventCreate(&P->ev0[b]) != cudaSuccess) return SPG_ERR_CUDA;
            if (!P->ev1[b] && cudaEventCreate(&P->ev1[b]) != cudaSuccess) return SPG_ERR_CUDA;
        }
    }
    P->timing = enable != 0;
    return SPG_OK;
}

spg_status spg_plan_bin_times(spg_plan *P, float *ms) {
    if (!P || !ms) return SPG_ERR_INVALID;
    for (int b = 0; b < NBINS; ++b) {
        ms[b] = 0.f;
        if (!P->timed || b == 0 || !P->host.hist[b]) continue;
        if (cudaEventSynchronize(P->ev1[b]) != cudaSuccess) return SPG_ERR_CUDA;
        if (cudaEventElapsedTime(&ms[b], P->ev0[b], P->ev1[b]) != cudaSuccess) return SPG_ERR_CUDA;
    }
    return SPG_OK;
}

spg_status spg_plan_op_counts(const spg_plan *P, int64_t *op_out, spg_stream stream) {
    if (!P || (!op_out && P->nB > 0)) return SPG_ERR_INVALID;
    if (P->nB == 0) return SPG_OK;
    return cuda_status(cudaMemcpyAsync(op_out, P->op(), (size_t)P->nB * 8, cudaMemcpyDeviceToDevice,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
