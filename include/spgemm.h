/*
 * spgemm.h -- C ABI of the GB300 (sm_103a) column-wise sparse product
 * C = A x B on CSC matrices, after arXiv 2303.02471 ("Optimization of SpGEMM
 * with RISC-V vector instructions").
 *
 * The method (Section 3.3, H-HASH(t)): every column j of B gets the
 * operation count Op_j = sum over stored B_kj of Z^A_k (Section 3.1, Z^A_k =
 * entries of column k of A).  Columns with Op_j >= t accumulate in a dense
 * sparse accumulator (SPA, Algorithm 1/2); lighter columns accumulate in a
 * hash table whose size follows Op_j (Section 3.2, "hash table size
 * adaptation").  Here the "sort by decreasing Op_j" of Section 3.1 becomes
 * binning of columns by Op_j, the dense SPA keeps its flags in a bitmap, and
 * each output column is emitted in ascending row order.
 *
 * Conventions for every entry point
 *   - Matrices are CSC (Section 2.1): column pointers int64[ncols + 1] with
 *     colptr[0] = 0 and colptr[ncols] = nnz, row indices int32[nnz], values
 *     double or float[nnz].  Rows inside an input column may come in any
 *     order but must not repeat.  All matrix arrays are DEVICE pointers.
 *   - The caller owns all device memory (inputs, outputs, workspace); the
 *     library never allocates device memory.  It owns only host-side
 *     objects: plans (spg_plan, freed by spg_plan_destroy) and handles
 *     (spg_handle: side streams, events and a small pinned host buffer,
 *     freed by spg_destroy).
 *   - Every call returns spg_status; no C++ exception crosses the ABI.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Kernels
 *     are enqueued on it; calls documented as synchronising wait for it.
 *   - Errors found by a kernel (bad input, table overflow) are written to an
 *     error word in the workspace and reported by the next synchronising
 *     call (spgemm_symbolic, spg_plan_check).
 *   - The output pattern is the structural boolean product of the stored
 *     patterns: an entry formed by at least one product A_ik * B_kj is
 *     stored even if the products cancel to 0 (Algorithm 1 flags every
 *     touched row).  Output rows are sorted ascending in every column.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *spg_stream;

typedef enum {
    SPG_OK = 0,
    SPG_ERR_INVALID = 1,        /* bad argument or malformed CSC input */
    SPG_ERR_WORKSPACE = 2,      /* workspace missing or too small */
    SPG_ERR_TABLE_OVERFLOW = 3, /* a hash table ran out of slots (bounded probe) */
    SPG_ERR_TIMEOUT = 4,        /* a bounded device loop hit its limit */
    SPG_ERR_CUDA = 5,           /* a CUDA runtime call failed */
    SPG_ERR_UNSUPPORTED = 6,    /* shape or option outside what is built */
    SPG_ERR_INDEX_OVERFLOW = 7  /* a size does not fit the index types */
} spg_status;

typedef enum { SPG_F64 = 0, SPG_F32 = 1 } spg_dtype;

/* A CSC matrix on the device (Section 2.1).  `values` may be NULL where only
 * the pattern is read (symbolic phase). */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const int64_t *colptr; /* device, ncols + 1 */
    const int32_t *rowidx; /* device, nnz */
    const void *values;    /* device, nnz elements of `dtype` */
    int32_t dtype;         /* spg_dtype */
} spg_csc;

/* Tuning knobs.  spg_config_default fills the defaults. */
typedef struct {
    /* Threshold t of H-HASH(t) (Section 3.3): a column with Op_j >= t uses
     * the dense SPA, a column with 0 < Op_j < t a hash table.  t = 0 sends
     * every non-empty column to the dense SPA; INT64_MAX ("infinity") sends
     * all to hash tables; a negative value picks the library default
     * ceil(m / 512) clamped to [257, hash_cta_max + 1], m = rows of A that
     * hold entries. */
    int64_t t;
    /* Largest Op_j served by shared-memory hash tables; must be one of
     * 256, 512, 1024, 2048, 4096 or 8192.  Hash columns above it use a
     * per-CTA global-memory table. */
    int32_t hash_cta_max;
    /* Threads per CTA for the CTA-per-column kernels (128..1024, multiple
     * of 32). */
    int32_t cta_threads;
    /* Nonzero: check the CSC inputs on the device in spgemm_symbolic
     * (colptr monotone with colptr[0] = 0 and colptr[n] = nnz, rows in
     * range) and fail with SPG_ERR_INVALID. */
    int32_t validate;
    /* Test knob, normally 0: divide every hash-table size by 2^shrink so
     * that the bounded probe loop reports SPG_ERR_TABLE_OVERFLOW. */
    int32_t table_shrink;
    /* Cap on the bytes of per-CTA global scratch (global hash tables and
     * bitmaps); the number of CTAs that use such scratch shrinks to fit. */
    int64_t scratch_cap_bytes;
    /* Bytes of workspace that keep the SPA flag bitmaps (m bits per column)
     * the symbolic phase builds for dense-SPA columns, so that the numeric
     * phase reuses them instead of walking the column's products twice.
     * Columns beyond the budget rebuild their flags.  0 disables;
     * default 2 GiB.  The batched calls keep flags the same way for dense
     * columns worked one per warp (every product at most 32768 rows), and
     * their workspace grows by up to this budget. */
    int64_t dense_cache_bytes;
    /* Nonzero (default): next to a dense bin, the bins that use no workspace
     * scratch run on the side streams, overlapping the dense kernel's tail.
     * 0: every bin runs in order on the caller's stream (then the per-bin
     * event times of spg_plan_bin_times measure each kernel on its own). */
    int32_t side_streams;
    /* Test knob, normally 0: nonzero makes the dense numeric kernel give up
     * its first wait for a column's kept flags at once, as if the bounded
     * wait had run out.  The copy it waited for still lands (the kernel
     * waits for it, bounded, before it exits), the columns left are not
     * written, and spg_plan_check reports SPG_ERR_TIMEOUT: the time-out path
     * runs without any fault. */
    int32_t test_wait_timeout;
    /* Accumulator of the lane-group bins (columns with Op_j <= 256):
     * SPG_ACC_HASH, the hash tables of Section 3.2, in both phases;
     * SPG_ACC_ESC, the ESC algorithm of Section 4 (the products of a tile of
     * columns are expanded into shared memory, sorted by (column, row) and
     * compressed), in both phases; SPG_ACC_AUTO (default), ESC for the
     * numeric phase and, for the symbolic phase's counts, ESC in the bins of
     * Op_j <= 64 (sorted by rank) and hash tables in the larger ones (the
     * cheaper in each case, measured on GB300).  A bin whose (column, row)
     * keys do not fit 32 bits keeps hash tables.  All give the
     * same C (the ESC sums do not depend on timing).  The single pass uses
     * ESC unless SPG_ACC_HASH.  Only the single products use it; the batched
     * calls keep hash tables. */
    int32_t small_accumulator;
    /* Size of the hash tables of the numeric and backward phases' CTA and
     * global bins (Section 3.2's table size), in slots per output entry of
     * the column, as a percentage: 125..400, default 150 (a load of at most
     * 2/3).  Larger tables probe less but take more shared memory, so a
     * bin's tables move to the workspace scratch sooner.  Results do not
     * depend on it. */
    int32_t table_slots_pct;
    /* Lanes per column of the lane-group bins (columns with Op_j <= 256):
     * 0 (default) gives a column the smallest group bin that holds its
     * Op_j; 1 or 2 moves it that many group bins up (at most the
     * Op_j <= 256 bin), so that it gets more lanes, registers and table
     * slots, and a warp holds fewer columns.  Results do not depend on it. */
    int32_t group_promote;
} spg_config;

enum { SPG_ACC_HASH = 0, SPG_ACC_ESC = 1, SPG_ACC_AUTO = 2 };

typedef struct spg_plan spg_plan;

/*
 * Library handle: the state that outlives single products on one device.
 * It holds the two side streams and three events onto which the symbolic
 * and numeric calls fork their lane-group bins (joined back to the caller's
 * stream before each call returns), and the 64 KiB mapped pinned host buffer
 * through which the synchronising calls read small results (bin histogram,
 * nnz(C), error word) back.  spg_create makes all of them at once for the
 * current device, so no later call made with the handle creates a stream,
 * an event or a host buffer; spg_destroy releases them.
 *   - Plans made with a handle use it until they are destroyed: destroy the
 *     plans first.
 *   - Calls made with one handle share its side streams, so their lane-group
 *     bins run in order; products meant to run concurrently on different
 *     caller streams take one handle each.
 *   - The read-back buffer is taken under a lock: a handle may be used by
 *     several host threads.
 *   - Every call that takes a handle also accepts NULL: the plan then
 *     creates its own side streams on its first forked call (released with
 *     the plan) and reads back through a buffer of the calling host thread.
 * The paper has no counterpart (it is the GPU form of process-wide state).
 * Errors: SPG_ERR_INVALID (NULL out pointer), SPG_ERR_CUDA (stream, event or
 * pinned allocation failed; nothing is left allocated).
 */
typedef struct spg_handle spg_handle;
spg_status spg_create(spg_handle **handle);
spg_status spg_destroy(spg_handle *handle);

/* Fill `cfg` with the defaults. */
spg_status spg_config_default(spg_config *cfg);

/* Human-readable name of a status code (static string, never NULL). */
const char *spg_status_string(spg_status s);

/*
 * Bytes of device workspace that spgemm_symbolic needs for C = A x B with
 * `cfg` (NULL = defaults).  Depends only on the shapes, nnz and dtype of A
 * and B, so it can be queried before any data exists.  The workspace also
 * holds the plan's device state (Op_j, bins) used later by spgemm_numeric
 * and spgemm_backward, so it must stay allocated and unmodified until the
 * plan is destroyed.  Does not touch the device.
 */
spg_status spgemm_workspace_size(const spg_csc *A, const spg_csc *B,
                                 const spg_config *cfg, size_t *bytes);

/*
 * Symbolic phase of C = A x B (Gustavson by columns, Section 2.1).
 *
 * Steps on `stream`: (optional) input validation; a numbering of the rows
 * of A that hold entries (a row of A without entries has none in C; when it
 * saves at least a tenth of the rows, the forward passes work on these rows
 * and map them back when C is written); Op_j of every column of B
 * (Section 3.1) and its bin (empty / hash table sized by Op_j / dense SPA,
 * Sections 3.2-3.3); per-bin column lists; nnz of every C column by the
 * bin's accumulator; exclusive scan into C_colptr.
 *
 * handle   from spg_create on the current device, or NULL (see spg_create);
 *          kept by the plan for its numeric, backward and check calls.
 * A, B     device CSC; values are not read.  A->ncols == B->nrows,
 *          A->dtype == B->dtype.
 * cfg      tuning (NULL = defaults); copied into the plan.
 * workspace, ws_bytes   device buffer of at least spgemm_workspace_size
 *          bytes, 256-byte aligned, owned by the caller.
 * C_colptr device int64[B->ncols + 1], written (C_colptr[0] = 0).
 * nnzC     host, receives nnz(C) = C_colptr[B->ncols].
 * plan     receives a new plan (host object) on success; NULL on error.
 *
 * Synchronises `stream` (it reads the bin histogram and nnz(C) back to the
 * host, through a small mapped pinned buffer of the calling thread, so these
 * reads do not wait behind the caller's copies on other streams).  Errors: SPG_ERR_INVALID (shapes, dtypes, NULL pointers, or a
 * malformed input when cfg->validate), SPG_ERR_WORKSPACE, SPG_ERR_INDEX_OVERFLOW
 * (a dimension beyond int32 rows), SPG_ERR_UNSUPPORTED (a column with
 * Op_j >= 2^31 products), SPG_ERR_TABLE_OVERFLOW, SPG_ERR_CUDA.
 */
spg_status spgemm_symbolic(spg_handle *handle, const spg_csc *A,
                           const spg_csc *B, const spg_config *cfg,
                           void *workspace,
                           size_t ws_bytes, int64_t *C_colptr, int64_t *nnzC,
                           spg_plan **plan, spg_stream stream);

/*
 * Numeric phase: values and sorted row indices of C = A x B into caller
 * buffers, column by column with the accumulator the plan chose per bin
 * (dense SPA of Algorithm 1 for Op_j >= t, hash table of Section 3.2
 * otherwise), then each column in ascending row order.
 *
 * plan     from spgemm_symbolic on the same A and B patterns (values may
 *          differ); its workspace must still be allocated.
 * A, B     device CSC with values of the plan's dtype.
 * C_colptr the array spgemm_symbolic wrote.
 * C_rowidx device int32[nnzC], written.
 * C_values device values[nnzC] of the plan's dtype, written.  Values are
 *          summed in the input dtype (float inputs accumulate in float).
 *
 * Asynchronous: does not synchronise.  When the plan has a dense bin and
 * lane-group bins, the group bins run on the two side streams of the plan's
 * handle (or, without a handle, two streams the plan creates on first use
 * and releases with the plan), forked from `stream` by an event and joined
 * back to it before the call returns, also when a launch fails, so later
 * work on `stream` sees all of C; the pattern is legal on the legacy default
 * stream and under stream capture.  The symbolic call does the same for its
 * group bins.  Kernel-side errors surface in
 * spg_plan_check: SPG_ERR_INVALID when a column's row count differs from the
 * plan's, or when A has an entry in a row that held none when the plan was
 * made (the plan numbers only the rows of A that hold entries; such an entry
 * is not walked and C's contents are then unspecified).  Errors returned
 * directly: SPG_ERR_INVALID (plan/shape mismatch, NULL pointers),
 * SPG_ERR_CUDA (launch failure).
 */
spg_status spgemm_numeric(spg_plan *plan, const spg_csc *A, const spg_csc *B,
                          const int64_t *C_colptr, int32_t *C_rowidx,
                          void *C_values, spg_stream stream);

/*
 * Backward of C = A x B with respect to the stored values of A and B (the
 * patterns are fixed):
 *   dA_ik = sum_{j: B_kj stored} dC_ij B_kj   for every stored (i, k) of A,
 *   dB_kj = sum_i A_ik dC_ij                  for every stored (k, j) of B,
 * i.e. dA = (dC B^T) sampled on pattern(A) and dB = (A^T dC) sampled on
 * pattern(B).  The paper has no backward; these are the derivatives of
 * C_ij = sum_k A_ik B_kj.  Both are masked products that walk the same
 * products as the forward, reusing the plan's bins: per column j, dC[:, j]
 * is loaded into the bin's accumulator (hash table or dense SPA) and every
 * product A_ik B_kj looks up dC_ij.
 *
 * C_colptr, C_rowidx   the forward's output pattern (sorted rows).
 * dC_values            device values[nnzC] (plan dtype).
 * dA_values            device values[A->nnz] or NULL (not computed).
 * dB_values            device values[B->nnz] or NULL (not computed).
 * Asynchronous; errors as for spgemm_numeric.
 */
spg_status spgemm_backward(spg_plan *plan, const spg_csc *A, const spg_csc *B,
                           const int64_t *C_colptr, const int32_t *C_rowidx,
                           const void *dC_values, void *dA_values,
                           void *dB_values, spg_stream stream);

/*
 * Single-pass form (no symbolic phase).  Section 3.2 sizes a column's hash
 * table from Op_j alone; taken one step further, every column gets a slot of
 * min(Op_j, m) entries (m = rows of the forward passes) in the workspace,
 * which bounds nnz(C_j) without counting it first.  Each bin's accumulator
 * (hash table, ESC or dense SPA, as in spgemm_numeric) writes its sorted
 * column into its slot and its entry count into C_colptr[j + 1]; the counts
 * are scanned into C_colptr.  spgemm_single_pass_copy then moves the columns
 * from their slots into the caller's C.  The slots cost sum_j min(Op_j, m)
 * entries of workspace and one copy of C, against the symbolic phase's walk
 * of every product: it pays where Op_j and nnz(C_j) are close (very sparse
 * columns).
 *
 * spgemm_single_pass_size: the workspace bytes spgemm_single_pass needs
 *   (they depend on Op_j, hence on the patterns).  Runs the preparation (input
 *   validation, row numbering, Op_j) in `workspace`, which must hold at least
 *   spgemm_workspace_size(A, B, cfg) bytes computed with
 *   cfg->dense_cache_bytes = 0 (the single pass keeps no flags); C_colptr
 *   (device int64[B->ncols + 1]) is used as scratch.  Synchronises.
 * spgemm_single_pass: A and B with values; workspace of at least the bytes
 *   above, 256-byte aligned; writes C_colptr (device int64[B->ncols + 1]) and
 *   nnzC (host), and returns a plan whose slots hold C.  The plan also serves
 *   spgemm_numeric (which recomputes C from the A and B it is given, into the
 *   caller's buffers), spgemm_backward and the plan queries.  Synchronises.
 * spgemm_single_pass_copy: C's rows (device int32[nnzC]) and values (device,
 *   plan dtype) from the plan's slots, in order; asynchronous.  The values are
 *   those of the A and B given to spgemm_single_pass.
 * Errors: as spgemm_symbolic; SPG_ERR_WORKSPACE when the workspace is smaller
 * than spgemm_single_pass_size says; SPG_ERR_INVALID for a plan that is not
 * a single-pass plan (copy).
 */
spg_status spgemm_single_pass_size(spg_handle *handle, const spg_csc *A,
                                   const spg_csc *B, const spg_config *cfg,
                                   void *workspace, size_t ws_bytes,
                                   int64_t *C_colptr, size_t *bytes,
                                   spg_stream stream);
spg_status spgemm_single_pass(spg_handle *handle, const spg_csc *A,
                              const spg_csc *B, const spg_config *cfg,
                              void *workspace, size_t ws_bytes,
                              int64_t *C_colptr, int64_t *nnzC,
                              spg_plan **plan, spg_stream stream);
spg_status spgemm_single_pass_copy(spg_plan *plan, const int64_t *C_colptr,
                                   int32_t *C_rowidx, void *C_values,
                                   spg_stream stream);

/*
 * Row-wise (CSR) form.  Section 2.1 notes that the method applies to rows of
 * CSR matrices as well as to columns of CSC ones.  A CSR matrix's arrays
 * (row pointers, column indices, values) are the CSC arrays of its
 * transpose, and C^T = B^T A^T, so these calls run the column-wise product
 * on (B^T, A^T): Op_j, bins and accumulators work on the rows of B and the
 * output's row pointers, column indices (ascending in each row) and values
 * are C in CSR.  Same conventions, ownership and errors as the CSC calls,
 * with rows for columns:
 *   A (m x k) and B (k x n) in CSR, device arrays; C_rowptr int64[m + 1];
 *   spgemm_csr_backward gives dA on pattern(A) and dB on pattern(B).
 * The plan belongs to the CSR calls (it holds the roles swapped).
 */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const int64_t *rowptr; /* device, nrows + 1 */
    const int32_t *colidx; /* device, nnz */
    const void *values;    /* device, nnz elements of `dtype` */
    int32_t dtype;         /* spg_dtype */
} spg_csr;

spg_status spgemm_csr_workspace_size(const spg_csr *A, const spg_csr *B,
                                     const spg_config *cfg, size_t *bytes);
spg_status spgemm_csr_symbolic(spg_handle *handle, const spg_csr *A,
                               const spg_csr *B, const spg_config *cfg,
                               void *workspace, size_t ws_bytes,
                               int64_t *C_rowptr, int64_t *nnzC,
                               spg_plan **plan, spg_stream stream);
spg_status spgemm_csr_numeric(spg_plan *plan, const spg_csr *A,
                              const spg_csr *B, const int64_t *C_rowptr,
                              int32_t *C_colidx, void *C_values,
                              spg_stream stream);
spg_status spgemm_csr_backward(spg_plan *plan, const spg_csr *A,
                               const spg_csr *B, const int64_t *C_rowptr,
                               const int32_t *C_colidx,
                               const void *dC_values, void *dA_values,
                               void *dB_values, spg_stream stream);

/* Synchronise `stream` and report the first kernel-side error recorded in
 * the plan's workspace since spgemm_symbolic (SPG_OK if none). */
spg_status spg_plan_check(spg_plan *plan, spg_stream stream);

/* Release the host plan (the workspace stays the caller's). */
spg_status spg_plan_destroy(spg_plan *plan);

/*
 * Plan introspection for tests and reports (host side, no device work):
 *   nbins        receives the number of bins (may be NULL);
 *   bin_counts   host int64[nbins]: columns per bin (may be NULL);
 *   products     receives sum_j Op_j (may be NULL);
 *   t_effective  receives the threshold t the plan used (may be NULL).
 * Bin order: 0 empty (Op_j = 0); 1..6 warp-level hash bins for
 * Op_j <= 8, 16, 32, 64, 128, 256; 7..11 CTA-level shared-memory hash bins for
 * Op_j <= 512 .. 8192; 12 global-memory hash; 13 dense SPA (Op_j >= t).
 */
spg_status spg_plan_info(const spg_plan *plan, int32_t *nbins,
                         int64_t *bin_counts, int64_t *products,
                         int64_t *t_effective);

/* Per-bin statistics of the plan, host arrays of spg_plan_info's nbins
 * entries (any may be NULL): sum of Op_j, sum of nnz(C_j), largest Op_j,
 * largest nnz(C_j) and sum of nnz(B_j) over the bin's columns.  No device
 * work. */
spg_status spg_plan_bin_stats(const spg_plan *plan, int64_t *bin_products,
                              int64_t *bin_nnz, int64_t *bin_max_op,
                              int64_t *bin_max_nnz, int64_t *bin_nnz_b);

/* Kernels one spgemm_symbolic call launched for this plan, and the kernels
 * one spgemm_numeric / spgemm_backward call launches (host, no device work). */
spg_status spg_plan_launch_count(const spg_plan *plan, int64_t *symbolic,
                                 int64_t *numeric, int64_t *backward);

/* Where each bin's numeric kernel runs (host int32[nbins]): 1 on a side
 * stream of the fork (its event times then include waiting for SMs held by
 * the dense kernel), 0 on the caller's stream.  No device work. */
spg_status spg_plan_bin_streams(const spg_plan *plan, int32_t *side);

/* Enable (nonzero) or disable event timing of every bin kernel in later
 * spgemm_numeric calls of this plan (CUDA events, no device memory). */
spg_status spg_plan_set_timing(spg_plan *plan, int32_t enable);

/* Milliseconds each bin kernel of the last timed spgemm_numeric call took
 * (host float[nbins]; 0 for bins without columns).  Waits for those events. */
spg_status spg_plan_bin_times(spg_plan *plan, float *ms);

/* Copy Op_j (int64[B->ncols], Section 3.1) from the plan's workspace into
 * the device buffer `op_out` on `stream` (asynchronous). */
spg_status spg_plan_op_counts(const spg_plan *plan, int64_t *op_out,
                              spg_stream stream);

/*
 * Transpose of a CSC matrix M (m x n) into CSC of M^T (n x m): row k of M
 * becomes column k.  Pure data movement; the Galerkin product P^T (A P) of
 * the differentiable workload needs P^T as a CSC operand.
 *
 * M            device CSC (values may be NULL: then T_values is not written);
 *              rows outside [0, M->nrows) are dropped.
 * T_colptr     device int64[M->nrows + 1], written.
 * T_rowidx     device int32[M->nnz], written; rows inside each output column
 *              are in ascending order (deterministic).
 * T_values     device values[M->nnz] (M's dtype) or NULL.
 * perm         device int64[M->nnz] or NULL: T_values[e] = M.values[perm[e]].
 * workspace    device buffer of spg_transpose_workspace_size bytes.
 * Asynchronous.  Errors: SPG_ERR_INVALID, SPG_ERR_WORKSPACE, SPG_ERR_CUDA.
 */
spg_status spg_transpose_workspace_size(const spg_csc *M, size_t *bytes);
spg_status spg_csc_transpose(const spg_csc *M, int64_t *T_colptr,
                             int32_t *T_rowidx, void *T_values, int64_t *perm,
                             void *workspace, size_t ws_bytes,
                             spg_stream stream);

/* ------------------------------------------------------------- batched
 * nb independent products C_i = A_i x B_i (uneven sizes, each pair with its
 * own dtype).  The columns of all products are binned together by Op_j and
 * each phase runs as one persistent kernel whose blocks take work items
 * (one column of a CTA-level bin, or a tile of columns of a warp-group bin;
 * in the symbolic and numeric phases of a batch whose products all have at
 * most 32768 rows, a tile of dense columns, one per warp) heaviest first.  The paper has no batched form; the per-column work is the
 * method of the single product (H-HASH(t), Section 3.3).  In the batched
 * kernels t is at most hash_cta_max + 1 (no global-memory hash tables), and
 * every product's bitmaps must fit shared memory (m_i up to ~2^20 rows);
 * otherwise the calls return SPG_ERR_UNSUPPORTED.
 *
 * A, B         host arrays of nb spg_csc (device pointers inside).
 * C_colptr     device int64[sum_i (B[i].ncols + 1)], concatenated: product
 *              i's column pointers start at sum_{i' < i} (B[i'].ncols + 1).
 */
typedef struct spg_bplan spg_bplan;

/* Workspace bytes of a batch (shapes only; no device work). */
spg_status spgemm_batched_workspace_size(int32_t nb, const spg_csc *A,
                                         const spg_csc *B,
                                         const spg_config *cfg, size_t *bytes);

/* Symbolic phase of the whole batch: validation (cfg->validate), Op_j and
 * bins over all columns, one persistent kernel for nnz(C_i[:, j]), a
 * segmented scan into C_colptr.  nnzC: host int64[nb].  handle: as for
 * spgemm_symbolic (its read-back buffer serves the batch's synchronising
 * reads), or NULL.  Synchronises. */
spg_status spgemm_batched_symbolic(spg_handle *handle, int32_t nb,
                                   const spg_csc *A, const spg_csc *B,
                                   const spg_config *cfg,
                                   void *workspace, size_t ws_bytes,
                                   int64_t *C_colptr, int64_t *nnzC,
                                   spg_bplan **plan, spg_stream stream);

/* Numeric phase of the whole batch in ONE persistent kernel launch.
 * C_rowidx, C_values: host arrays of nb device pointers (nnzC[i] entries).
 * use_graph: nonzero captures the launch (with its counter reset) into a CUDA
 * graph on the first call and replays it while the pointers stay the same
 * (re-captured when they change).  The legacy default stream (0) cannot be
 * captured: there the launch runs directly, as with use_graph = 0.
 * Asynchronous. */
spg_status spgemm_batched_numeric(spg_bplan *plan, const spg_csc *A,
                                  const spg_csc *B, const int64_t *C_colptr,
                                  int32_t *const *C_rowidx,
                                  void *const *C_values, int32_t use_graph,
                                  spg_stream stream);

/* Backward of every product (as spgemm_backward) in one persistent launch.
 * dA_values / dB_values: host arrays of nb device pointers or NULL arrays;
 * an individual NULL pointer skips that gradient.  Asynchronous. */
spg_status spgemm_batched_backward(spg_bplan *plan, const spg_csc *A,
                                   const spg_csc *B, const int64_t *C_colptr,
                                   const int32_t *const *C_rowidx,
                                   const void *const *dC_values,
                                   void *const *dA_values,
                                   void *const *dB_values, spg_stream stream);

/* Synchronise and report the first kernel-side error of the batch. */
spg_status spg_bplan_check(spg_bplan *plan, spg_stream stream);

/* Host statistics: columns per bin (int64[nbins]), total products, and the
 * kernels launched by the symbolic, numeric and backward calls (int64[3]). */
spg_status spg_bplan_info(const spg_bplan *plan, int64_t *bin_counts,
                          int64_t *products, int64_t *launches);

spg_status spg_bplan_destroy(spg_bplan *plan);

/*
 * Permute a value array on the device: dst[i] = src[idx[i]] (scatter = 0) or
 * dst[idx[i]] = src[i] (scatter = 1), i < n.  With the permutation of
 * spg_csc_transpose this moves values (or their gradients) between M and
 * M^T.  idx must be a permutation of [0, n) for scatter.  Asynchronous.
 * Errors: SPG_ERR_INVALID, SPG_ERR_CUDA.
 */
spg_status spg_permute_values(const void *src, const int64_t *idx, void *dst,
                              int64_t n, int32_t dtype, int32_t scatter,
                              spg_stream stream);

/*
 * spg_csc_transpose for callers that cannot allocate device memory and
 * cannot pass a workspace: code that runs where cudaMalloc is unavailable or
 * forbidden (a plug-in whose host owns every allocation, a fixed device
 * memory budget, a pool that hands out only the inputs and outputs).  The
 * paper has no counterpart; it is a service of this library.
 *
 * Same arguments and results as spg_csc_transpose minus the workspace: the
 * scratch is a file-scope device array of SPG_NOALLOC_SCRATCH_BYTES inside
 * this library, which every GPU that loads the library holds until the
 * process exits.  Nothing is allocated by the call.
 *   - The matrix must satisfy spg_transpose_workspace_size(M) <=
 *     SPG_NOALLOC_SCRATCH_BYTES (32 MiB, about 1.3 million entries);
 *     larger ones are rejected with SPG_ERR_WORKSPACE before any device work.
 *   - The first call on a device looks up the array's device address on the
 *     current device (cudaGetSymbolAddress); make that first call before any
 *     stream capture on that device.  The address is kept per device and
 *     CUDA context: after a device reset, or in another context, the next
 *     call looks it up again (so make that call outside a capture too).
 *   - All calls on a device share the array, which keeps the last call's
 *     contents (the parts that must start at zero are cleared by every
 *     call); calls whose work overlaps on the GPU race on it, so order them,
 *     e.g. on one stream.
 * Errors: as spg_csc_transpose, plus SPG_ERR_WORKSPACE for a matrix beyond
 * the limit and SPG_ERR_CUDA if the address lookup fails.
 */
#define SPG_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
spg_status spg_csc_transpose_noalloc(const spg_csc *M, int64_t *T_colptr,
                                     int32_t *T_rowidx, void *T_values,
                                     int64_t *perm, spg_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_GB300_H */
