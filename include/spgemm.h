/*
 * spgemm.h -- C ABI of the GB300 (sm_103a) semiring SpGEMM library.
 *
 * The library computes C = A (x).(+) B for sparse matrices in CSR form over a
 * semiring chosen by id: the local multiplication at the core of distributed
 * Sparse SUMMA (McFarland, Bellavita, Guidi, "Parallel GPU-Enabled
 * Algorithms for SpGEMM on Arbitrary Semirings with Hybrid Communication",
 * ICPE'25; SpGEMM and Sparse SUMMA: Section 2.1; semirings: Section 2.2;
 * CSR: Section 2.4; merge of per-stage products: Section 3.4).
 *
 * Definition computed (every entry point that multiplies):
 *     C[i,j] = (+)_{k in cols(A_i), j in cols(B_k)}  A[i,k] (x) B[k,j]
 * and (i,j) is stored iff at least one product exists (structural pattern;
 * no entry is dropped because of its value).
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Matrices are CSR: row_ptr is int64 [nrows+1] with row_ptr[0] == 0 and
 *   non-decreasing; col is int32 [nnz] with column ids in [0, ncols) strictly
 *   ascending inside each row; val is [nnz] values of the semiring's input type
 *   (NULL for SPG_SR_BOOL_OR_AND).  Outputs follow the same rules.
 * - Unless an entry point says "host", every pointer is a DEVICE pointer owned
 *   by the caller.  The library never frees caller memory and never keeps a
 *   pointer past the call.  Scratch memory comes from the caller's workspace.
 * - Work is queued on the caller's CUDA stream (`stream`, a cudaStream_t; NULL
 *   is the legacy default stream) and runs asynchronously, except where a
 *   call returns a host count (it then synchronises that stream).
 * - Argument errors are returned synchronously.  Errors found by kernels
 *   (hash-table overflow, counts that disagree with the row pointers given)
 *   are recorded in the workspace and reported by the next call that
 *   synchronises, or by spgemm_check().  No kernel of the library waits on
 *   another kernel, a flag or a peer, so no call can time out.
 * - B.nrows must equal A.ncols.  Empty matrices and empty rows are valid and
 *   give empty output rows.
 */
#ifndef SPGEMM_H
#define SPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPG_OK = 0,
    SPG_ERR_INVALID_ARG = 1,   /* a NULL pointer, a bad id or mismatched shapes      */
    SPG_ERR_INVALID_CSR = 2,   /* spgemm_validate_csr found a malformed matrix       */
    SPG_ERR_OOM = 3,           /* a device buffer of the host API could not be had:
                                  cudaMalloc failed, or the buffers would exceed
                                  spg_tuning.host_alloc_limit                       */
    SPG_ERR_CUDA = 4,          /* a CUDA runtime call failed (see spgemm_last_error) */
    SPG_ERR_UNSUPPORTED = 5,   /* shape beyond the library's index range             */
    SPG_ERR_OVERFLOW = 6,      /* a hash table ran out of slots (capacity too small) */
                               /* 7: not used                                        */
    SPG_ERR_WORKSPACE = 8      /* workspace NULL or smaller than required            */
} spg_status;

/* Semirings (Section 2.2): (+) must be commutative and associative, (x) associative. */
typedef enum {
    SPG_SR_PLUS_TIMES_F64 = 0, /* (+)=+, (x)=*, double in and out                           */
    SPG_SR_BOOL_OR_AND = 1,    /* pattern only: val pointers are ignored (pass NULL)         */
    SPG_SR_MIN_PLUS_F32 = 2,   /* (+)=min, (x)=+, float; min orders -0 below +0; no NaN     */
    SPG_SR_OVERLAP_I32 = 3,    /* in: int32 position of a k-mer in its read; out: spg_overlap */
    SPG_SR_PLUS_TIMES_I64 = 4, /* int64, wrap-around modulo 2^64                             */
    SPG_SR_PLUS_TIMES_F32 = 5  /* float: the "float" semiring of the paper's experiments    */
} spg_semiring;

/* One CSR matrix (see conventions above). */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* val;
} spg_csr;

/*
 * Output record of SPG_SR_OVERLAP_I32 (20 bytes, no padding).  For reads i, j
 * sharing k-mers: count = number of shared k-mers; (a0,b0) and (a1,b1) are the
 * two lexicographically smallest (position in read i, position in read j)
 * pairs, a0 <= a1.  A missing second pair is (INT32_MAX, INT32_MAX).
 * (x) makes {1, (a,b), none}; (+) adds counts and keeps the two smallest pairs.
 */
typedef struct {
    int32_t count, a0, b0, a1, b1;
} spg_overlap;

/* Kernel tier limits; 0 in any field keeps the library default. */
typedef struct {
    int64_t sym_warp_max_ub;    /* symbolic: ub_i <= this -> one warp per row, hash     */
    int64_t sym_block_max_ub;   /* symbolic: ub_i <= this -> one CTA per row, hash      */
    int64_t num_warp_max_nnz;   /* numeric: nnz(C_i) <= this -> warp hash + warp sort  */
    int64_t num_block_max_nnz;  /* numeric: nnz(C_i) <= this -> CTA hash + CTA sort   */
    int64_t dense_slab_cols;    /* numeric dense tier: columns per shared-memory slab   */
    int64_t sym_slab_cols;      /* symbolic dense tier: columns per bitmap slab         */
    int64_t bitmap_cache_bytes; /* workspace bytes that keep the symbolic phase's row
                                   bitmaps for the numeric dense tier (< 0: none)      */
    int64_t host_panel_bytes;   /* host API: outputs larger than this are produced in
                                   row panels of about this size, each panel's download
                                   overlapping the next panel's kernels (0: 1 GiB)     */
    int64_t deterministic;      /* != 0: plus-times FP64/FP32 values are summed in the
                                   order of A's entries (k ascending, a left fold from
                                   the first product): bit-identical run to run and to a
                                   sequential Gustavson; costs an extra ordered pass    */
    int64_t host_alloc_limit;   /* host API: most device bytes the handle may hold for
                                   its copies of A, B, C and the workspace; the buffer
                                   that would cross it is not allocated and the call
                                   returns SPG_ERR_OOM (buffers already held stay with
                                   the handle).  0: no limit beyond the device's        */
    int64_t rank_light_ub;      /* numeric dense tier: rows with fewer products than
                                   this (rounded up to a power of two) whose outputs
                                   fit one pass of a half-SM CTA run two per SM
                                   (0: 8192; < 0: never)                                */
} spg_tuning;

/* Counters of the last analysis on a handle (host copy, filled by spgemm_symbolic). */
typedef struct {
    int64_t products;           /* P = sum_i sum_{k in A_i} nnz(B_k)                      */
    int64_t nnz_c;              /* nnz(C)                                                */
    int64_t rows_per_tier[4];   /* symbolic rows: dense, block, warp, empty              */
    int64_t launches;           /* kernels launched by the last symbolic / numeric call   */
    int64_t learned_rows;       /* learned path: rows finished without the symbolic pass  */
    int64_t overflow_rows;      /* learned path: rows whose capacity was too small         */
    int64_t staging_entries;    /* learned path: sum of the capacities of learned rows     */
    int64_t learned_nnz;        /* learned path: nnz(C) of the rows it finished            */
    int64_t reserved[1];
} spg_stats;

typedef struct spg_handle spg_handle;

/* Create / destroy a handle (holds tuning, the current device's properties and
 * the last error text).  A handle is used by one host thread at a time.
 * Library services with no counterpart in the paper.  Errors: SPG_ERR_INVALID_ARG
 * (NULL pointer), SPG_ERR_CUDA (no usable device for spgemm_create). */
spg_status spgemm_create(spg_handle** handle);
spg_status spgemm_destroy(spg_handle* handle);

/* Text of the last error on this handle ("" if none).  Owned by the handle. */
const char* spgemm_last_error(const spg_handle* handle);

/* Tier limits (see spg_tuning).  They change speed only, never C (the
 * paper's GALATIC configuration knobs, Section 3.3, play this role there).
 * Counters (spg_stats) of the last call.  Errors: SPG_ERR_INVALID_ARG. */
spg_status spgemm_set_tuning(spg_handle* handle, const spg_tuning* tuning);
spg_status spgemm_get_tuning(const spg_handle* handle, spg_tuning* tuning);
spg_status spgemm_get_stats(const spg_handle* handle, spg_stats* stats);

/*
 * Bytes of device workspace needed by spgemm_symbolic + spgemm_numeric for
 * these shapes (only nrows, ncols and nnz of A and B are read).  The same
 * workspace must be passed to both calls, unchanged in between; the caller
 * owns it.  Errors: SPG_ERR_INVALID_ARG (shapes, B.nrows != A.ncols),
 * SPG_ERR_UNSUPPORTED (beyond the index range).
 */
spg_status spgemm_workspace_size(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                 const spg_csr* B, size_t* bytes);

/*
 * Symbolic phase (Gustavson, Section 2.1 definition): row analysis and
 * binning, exact nnz(C_i) per row, and the exclusive scan into C's row_ptr.
 *   c_row_ptr : device int64 [A.nrows + 1], written.
 *   c_nnz     : HOST int64, written; the call synchronises `stream` for it.
 * Errors: SPG_ERR_INVALID_ARG, SPG_ERR_WORKSPACE, SPG_ERR_CUDA, SPG_ERR_OVERFLOW.
 */
spg_status spgemm_symbolic(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                           const spg_csr* B, int64_t* c_row_ptr, int64_t* c_nnz,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * Numeric phase (Section 2.1 definition, with the (x) and (+) of the semiring,
 * Section 2.2): accumulates every product with the semiring and writes each
 * row sorted by column.  Requires the c_row_ptr and workspace of the
 * spgemm_symbolic call for the same A and B (values of A and B may differ
 * from that call; patterns may not).
 *   c_col : device int32 [nnz(C)], written.
 *   c_val : device [nnz(C)] of the output type (double, float, int64 or
 *           spg_overlap), written; ignored for SPG_SR_BOOL_OR_AND.
 * Asynchronous.  Errors found by the kernels surface in spgemm_check().
 */
spg_status spgemm_numeric(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                          const spg_csr* B, const int64_t* c_row_ptr, int32_t* c_col,
                          void* c_val, void* workspace, size_t workspace_bytes,
                          void* stream);

/*
 * Batched form: nprob independent products C_p = A_p (x).(+) B_p (1 <= nprob
 * <= 128) in one call, e.g. the uneven block products of all stages of an
 * emulated Sparse-SUMMA grid (Section 2.1).  The rows of all products are
 * binned together and each tier runs as ONE persistent launch over all of
 * them, heaviest rows first.  Arrays of nprob descriptors / pointers:
 *   c_row_ptr[p] : device int64 [A_p.nrows + 1];  c_nnz : HOST int64 [nprob].
 * Same workspace rules as the single form (spgemm_workspace_size_batched).
 * c_nnz may be NULL in spgemm_symbolic_batched: the call then queues its
 * work and returns without copying anything to the host or synchronising
 * (kernel-detected errors surface in spgemm_check); the caller has sized C
 * from an earlier call on the same patterns.  Such a call can be captured
 * in a CUDA graph together with the numeric and merge calls.
 */
spg_status spgemm_workspace_size_batched(spg_handle* handle, spg_semiring sr, int nprob,
                                         const spg_csr* A, const spg_csr* B, size_t* bytes);
spg_status spgemm_symbolic_batched(spg_handle* handle, spg_semiring sr, int nprob,
                                   const spg_csr* A, const spg_csr* B,
                                   int64_t* const* c_row_ptr, int64_t* c_nnz, void* workspace,
                                   size_t workspace_bytes, void* stream);
spg_status spgemm_numeric_batched(spg_handle* handle, spg_semiring sr, int nprob,
                                  const spg_csr* A, const spg_csr* B,
                                  const int64_t* const* c_row_ptr, int32_t* const* c_col,
                                  void* const* c_val, void* workspace, size_t workspace_bytes,
                                  void* stream);

/*
 * Merge of per-stage partial products (Sections 2.1 and 3.4):
 *     C[i,j] = P_0[i,j] (+) P_1[i,j] (+) ... (+) P_{S-1}[i,j]
 * over the entries present, folded in stage order (deterministic).  The S
 * partials (1 <= S <= 16) share C's shape; their values have the semiring's
 * OUTPUT type (spg_overlap records for the overlap semiring).
 * Two calls with the same workspace:
 *   1. c_col == NULL: writes c_row_ptr (device int64 [nrows + 1]) and c_nnz
 *      (HOST); synchronises `stream`.
 *   2. c_col != NULL: writes C.col / C.val (c_row_ptr from call 1).
 */
spg_status spgemm_merge_workspace_size(spg_handle* handle, spg_semiring sr, int nmerge,
                                       const int* nparts, const spg_csr* parts, size_t* bytes);
spg_status spgemm_merge_stages(spg_handle* handle, spg_semiring sr, int nstages,
                               const spg_csr* parts, int64_t* c_row_ptr, int64_t* c_nnz,
                               int32_t* c_col, void* c_val, void* workspace,
                               size_t workspace_bytes, void* stream);
/* Batched merges (1 <= nmerge <= 32): merge m combines parts[off_m ..
 * off_m + nparts[m]) with off_m = nparts[0] + ... + nparts[m-1].  Count call:
 * c_col == NULL (the array); c_nnz HOST [nmerge], or NULL: no host copy and
 * no synchronisation (as spgemm_symbolic_batched with c_nnz NULL).
 * Merges of at most 2^18 columns run row by row (a warp sorts rows of at
 * most 32 entries in registers; a CTA merges a longer row through a bitmap of
 * its columns) and need no copy of the partials' entries in the workspace;
 * wider ones sort every entry into its merged position. */
spg_status spgemm_merge_stages_batched(spg_handle* handle, spg_semiring sr, int nmerge,
                                       const int* nparts, const spg_csr* parts,
                                       int64_t* const* c_row_ptr, int64_t* c_nnz,
                                       int32_t* const* c_col, void* const* c_val,
                                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * Column split (the block layout of Sparse SUMMA, Section 2.1): part p keeps
 * columns [cuts[p], cuts[p+1]) of every row of M, renumbered from 0.  Row
 * blocks of a CSR are views (row_ptr + first row, same col/val base).
 *   cuts          : HOST int32 [nparts + 1], cuts[0] = 0, cuts[nparts] = ncols,
 *                   non-decreasing
 *   part_row_ptr  : device int64 [nparts * (M.nrows + 1)], part p at p*(nrows+1),
 *                   offsets relative to part p's first entry
 *   part_col/val  : device [M.nnz] (values value_bytes each), part after part
 *   part_nnz      : HOST int64 [nparts], written; synchronises `stream`.
 */
spg_status spgemm_split_workspace_size(spg_handle* handle, const spg_csr* M, int nparts,
                                       size_t* bytes);
spg_status spgemm_split_columns(spg_handle* handle, const spg_csr* M, int nparts,
                                const int32_t* cuts, int value_bytes, int64_t* part_row_ptr,
                                int32_t* part_col, void* part_val, int64_t* part_nnz,
                                void* workspace, size_t workspace_bytes, void* stream);

/* Synchronises `stream` and returns the first kernel-detected error recorded
 * in `workspace` since the last spgemm_symbolic (SPG_OK if none). */
spg_status spgemm_check(spg_handle* handle, void* workspace, void* stream);

/*
 * CSR validity check: row_ptr non-decreasing from row_ptr[0] >= 0 to
 * row_ptr[0] + nnz (row_ptr[0] > 0 for a row view), columns in [0, ncols) and
 * strictly ascending per row.  A malformed matrix is never read beyond its
 * bounds: a row whose bounds are out of range is reported without reading
 * its columns.  Synchronises `stream`.  Needs 64 bytes of workspace.  Returns
 * SPG_OK or SPG_ERR_INVALID_CSR.
 */
spg_status spgemm_validate_csr(spg_handle* handle, const spg_csr* M, void* workspace,
                               size_t workspace_bytes, void* stream);

/*
 * Optional per-stage timing with CUDA events recorded on the call's stream
 * (stages: see spgemm_get_stage_times).  enable = 0 turns it off.
 */
spg_status spgemm_set_timing(spg_handle* handle, int enable);

/*
 * Milliseconds per stage of the last spgemm_symbolic or spgemm_numeric call
 * (waits for its last event).  ms must hold SPG_STAGE_COUNT floats, indexed:
 *  1 analysis+binning  2 symbolic dense  3 symbolic block  4 symbolic warp
 *  5 scan              6 numeric binning 7 slab table      8 numeric dense
 *  9 numeric block    10 numeric warp   11 stage merge    12 learned path
 *  (0 unused)
 */
#define SPG_STAGE_COUNT 13
spg_status spgemm_get_stage_times(spg_handle* handle, float* ms, int n);

/*
 * Host-memory API: A and B in HOST memory (pinned memory makes the copies
 * asynchronous and fast; pageable memory works).  The handle uploads them
 * to device buffers it owns (kept and reused across calls, freed by
 * spgemm_destroy), runs spgemm_symbolic, and copies C's row pointers back.
 *   c_row_ptr : HOST int64 [A.nrows + 1], written;  c_nnz : HOST, written.
 * If A and B are the same host arrays, they are uploaded once.
 * Synchronous (returns when the host copies are complete).
 */
spg_status spgemm_host_symbolic(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                const spg_csr* B, int64_t* c_row_ptr, int64_t* c_nnz);

/*
 * Numeric phase of the inputs of the last spgemm_host_symbolic call on this
 * handle (same semiring); copies C.col and C.val to HOST memory.  Outputs
 * larger than spg_tuning.host_panel_bytes are computed in row panels (a
 * symbolic + numeric call per panel into one of two device buffers) and each
 * panel is downloaded on a second stream while the next one is computed.
 *   c_col : HOST int32 [nnz(C)];  c_val : HOST [nnz(C)] of the output type.
 * Synchronous; returns kernel-detected errors (as spgemm_check).
 */
spg_status spgemm_host_numeric(spg_handle* handle, spg_semiring sr, int32_t* c_col, void* c_val);

/*
 * CSR transpose T = A^T with values carried (Section 3.1: the identity
 * AB = (B^T A^T)^T; also forms A^T for C = A A^T).  Output rows are sorted.
 *   value_bytes : bytes per value to carry (0 = pattern only; 4, 8, 20, ... <= 64)
 *   t_row_ptr   : device int64 [A.ncols + 1], written
 *   t_col       : device int32 [A.nnz], written (row ids of A)
 *   t_val       : device [A.nnz * value_bytes], written (NULL if value_bytes == 0)
 * Requires A.nnz < 2^31 - 1.  Asynchronous.
 */
spg_status spgemm_transpose_workspace_size(spg_handle* handle, const spg_csr* A, size_t* bytes);
spg_status spgemm_transpose(spg_handle* handle, const spg_csr* A, int value_bytes,
                            int64_t* t_row_ptr, int32_t* t_col, void* t_val, void* workspace,
                            size_t workspace_bytes, void* stream);

/*
 * spgemm_transpose without any allocation.  The paper has no counterpart:
 * this entry point is for callers that cannot call cudaMalloc where they
 * need a transpose (inside allocation-free graph-building frameworks, custom
 * allocators' own callbacks, processes whose device memory is reserved by a
 * pool they do not own).  It runs the kernels of spgemm_transpose (same
 * arguments and output) with their scratch in a 32 MiB device array that
 * the library holds on every GPU that loads it, until the process exits.
 *   - No handle; no cudaMalloc / cudaFree or allocating library call.
 *   - Limit: 8 * A.ncols + 8 * A.nnz (plus ~8 bytes per 2048 columns and
 *     alignment) must fit in 32 MiB; larger inputs return SPG_ERR_UNSUPPORTED
 *     before any GPU work.
 *   - The first call on a device looks the array's address up (once per
 *     device, with that device current); make that first call before any
 *     stream capture.
 *   - Every call shares the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and corrupt each other; order
 *     them on one stream.  Each call clears what it needs; the array keeps
 *     the last call's contents.
 * Asynchronous on `stream`.  Errors: SPG_ERR_INVALID_ARG, SPG_ERR_UNSUPPORTED,
 * SPG_ERR_CUDA.
 */
spg_status spgemm_transpose_noalloc(const spg_csr* A, int value_bytes, int64_t* t_row_ptr,
                                    int32_t* t_col, void* t_val, void* stream);

/*
 * ---- Learned output sizing -------------------------------------------------
 * The paper sizes every output row by a symbolic pass (Section 2.1,
 * Gustavson).  Here a small network predicts r_i = nnz(C_i) / ub_i, with
 * ub_i = sum_{k in A_i} nnz(B_k) the row's product count, so that rows with a
 * small predicted output go straight to a numeric pass into a staging area of
 * capacity cap_i and skip the symbolic pass.  A row that finds more distinct
 * columns than cap_i stops and is redone by the exact symbolic + numeric
 * kernels: C is always exactly the C of spgemm_symbolic + spgemm_numeric
 * (bit-identical for every semiring but the floating plus-times ones, whose
 * atomic summation order is free).  Single products only (no batches).
 *
 * Network (spgemm_mlp_*): features f_i = log1p of (nnz(A_i), ub_i,
 * max_k nnz(B_k), mean_k nnz(B_k)); 4 -> 64 -> 64 -> 1, ReLU, r = sigmoid(z).
 * Parameters: SPGEMM_MLP_PARAMS values in the order W1[64][4] b1[64]
 * W2[64][64] b2[64] W3[64] b3 (row-major, W[out][in]); BF16 on the device for
 * inference, FP32 master copy for training.  Features, hidden activations
 * and weights are rounded to BF16; every sum accumulates in FP32.
 */
#define SPGEMM_MLP_PARAMS 4545

typedef struct {
    const void* model;     /* device BF16 [SPGEMM_MLP_PARAMS], or NULL: cap_i = min(ub_i, ncols)
                              (the "ub-sized" path: no prediction)                               */
    float margin;          /* cap_i = ceil(ub_i * r_i * margin), clamped to [1, min(ub_i, ncols)];
                              <= 0: 1.0                                                           */
    int64_t exact_max_ub;  /* rows with ub_i <= this use cap_i = min(ub_i, ncols) (0: 32); the
                              network runs only on the other rows                              */
    int64_t learned_max;   /* rows with cap_i above this take the exact path (0: 2048; clamped to
                              what one CTA's shared-memory table holds for the semiring)         */
    int64_t reserved[4];
} spg_learned_opts;

/*
 * Workspace of the learned path: the plain path's workspace plus about 30
 * bytes per row of A.  The same workspace goes to the plan, symbolic and numeric
 * calls, unchanged in between.
 */
spg_status spgemm_learned_workspace_size(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                         const spg_csr* B, size_t* bytes);

/*
 * Step 1: row features, network inference, capacities and staging offsets.
 *   opts          : HOST, may be NULL (all defaults, no model)
 *   staging_bytes : HOST, written: bytes of the staging buffer that steps 2
 *                   and 3 need (columns + values of sum cap_i entries).
 * Synchronises `stream`.
 */
spg_status spgemm_learned_plan(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                               const spg_csr* B, const spg_learned_opts* opts, void* workspace,
                               size_t workspace_bytes, size_t* staging_bytes, void* stream);

/*
 * Step 2: learned rows accumulate into staging; overflowing and large rows
 * run the exact symbolic pass; all counts are scanned into C's row pointers.
 *   c_row_ptr : device int64 [A.nrows + 1], written;  c_nnz : HOST, written.
 *   staging   : device buffer of at least staging_bytes (from step 1).
 * Synchronises `stream`.  spgemm_get_stats then reports learned_rows,
 * overflow_rows and staging_entries.
 */
spg_status spgemm_learned_symbolic(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                   const spg_csr* B, int64_t* c_row_ptr, int64_t* c_nnz,
                                   void* workspace, size_t workspace_bytes, void* staging,
                                   size_t staging_bytes, void* stream);

/*
 * Step 3: learned rows are copied from staging into C; the other rows run the
 * plain numeric kernels.  Output arguments as spgemm_numeric.  A and B must
 * be those of steps 1-2, unchanged (learned rows' values were computed in
 * step 2).  Asynchronous.
 */
spg_status spgemm_learned_numeric(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                  const spg_csr* B, const int64_t* c_row_ptr, int32_t* c_col,
                                  void* c_val, void* workspace, size_t workspace_bytes,
                                  const void* staging, size_t staging_bytes, void* stream);

/*
 * Row features of C = A B for the network: feat device float [A.nrows][4];
 * ub device int64 [A.nrows] (product count per row) or NULL.  feat must be
 * 16-byte aligned.  Asynchronous.
 * workspace: any workspace valid for spgemm_symbolic of A and B (only its
 * head, the product descriptor, is written).
 */
spg_status spgemm_row_features(spg_handle* handle, const spg_csr* A, const spg_csr* B,
                               float* feat, int64_t* ub, void* workspace, size_t workspace_bytes,
                               void* stream);

/* Inference: z device float [n] = network output (logit of r) for feat [n][4]. */
spg_status spgemm_mlp_forward(spg_handle* handle, const float* feat, int64_t n,
                              const void* params_bf16, float* z, void* stream);

/*
 * Training step pieces.  Loss (mean over the n rows) is the pinball loss of
 * quantile tau on log r:  u = log_target - log sigmoid(z),
 * L = tau * u if u > 0 else (tau - 1) * u.
 *   spgemm_mlp_grad : grad device float [SPGEMM_MLP_PARAMS] = dL/dparams (at the
 *                     BF16 weights), loss device float [1]; workspace of
 *                     spgemm_mlp_train_workspace_size(n) bytes.
 *   spgemm_mlp_adam : one Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step
 *                     counts from 1) on FP32 master weights, m, v (device
 *                     float [SPGEMM_MLP_PARAMS] each), refreshing the BF16 copy.
 *   spgemm_mlp_to_bf16 : BF16 copy of FP32 master weights.
 * Asynchronous.
 */
size_t spgemm_mlp_train_workspace_size(int64_t n);
spg_status spgemm_mlp_grad(spg_handle* handle, const float* feat, const float* log_target,
                           int64_t n, float tau, const void* params_bf16, float* grad,
                           float* loss, void* workspace, size_t workspace_bytes, void* stream);
spg_status spgemm_mlp_adam(spg_handle* handle, float* master, float* m, float* v,
                           const float* grad, void* params_bf16, float lr, int step, void* stream);
spg_status spgemm_mlp_to_bf16(spg_handle* handle, const float* master, void* params_bf16,
                              void* stream);

/*
 * Masked product: C = (A (x).(+) B) restricted to the pattern of a mask M
 * (M.nrows = A.nrows, M.ncols = B.ncols, columns ascending per row, values
 * ignored): C[i,j] is present iff (i,j) is in M and at least one product
 * A[i,k] (x) B[k,j] exists; its value is the (+) of those products (the
 * Section 2.1 definition on M's positions).  Each mask entry owns an
 * accumulator in the workspace (masked_workspace_size: about
 * nnz(M) * (slot + 1) bytes), so the work follows the products and the mask,
 * not nnz(A B).
 *   spgemm_masked_symbolic: accumulates every product that falls on M and
 *     writes C's row pointers (device int64 [A.nrows + 1]); c_nnz HOST,
 *     synchronises `stream`.
 *   spgemm_masked_numeric: writes C.col / C.val from the accumulators of the
 *     symbolic call (same workspace, same A, B, M).  Asynchronous.
 */
spg_status spgemm_masked_workspace_size(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                        const spg_csr* B, const spg_csr* M, size_t* bytes);
spg_status spgemm_masked_symbolic(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                  const spg_csr* B, const spg_csr* M, int64_t* c_row_ptr,
                                  int64_t* c_nnz, void* workspace, size_t workspace_bytes,
                                  void* stream);
spg_status spgemm_masked_numeric(spg_handle* handle, spg_semiring sr, const spg_csr* A,
                                 const spg_csr* B, const spg_csr* M, const int64_t* c_row_ptr,
                                 int32_t* c_col, void* c_val, void* workspace,
                                 size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_H */
