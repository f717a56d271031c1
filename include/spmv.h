/*
 * spmv.h -- C ABI of the GB300 (sm_103a) SpMV engine.
 *
 * The operation is the sparse matrix-vector product of Section 2.2 of
 * Auto-SpMV (arXiv 2302.05662), Y = A X, extended with the BLAS scalars:
 *
 *     y <- alpha * A * x + beta * y
 *
 * for a sparse m x n matrix A held on the GPU in one of the storage formats
 * of Section 2.3 (CSR, ELL, and a blocked format -- here BSR, the row-block
 * form of the paper's BELL) or in COO and HYB (ELL + COO), and the kernel
 * and launch parameters of Section 4 (thread-block size, register cap,
 * L1/shared-memory split) plus threads-per-row and unroll form the tuned
 * space.  The matrix arrives as COO triplets, the form the paper's input
 * collection ships in (Section 7.5), and is converted on the device.
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  All device work is ordered on that stream.  Calls that must
 *     learn a size on the host (create, set_config, features, select)
 *     synchronise that stream once; spmv_run never synchronises (except in
 *     the checked mode below).
 *   - Every function returns an spmv_status (0 = success).  On failure
 *     spmv_last_error() returns a message for the calling thread.  No C++
 *     exception or process exit crosses this boundary.
 *   - Value types: SPMV_F64 values use double x and y and accumulate in
 *     double; SPMV_F32 and SPMV_BF16 values use float x and y and
 *     accumulate in float.  Indices are int32 (m, n < 2^31, nnz < 2^31).
 *   - A handle is not thread-safe; runs on one handle must be ordered on
 *     one stream (they share the handle's reduction scratch).
 *   - Checked products (a debug mode): with the environment variable
 *     SPMV_CHECKED=1, spmv_run first verifies every stored index of the
 *     active format against the matrix bounds (one extra pass and a
 *     synchronisation of `stream`); a bad index sets the handle's status
 *     word and spmv_run returns SPMV_ERR_BOUNDS without launching the
 *     product.  Unset (the default), spmv_run does no such pass.
 *   - Fault injection (for testing callers' error paths): with the
 *     environment variable SPMV_FAULT_ALLOC=k (k >= 1), the k-th device
 *     allocation made inside each call fails as if the device were out of
 *     memory; the call returns SPMV_ERR_OOM after releasing what it had
 *     allocated.  Unset (the default), nothing is injected.
 */
#ifndef SPMV_GB300_SPMV_H
#define SPMV_GB300_SPMV_H

#include <stdint.h>

#if defined(__GNUC__)
#define SPMV_API __attribute__((visibility("default")))
#else
#define SPMV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmv_matrix *spmv_handle;

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID = -1,     /* bad argument or triplet out of range     */
    SPMV_ERR_OOM = -2,         /* device allocation failed                 */
    SPMV_ERR_CUDA = -3,        /* a CUDA runtime call failed               */
    SPMV_ERR_UNSUPPORTED = -4, /* valid but not supported (e.g. ELL width) */
    SPMV_ERR_BOUNDS = -5,      /* a checked kernel skipped an out-of-range
                                  index (spmv_check)                       */
    SPMV_ERR_TIMEOUT = -6      /* a kernel gave up waiting for a copy
                                  (spmv_check)                             */
} spmv_status;
/* Out-of-range triplets are found by a device check in spmv_create and
 * reported as SPMV_ERR_INVALID.  No kernel spins on another work unit: rows
 * shared by work units are joined by whichever unit arrives last, the
 * batched kernel takes work from one atomic counter, and conjugate
 * gradients stop through a graph conditional node.  The one wait on the
 * device is for the copy engine: the staged CSR kernel waits on a shared-
 * memory barrier for each bulk copy, for at most one second, after which it
 * records a timeout in the handle's device status word and returns; the
 * asynchronous spmv_run cannot report it, spmv_check does. */

typedef enum { SPMV_F64 = 0, SPMV_F32 = 1, SPMV_BF16 = 2 } spmv_dtype;

typedef enum {
    SPMV_FMT_CSR = 0, /* Section 2.3: Data, Column Index, Row Index        */
    SPMV_FMT_ELL = 1, /* Section 2.3: m x max_nnz padded, column-major     */
    SPMV_FMT_COO = 2, /* (row, col, val) triplets sorted by row            */
    SPMV_FMT_HYB = 3, /* ELL part + COO overflow                           */
    SPMV_FMT_BSR = 4, /* r x r dense blocks (blocked format of Sec. 2.3)   */
    SPMV_FMT_SELL = 5 /* sliced ELL, 32-row slices of rows sorted by      */
                      /* descending length (Sec. 2.3 SELL)                 */
} spmv_format;

/* threads_per_row value that selects the nnz-balanced CSR kernels (Sec. 2.3:
 * CSR's load imbalance on uneven rows).  Two forms, chosen by hyb_ell_width:
 * warp chunks (0, the default): chunks of 4 x unroll x 32 nonzeros, one warp
 * each, a lane summing 4 x unroll consecutive entries, the rows recovered
 * from the row pointers (no row index per entry) and joined across lanes and
 * chunks; or staged tiles (hyb_ell_width nonzeros per tile): each tile
 * bulk-copied into shared memory while the thread block multiplies the
 * previous one, rows summed by groups of lanes (1..8 from the mean row
 * length) and joined across tiles. */
#define SPMV_TPR_SPLIT (-1)

/*
 * Kernel and launch parameters (Section 4, items 1-3, plus the format of
 * item 4).  A zero field takes the library default.
 *   format            spmv_format.
 *   threads_per_block 32..1024, a power of two (default 256).
 *   threads_per_row   CSR: lanes cooperating on one row, 1/2/4/8/16/32, or
 *                     SPMV_TPR_SPLIT for the nnz-balanced split (default:
 *                     the largest power of two up to 32 that leaves each
 *                     lane at least 8 entries of a mean-length row).  BSR: blocks handled at once per block row,
 *                     1/2/4/8 (default 1).  Ignored by ELL, COO, HYB and
 *                     SELL (one lane per row).
 *   unroll            1, 2 or 4 (8 also for ELL, HYB and SELL): loads in
 *                     flight per lane (ELL, SELL, CSR) or items per lane / 4
 *                     (COO, HYB tail, split CSR; at most 16 items).  0 =
 *                     default: ELL and HYB 2 with fp64 values, 4 with
 *                     fp32/bf16; SELL 8 (1 with fp64 values in the
 *                     column-major layout); every other format 2.
 *   regcap            register cap per thread, 32 (the paper's
 *                     maxrregcount knob) or 64 (the ceiling that keeps
 *                     1024-thread blocks launchable); 48 also for ELL, HYB
 *                     and SELL.  0 = default: 32 for ELL and HYB with fp64
 *                     values, 64 otherwise.
 *   carveout          preferred shared-memory carveout in percent (0..100),
 *                     or -1 to leave the driver default (Section 4 item 3).
 *                     Zero means 0 % (maximum L1), not "default".
 *   bsr_block         BSR block size r: 2 or 4 (default 4).  SELL: column
 *                     groups, 4 (a lane's four entries of four consecutive
 *                     columns side by side: 16-byte loads) or 1 (column-
 *                     major); 0 = 4 unless the longest row exceeds 32 mean
 *                     rows plus 32 (power-law rows: mostly narrow slices,
 *                     where column-major runs faster) or, with fp64 values,
 *                     fewer than a quarter of consecutive stored entries
 *                     have consecutive columns (scattered columns), then 1.
 *                     CSR with 1
 *                     or 2 lanes per row: entries per lane load, 8 (32-byte
 *                     loads) or 4 (16-byte loads); 0 = 8 when a lane's part
 *                     of a mean-length row holds 16 or more entries, else 4
 *                     (wider groups mask more slots at a part's ends).
 *   hyb_ell_width     HYB ELL width; 0 applies the width rule (the largest
 *                     k such that at least max(4096, m/3) rows hold k or
 *                     more nonzeros).  SELL: columns of a slice per work
 *                     item, a multiple of 4 in 8..65536 (0 = 128); wider
 *                     slices are split into several items joined in order.  CSR with
 *                     SPMV_TPR_SPLIT: 0 = warp chunks, else nonzeros per
 *                     tile staged through shared memory, a multiple of 256
 *                     in [256, 8192].
 * spmv_config_default() fills the defaults (carveout = -1; unroll and
 * regcap 0, resolved per format and value type when the configuration is
 * applied; spmv_get_config returns the resolved values).
 */
typedef struct {
    int32_t format;
    int32_t threads_per_block;
    int32_t threads_per_row;
    int32_t unroll;
    int32_t regcap;
    int32_t carveout;
    int32_t bsr_block;
    int32_t hyb_ell_width;
} spmv_config;

/* Sizes of a handle's matrix and of its active format. */
typedef struct {
    int64_t m, n;
    int64_t nnz;          /* stored entries after merging duplicate pairs  */
    int64_t max_row;      /* longest row                                   */
    int64_t ell_width;    /* ELL width (ELL), or ELL-part width (HYB)      */
    int64_t hyb_coo_nnz;  /* entries in the HYB COO part                   */
    int64_t bsr_blocks;   /* nonzero r x r blocks (BSR)                    */
    int64_t sell_slots;   /* stored entries incl. padding (SELL)           */
    int64_t format_bytes; /* device bytes the active format's kernel reads */
    int32_t value_type;   /* spmv_dtype                                    */
    int32_t format;       /* active spmv_format                            */
    int32_t panels;       /* row panels the matrix is held in (>= 1)       */
    int32_t reserved;
} spmv_info;

/* Fills *cfg with the library defaults for `format` (carveout = -1; unroll
 * and regcap 0, resolved when the configuration is applied). */
SPMV_API void spmv_config_default(spmv_config *cfg, int32_t format);

/*
 * Build a matrix handle from COO triplets on the device (Section 5.3, step
 * 4: conversion from the input COO to the chosen format; Section 7.5: the
 * input is COO).  d_rows[k], d_cols[k], d_vals[k] (k < nnz) give entry
 * (row, col, value); the triplets may come in any order and may repeat a
 * (row, col) pair, whose values are then summed in triplet order.  Values
 * are of `value_type` (double, float or bf16 bits).  The triplet arrays are
 * borrowed for the duration of the call only; the handle owns copies in
 * the converted format.  `cfg` (may be NULL = default CSR) selects the
 * active format and kernel.  m, n may be 0; nnz may be 0.
 * Errors: SPMV_ERR_INVALID for negative sizes, a NULL array with nnz > 0,
 * or any triplet outside [0,m) x [0,n) (checked on the device);
 * SPMV_ERR_UNSUPPORTED for m or n >= 2^31 or a format whose padded
 * storage exceeds 8 nnz + 2^24 value slots (ELL width x rows; BSR blocks x
 * r^2; SELL slices x 32 x slice width); SPMV_ERR_OOM; SPMV_ERR_CUDA.
 * Synchronises `stream`.
 */
SPMV_API int spmv_create(spmv_handle *out, int64_t m, int64_t n, int64_t nnz,
                const int32_t *d_rows, const int32_t *d_cols,
                const void *d_vals, int32_t value_type,
                const spmv_config *cfg, void *stream);

/*
 * Switch the active format and kernel parameters (Section 5.3 step 4, the
 * re-pack once a better format is chosen; Section 5.2, the compile-time
 * parameters, here pre-built kernel variants).  Packs the new format from
 * the handle's CSR arrays on the device; frees the previous non-CSR arrays.
 * Errors as for spmv_create.  Synchronises `stream`.
 */
SPMV_API int spmv_set_config(spmv_handle h, const spmv_config *cfg, void *stream);

/* Copies the active (resolved, defaults filled) configuration. */
SPMV_API int spmv_get_config(spmv_handle h, spmv_config *out);

/* Copies the handle's sizes into *out. */
SPMV_API int spmv_get_info(spmv_handle h, spmv_info *out);

/*
 * y <- alpha * A * x + beta * y (Section 2.2), using the active format.
 * d_x holds n values and d_y m values, of type double (SPMV_F64) or float
 * (SPMV_F32, SPMV_BF16); both are caller-owned device buffers, and x must
 * not overlap y.  beta == 0 means y is not read (NaN in y is ignored).
 * One or two kernel launches on `stream` per row panel (one panel unless
 * the matrix has more triplets than the panel limit); never synchronises.
 * Errors: SPMV_ERR_INVALID for a NULL handle or a NULL vector with a
 * nonzero size; SPMV_ERR_CUDA if a launch fails; SPMV_ERR_BOUNDS in the
 * checked mode (SPMV_CHECKED=1) when a stored index is out of bounds.
 */
SPMV_API int spmv_run(spmv_handle h, double alpha, const void *d_x, double beta,
             void *d_y, void *stream);

/* Array ids for spmv_export / spmv_export_bytes (test and debug access). */
typedef enum {
    SPMV_ARR_CSR_ROWPTR = 0,  /* int32[m+1]                                  */
    SPMV_ARR_CSR_COLIDX = 1,  /* int32[nnz]                                  */
    SPMV_ARR_CSR_VALS = 2,    /* value_type[nnz]                             */
    SPMV_ARR_ELL_COLIDX = 3,  /* int32[width][pitch], -1 = padding           */
    SPMV_ARR_ELL_VALS = 4,    /* value_type[width][pitch], 0 = padding       */
    SPMV_ARR_COO_ROWS = 5,    /* int32[nnz] (COO) or int32[coo_nnz] (HYB)    */
    SPMV_ARR_COO_COLS = 6,    /* int32[...] as above                         */
    SPMV_ARR_COO_VALS = 7,    /* value_type[...] as above                    */
    SPMV_ARR_BSR_ROWPTR = 8,  /* int32[ceil(m/r)+1]                          */
    SPMV_ARR_BSR_COLIDX = 9,  /* int32[blocks]: block column                 */
    SPMV_ARR_BSR_VALS = 10,   /* value_type[blocks][r][r], row-major blocks  */
    SPMV_ARR_ELL_PITCH = 11,  /* (size query only) pitch in elements          */
    SPMV_ARR_SELL_PTR = 12,   /* int32[slices+1]: first slot of each slice     */
    SPMV_ARR_SELL_COLIDX = 13,/* int32[slots]: slice s of width w, entry k,    */
                              /* lane l at ptr[s] + 128 (k/4) + 4 l + k%4 for  */
                              /* k < (w & ~3), else at ptr[s] + 32 (w & ~3) +   */
                              /* 32 (k - (w & ~3)) + l; -1 = padding            */
    SPMV_ARR_SELL_VALS = 14,  /* value_type[slots], 0 = padding                */
    SPMV_ARR_SELL_PERM = 15   /* int32[m]: matrix row held by sorted row p     */
                              /* (rows sorted by descending length, stable)    */
} spmv_array_id;

/*
 * Size in bytes of an internal array of the active format (0 if the format
 * does not hold it).  For SPMV_ARR_ELL_PITCH, *bytes receives the pitch in
 * elements instead.
 */
SPMV_API int spmv_export_bytes(spmv_handle h, int32_t array_id, int64_t *bytes);

/*
 * Copy an internal array (see spmv_array_id) into the caller's device
 * buffer d_dst of `bytes` bytes (must equal spmv_export_bytes).  Stream-
 * ordered device-to-device copy.  For tests of the conversions.
 */
SPMV_API int spmv_export(spmv_handle h, int32_t array_id, void *d_dst, int64_t bytes,
                void *stream);

/*
 * Largest nnz spmv_coo_run_noalloc accepts (2^25).  Its scratch is one fixed
 * device array of about 4.5 MiB, compiled into the library, that every GPU
 * which loads the library holds until the process exits.
 */
#define SPMV_NOALLOC_MAX_NNZ 33554432

/*
 * y <- alpha * A * x + beta * y for a matrix given as COO triplets sorted by
 * row, without allocating any device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * running inside another library's memory pool or callback, real-time or
 * embedded code that may not allocate after start-up, or processes whose
 * device allocator is exhausted or off limits.  It runs the segmented-
 * reduction COO kernel straight on the caller's arrays and keeps the
 * kernel's scratch (per-chunk metadata, partial row sums, arrival counters
 * and exchange slots) in the library's fixed device array instead of in
 * allocated memory.
 *
 * d_rows, d_cols, d_vals hold nnz triplets with rows in nondecreasing order
 * (columns in any order; repeated pairs are summed), values of value_type;
 * d_x has n entries and d_y m entries (double for SPMV_F64, else float).
 * d_rows, d_cols and d_vals must start on 16-byte boundaries (the kernel
 * reads them with 16-byte vector loads; cudaMalloc'd arrays and tensors
 * that start their storage always do, a view that starts mid-array may not).
 * All arrays stay owned by the caller.  beta == 0 means y is not read.
 *
 * Errors: SPMV_ERR_UNSUPPORTED when nnz > SPMV_NOALLOC_MAX_NNZ, m or n >=
 * 2^31, or `stream` is being captured into a graph; SPMV_ERR_INVALID for
 * bad sizes, NULL arrays, triplet arrays not 16-byte aligned (checked on
 * the host, nothing launched), or triplets that are out of range or not
 * sorted by row (checked on the device before any product is formed); in
 * every error case y is left unchanged; SPMV_ERR_CUDA.
 *
 * A call with nnz > 0 synchronises `stream` once, to read the triplet
 * check.  The first call on a device does the set-up: it looks up the
 * device address of the fixed array on that device (once per device, with
 * the device current; the address is kept for the life of the process, so
 * do not use this entry point on a device after cudaDeviceReset), and the
 * CUDA driver loads the library's kernels then if it has not yet done so;
 * make that first call before any stream capture.  Later calls allocate
 * nothing.  Every call shares the one array, and each call clears the parts
 * that must start at zero, so calls are correct one after another; calls
 * whose kernels overlap on the GPU (other threads, other streams) race on
 * the array and give wrong results.
 */
SPMV_API int spmv_coo_run_noalloc(int64_t m, int64_t n, int64_t nnz,
                                  const int32_t *d_rows, const int32_t *d_cols,
                                  const void *d_vals, int32_t value_type,
                                  double alpha, const void *d_x, double beta,
                                  void *d_y, void *stream);

/* Number of sparsity features spmv_features / spmv_select produce. */
#define SPMV_NUM_FEATURES 20

/*
 * Sparsity features of the handle's matrix (Section 5.5, Table 2, plus the
 * selector's structural extras), computed on the device from the CSR
 * arrays and copied to h_out[SPMV_NUM_FEATURES] (host), in this order:
 *   0 n (rows)  1 nnz  2 density nnz/(m n)  3 mean row length (Avg_nnz)
 *   4 population variance of row lengths (Var_nnz)  5 its square root
 *   (Std_nnz)  6 min  7 max row length  8 median (lower middle)  9 mode
 *   (smallest on ties)  10 ELL_ratio nnz/(m max)  11 Gini coefficient of
 *   row lengths  12 coefficient of variation  13 fraction of empty rows
 *   14 bandwidth max|i-j|  15 mean |i-j|  16 fraction of diagonal entries
 *   17 4x4 block fill nnz/(16 blocks)  18 2x2 block fill  19 fraction of
 *   nonzeros beyond the HYB ELL width.
 * Ratios with a zero denominator are 0.  Synchronises `stream`.
 */
SPMV_API int spmv_features(spmv_handle h, double *h_out, void *stream);

/*
 * Load the selector: a 2-layer MLP classifier (Section 5.4: one classifier
 * mapping features to the best configuration) for the current device.
 * h_blob holds `count` floats: magic 2302, version (1 or 2), F (= 20), H,
 * K; then mu[F], sigma[F] (input standardisation after log1p of the
 * count-like features 0,1,3-9,14,15), W1[H][F], b1[H], W2[K][H], b2[K];
 * then K label configurations of 8 values each (the spmv_config fields in
 * order; 0 = library default).  Version 2 appends the time head W3[K+1][H],
 * b3[K+1] (natural log of microseconds per product for each label class,
 * then for default CSR, linear in the hidden layer) and the conversion-cost
 * model: for each format 0..5, {a, b, c} with cost a + b nnz + c m in
 * microseconds.
 * H <= 256, K <= 512.  Copies the weights to the device.  A NULL blob with
 * count 0 unloads the selector.  Errors: SPMV_ERR_INVALID for a malformed
 * blob.
 */
SPMV_API int spmv_selector_load(const float *h_blob, int64_t count);

/*
 * Load a selector for handles of one value type only (SPMV_F64, SPMV_F32,
 * SPMV_BF16), in the blob format above: spmv_select and spmv_select_runtime
 * on a handle of that type use it, and the one spmv_selector_load loaded
 * for the other types (labels measured on one value type need not carry to
 * another: on GB300 fp64 products are bound by the fp64 pipe as much as by
 * HBM).  A NULL blob with count 0 unloads it.  spmv_selector_infer uses the
 * shared selector only.  Errors: SPMV_ERR_INVALID for an unknown value type
 * or a malformed blob.
 */
SPMV_API int spmv_selector_load_vt(int32_t value_type, const float *h_blob, int64_t count);

/*
 * Run the selector's fused inference kernel on host features (20 doubles):
 * writes the chosen class to *choice and, when h_logits is not NULL, the K
 * output logits (fp32).  Synchronises `stream`.  SPMV_ERR_INVALID if no
 * selector is loaded on the current device.
 */
SPMV_API int spmv_selector_infer(const double *h_features, float *h_logits,
                                 int32_t *choice, void *stream);

/*
 * Pick the format and kernel parameters for the handle's matrix (Section
 * 5.3 steps 1-2): features on the device, then the loaded selector's fused
 * inference kernel; *out_cfg receives the chosen label configuration, or
 * the default CSR configuration when no selector is loaded.  The features
 * are also copied to h_features (may be NULL).  Does not change the handle;
 * apply the choice with spmv_set_config.  Synchronises `stream`.
 */
SPMV_API int spmv_select(spmv_handle h, spmv_config *out_cfg, double *h_features,
                         void *stream);

/*
 * Batched SpMV (a batch of independent products y_i <- alpha_i A_i x_i +
 * beta_i y_i in one persistent launch).  The paper runs one kernel per
 * matrix; a batch of hundreds of uneven matrices would then pay one launch
 * each.  A batch plan holds, for every matrix, a mode and a list of warp
 * work items over all matrices that a grid of resident thread blocks
 * consumes through one atomic counter.  A matrix whose handle holds ELL or
 * SELL runs in that format (ELL: 32 rows per item, a row per lane; SELL:
 * the handle's work items; mode -1 and -5), a COO handle as COO chunks of
 * 32*items entries per warp (mode -2) and a BSR handle as groups of 32 / r
 * block rows with r lanes each (mode -4), unless the tuner finds a CSR mode
 * faster; any other handle runs from its CSR arrays as nonzero chunks of
 * 32*items entries per warp (split, mode 0) or 32-row groups with 1..32
 * lanes per row (vector, mode = lanes per row).
 * The counter reset and the kernel are captured in a CUDA graph.
 *
 * spmv_batch_create: hs[i] (all of one value type), alpha[i], beta[i] (host
 * arrays) and device vectors d_x[i] (n_i entries), d_y[i] (m_i entries), i <
 * count.  The plan reads the handles' arrays (and a SELL handle's join
 * scratch): the handles and vectors must outlive the plan, keep their
 * addresses and formats, and not run other products while the plan does.  Default modes come from
 * row-length statistics.  Synchronises `stream`.
 * spmv_batch_tune: autotuner -- times every CSR mode (and COO chunks or BSR
 * block rows for a COO or BSR handle) per matrix, each on one launch over enough copies of the
 * matrix to fill the GPU (about 4M entries), then the chunk size (items 4/8/16) and block size
 * (128/256/512) on the whole batch, keeps the fastest and re-captures the
 * graph.  Overwrites y.  Synchronises `stream`.
 * spmv_batch_launch: replays the graph on `stream` (no synchronisation).
 * spmv_batch_get_plan: copies the per-matrix modes (0 = split, lanes per
 * row for vector CSR, -1 ELL, -2 COO chunks, -4 BSR, -5 SELL; h_modes may be
 * NULL), the items and
 * the block size.
 * spmv_batch_run: create + launch + destroy in one call (synchronises).
 * Errors: SPMV_ERR_INVALID (NULL arrays or handles, mixed value types),
 * SPMV_ERR_UNSUPPORTED (a handle held in row panels), SPMV_ERR_OOM,
 * SPMV_ERR_CUDA.
 */
typedef struct spmv_batch *spmv_batch_handle;

SPMV_API int spmv_batch_create(spmv_batch_handle *out, const spmv_handle *hs,
                               int32_t count, const double *alpha,
                               const void *const *d_x, const double *beta,
                               void *const *d_y, void *stream);
SPMV_API int spmv_batch_tune(spmv_batch_handle b, void *stream);
SPMV_API int spmv_batch_launch(spmv_batch_handle b, void *stream);
SPMV_API int spmv_batch_get_plan(spmv_batch_handle b, int32_t *h_modes,
                                 int32_t *items, int32_t *threads_per_block);
SPMV_API int spmv_batch_destroy(spmv_batch_handle b);
SPMV_API int spmv_batch_run(const spmv_handle *hs, int32_t count,
                            const double *alpha, const void *const *d_x,
                            const double *beta, void *const *d_y, void *stream);

/*
 * Run-time mode decision (Section 5.3 steps 3-4: estimate the optimisation
 * overhead, convert only if the predicted benefit is larger).
 */
typedef struct {
    int32_t convert;               /* 1: converting pays off over expected_runs */
    int32_t current_class;         /* label class of the handle's configuration,
                                      -1 when it is default CSR (own time head) */
    int32_t selected_class;        /* label class the classifier picks          */
    int32_t pad;
    double predicted_us_current;   /* predicted time of one product, now        */
    double predicted_us_selected;  /* ... in the selected configuration         */
    double predicted_pack_us;      /* predicted conversion (re-pack) time       */
    double measured_select_us;     /* features + inference, measured            */
} spmv_runtime_decision;

/*
 * Like spmv_select, plus the decision: with a version-2 selector (time head
 * predicting the log-time of every label configuration and of default CSR,
 * and a per-format conversion-cost model a + b nnz + c m), *out->convert is
 * 1 when (predicted current time - predicted selected time) x expected_runs
 * exceeds the measured feature + inference time plus the predicted
 * conversion time.  The handle is not changed; apply *out_cfg with
 * spmv_set_config when convert is 1.  Errors: SPMV_ERR_INVALID without a
 * version-2 selector.  Synchronises `stream`.
 */
SPMV_API int spmv_select_runtime(spmv_handle h, int64_t expected_runs,
                                 spmv_config *out_cfg, spmv_runtime_decision *out,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * Conjugate gradients with the handle's SpMV.  Section 7.5 names the
 * (preconditioned) conjugate gradient method as the iterative setting in
 * which one matrix is multiplied many times, so feature extraction,
 * selection and conversion are paid once.  The iteration is Hestenes and
 * Stiefel's, unpreconditioned:
 *   r_0 = b - A x_0, p_0 = r_0, rho_k = r_k.r_k;
 *   while k < maxit and rho_k > tol^2 (b.b):
 *     q = A p_k; stop with breakdown = 1 if p_k.q <= 0;
 *     alpha = rho_k / (p_k.q); x += alpha p_k; r -= alpha q;
 *     p_{k+1} = r_{k+1} + (rho_{k+1} / rho_k) p_k.
 * A must be square and symmetric positive definite; every product runs in
 * the handle's current format and configuration.
 *
 * d_b: device, m entries (double for SPMV_F64 handles, float otherwise),
 *      read only.  d_x: device, same type; in: x_0, out: the last iterate.
 * d_rho: NULL, or device double[maxit + 1] receiving rho_0 .. rho_iterations.
 * Dot products accumulate in fp64 in a fixed order (repeat calls are
 * bit-identical).  The whole loop is one CUDA graph whose WHILE node the
 * device stops: no host round trip per iteration.  The handle keeps the
 * graph and three m-vectors of scratch for the next call with the same
 * (d_b, d_x, tol, maxit); spmv_set_config and spmv_destroy release them.
 * Synchronises `stream`, then fills *out.
 * Errors: SPMV_ERR_INVALID (NULL handle/result/vector, m != n, tol < 0 or
 * not finite, maxit < 0 or > SPMV_CG_MAX_ITERATIONS), SPMV_ERR_CUDA.
 * ------------------------------------------------------------------------- */
#define SPMV_CG_MAX_ITERATIONS 16777216

typedef struct {
    int32_t iterations;  /* products A p_k performed */
    int32_t converged;   /* rho_iterations <= tol^2 (b.b) */
    int32_t breakdown;   /* stopped on p_k.A p_k <= 0 (A not SPD) */
    int32_t reserved;
    double rho0;         /* r_0.r_0 */
    double rho;          /* r.r at exit (the recursively updated residual) */
    double bb;           /* b.b */
} spmv_cg_result;

SPMV_API int spmv_cg(spmv_handle h, const void *d_b, void *d_x, double tol,
                     int32_t maxit, double *d_rho, spmv_cg_result *out,
                     void *stream);

/* ---------------------------------------------------------------------------
 * Row panels.  One handle indexes its nonzeros with int32 offsets, so a
 * matrix given with more triplets than the panel limit is held as several
 * sub-handles over contiguous row ranges (boundaries at multiples of 4 rows,
 * each range with at most `limit` triplets); spmv_run, spmv_set_config,
 * spmv_features, spmv_select(_runtime) and spmv_cg treat it as one matrix
 * (features and results as for a single handle; each panel runs its own
 * kernels on its rows of y).  spmv_export and spmv_batch_create refuse a
 * panelled handle (SPMV_ERR_UNSUPPORTED), and so does spmv_create when four
 * consecutive rows alone hold more than `limit` triplets.  The default and
 * largest limit, SPMV_PANEL_LIMIT_MAX = 2^31 - 2^20, keeps every offset and
 * loop counter of a panel's kernels inside int32 with headroom; a smaller
 * limit (process-wide, for handles created afterwards) exercises panels on
 * small matrices or bounds the conversion scratch.
 * Errors: SPMV_ERR_INVALID for a limit outside [1, SPMV_PANEL_LIMIT_MAX].
 * ------------------------------------------------------------------------- */
#define SPMV_PANEL_LIMIT_MAX 2146435072LL
SPMV_API int spmv_set_panel_limit(int64_t max_triplets);
SPMV_API int64_t spmv_get_panel_limit(void);

/*
 * Reads and clears the handle's device status word (no counterpart in the
 * paper).  Kernels launched by spmv_run cannot return a status to the host,
 * so a kernel that gives up waiting for a bulk copy (one second; the staged
 * CSR kernel) records it in a word on the device, as does a kernel that
 * finds and skips an out-of-range index.  spmv_check synchronises `stream`,
 * then returns SPMV_ERR_BOUNDS or SPMV_ERR_TIMEOUT if any product since the
 * last check recorded one (the products concerned are incomplete), else
 * SPMV_OK.  Errors: SPMV_ERR_INVALID (NULL handle), SPMV_ERR_CUDA.
 */
SPMV_API int spmv_check(spmv_handle h, void *stream);

/* Frees every device array of the handle.  NULL is accepted. */
SPMV_API int spmv_destroy(spmv_handle h);

/* Message of the last failing call on this thread ("" if none). */
SPMV_API const char *spmv_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_GB300_SPMV_H */
