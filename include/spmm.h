/*
 * spmm.h - C ABI of the GB300 (sm_103a) CSR x dense SpMM library.
 *
 * Method: "Design Principles for Sparse Matrix Multiplication on the GPU"
 * (Yang, Buluc, Owens, arXiv 1803.08601).  Given an m x k sparse matrix A in
 * CSR form and a k x n dense row-major matrix B, the library computes the
 * m x n dense row-major product C = A B (Section 1), with the paper's two
 * algorithm families and its selection heuristic:
 *   - row split (Section 4.1, Fig. 3): a group of lanes per row of A, lanes
 *     striding the columns of B with 128-bit coalesced loads, column indices
 *     and values broadcast between lanes by warp shuffles;
 *   - merge based (Section 4.2, Algorithm 1): a merge-path partition of
 *     rows + nonzeros into equal tiles, a compute pass per tile, and a
 *     carry-out fix-up for rows that cross tiles;
 *   - the Section 5.4 heuristic: merge based when nnz / m < 9.35.
 * Beyond the paper: a GB300-calibrated selector, SpMV kernels of both
 * families for n = 1, 16-bit storage forms, semiring products, an A/B-tiled
 * kernel, the backward pass (transpose, SDDMM), batched plans and a
 * host-buffer entry point.
 *
 * Conventions shared by every entry point unless stated otherwise:
 *   - Array arguments are DEVICE pointers owned by the caller; the library
 *     keeps no reference after the call returns.
 *   - Indices are 0-based int32.  row_ptr has m + 1 entries, row_ptr[0] = 0,
 *     non-decreasing; 0 <= col_ind[p] < k.  Column indices inside a row need
 *     not be sorted (except for SPMM_ALG_TILED); repeated indices are summed.
 *     Out-of-range indices are a precondition violation (not checked; the
 *     result is undefined).
 *   - Dense matrices are row-major with leading dimension (row stride, in
 *     elements) ldb >= n, ldc >= n.
 *   - C is overwritten (beta = 0); rows of A without nonzeros give zero rows.
 *   - Accumulation is float32 in every precision form.  16-bit outputs are
 *     rounded to nearest even once per element.
 *   - `stream` is a cudaStream_t handle (NULL = the legacy default stream).
 *     Work is enqueued asynchronously; a return of SPMM_OK means the launch
 *     was accepted, not that the kernels finished.  Errors found on the
 *     device are written to the optional device status word `d_status`:
 *     SPMM_ERR_TIMEOUT for a bounded wait that ran out, SPMM_ERR_BAD_CSR for
 *     an inconsistent fix-up run or (SPMM_ALG_TILED) a row whose columns go
 *     backwards.  The first error stays; the caller clears the word.
 *   - No entry point aborts, throws, or falls back to the CPU.
 */
#ifndef SPMM_GB300_H
#define SPMM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMM_ALG_AUTO = 0,      /* Section 5.4 heuristic on the mean row length     */
    SPMM_ALG_ROW_SPLIT = 1, /* Section 4.1, Algorithm I                         */
    SPMM_ALG_MERGE = 2,     /* Section 4.2, Algorithm II (Algorithm 1)          */
    SPMM_ALG_AUTO_GB300 = 3, /* mean row length recalibrated on GB300 plus a
                               longest-row guard against Type 1 imbalance
                               (Section 3.2); see spmm_select_alg_gb300      */
    SPMM_ALG_TILED = 4,      /* row blocks of A times k-panels of B held in
                               shared memory: the tiling of A and B that
                               Section 6 proposes for denser matrices.  Rows
                               must list their columns in increasing order
                               (an entry that goes backwards is skipped and
                               reported as SPMM_ERR_BAD_CSR in d_status).
                               Needs 16-byte access to B and C; otherwise
                               the call runs the row split.  Measured slower
                               than the row split on GB300 at every density
                               tried; no selector picks it               */
    SPMM_ALG_ROW_SPLIT_HYBRID = 5 /* row split whose granularity (Section 4.1)
                               follows the row: a warp owns a block of
                               consecutive rows, and its lane groups split
                               the block's rows of at most
                               tuning->long_row_len nonzeros into runs of
                               equal nonzero count (no row is split; a batch
                               of gathers may serve several rows, against
                               the Type 2 imbalance of Section 3.2); longer
                               rows (Type 1) are queued on the device and
                               taken by one lane group, or cut into
                               segments of a warp each whose partial sums
                               are added in segment order.  Needs a
                               workspace (spmm_csr_workspace_size)       */
} spmm_alg_t;

typedef enum {
    SPMM_F32 = 0,  /* IEEE binary32            */
    SPMM_BF16 = 1, /* bfloat16 (8-bit exponent) */
    SPMM_F16 = 2   /* IEEE binary16            */
} spmm_dtype_t;

typedef enum {
    SPMM_OK = 0,
    SPMM_ERR_INVALID_VALUE = 1, /* a size, pointer, stride or enum is invalid   */
    SPMM_ERR_ALLOC = 2,         /* device memory could not be obtained          */
    SPMM_ERR_LAUNCH = 3,        /* a kernel launch was rejected                 */
    SPMM_ERR_BAD_CSR = 4,       /* reserved for CSR structure checks            */
    SPMM_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out           */
    SPMM_ERR_UNSUPPORTED = 6,   /* dtype combination not provided               */
    SPMM_ERR_CUDA = 7,          /* another CUDA runtime error                   */
    SPMM_ERR_WORKSPACE = 8      /* workspace pointer NULL or too small          */
} spmm_status_t;

/* Optional launch shape.  Zero in a field selects the library's choice. */
typedef struct {
    int lanes_per_row;       /* lanes that share one row of A: 1, 2, 4, 8, 16 or 32        */
    int column_slabs;        /* split the n columns into this many slabs (grid y); B's
                                rows are then gathered one slab at a time, which keeps
                                a slab of B resident in L2                              */
    int items_per_subwarp;   /* merge based: merge-path items (rows + nonzeros) per
                                lane group; a tile holds 256 / lanes_per_row groups     */
    int long_row_len;        /* SPMM_ALG_ROW_SPLIT_HYBRID: rows with more nonzeros than
                                this leave the row-block pass (queued rows of up to 4x
                                this are taken by one lane group, with 4 or more lanes
                                per row those above 2x first; longer ones by warp
                                segments); 0 selects max(32, lanes per row)            */
    double merge_threshold;  /* heuristic threshold on nnz / m; <= 0 selects 9.35       */
    long long max_row_len;   /* SPMM_ALG_AUTO_GB300: longest row of A when the caller
                                knows it; 0 makes the call measure it on the device
                                (a reduction and a 4-byte copy that synchronises)       */
    int block_rows;          /* SPMM_ALG_ROW_SPLIT_HYBRID: consecutive rows per warp in
                                the row-block pass, 1-256 (larger values act as 256);
                                0 selects 128, or 64 for >= 16 lanes per row            */
} spmm_tuning_t;

/* Human-readable name of a status code (static storage).  The paper defines
   no error reporting; the codes are this library's own. */
const char *spmm_status_string(int status);

/* Library ABI version (major * 100 + minor). */
int spmm_version(void);

/* Number of kernels this library has launched in this process (all devices).
   Host-side counter, incremented at every successful launch. */
long long spmm_launch_count(void);

/*
 * Section 5.4 heuristic.  d = nnz / m is the mean row length of A; returns
 * SPMM_ALG_MERGE when d < threshold and SPMM_ALG_ROW_SPLIT otherwise
 * (threshold <= 0 selects the paper's 9.35).  m == 0 returns row split.
 * Pure host function.
 */
int spmm_select_alg(int m, long long nnz, double threshold);

/*
 * GB300 selector (SPMM_ALG_AUTO_GB300), pure host function, fitted on GB300
 * sweeps of the three families (float32 B; the paper's single 9.35 was
 * measured on a K40c).  With row bytes = n * element size of B and
 * d = nnz / m:
 *   - when the longest row is long enough to be the critical path of row split
 *     (Type 1 imbalance, Section 3.2: max_row_len > 1024 and
 *     max_row_len * 8192 >= nnz, fitted on dense-as-CSR matrices from
 *     2 x 2^23 to 2^23 x 2): SPMM_ALG_ROW_SPLIT_HYBRID when rows of B are at
 *     most 128 bytes and the longest row is at least 16 d (most rows short
 *     beside the long ones: on 10^6 x 10^6 power-law matrices the hybrid is
 *     ahead at 32- and 128-byte rows, merge from 256), else SPMM_ALG_MERGE
 *     (rows all long: merge's equal tiles win);
 *   - d >= 768 with rows of B under 256 bytes: SPMM_ALG_MERGE;
 *   - rows of B under 64 bytes: SPMM_ALG_ROW_SPLIT;
 *   - d < 3: SPMM_ALG_ROW_SPLIT_HYBRID (its lane groups pack runs of short
 *     rows), or SPMM_ALG_MERGE for rows of B of 512 bytes or more when the
 *     longest row is at least 2d (uneven rows);
 *   - rows of B under 256 bytes: SPMM_ALG_ROW_SPLIT;
 *   - SPMM_ALG_MERGE when d < T, T = 8 for uneven rows, else 5 for rows of B
 *     of 512 bytes or more and 3 for 256-511 bytes; SPMM_ALG_ROW_SPLIT
 *     otherwise (measured crossovers for uniform and Poisson row lengths).
 * m == 0 returns row split.
 */
int spmm_select_alg_gb300(int m, long long nnz, long long max_row_len, int n, int b_type);

/*
 * Expected reuse of one staged B row under SPMM_ALG_TILED: the rows of A per
 * CTA block (2048 / lanes per row; lanes = the power of two covering n in
 * 16-byte vectors) times the density nnz / (m * k), i.e. how many of the
 * block's nonzeros share each B row the tiling stages once.  0 for empty
 * shapes.  Pure host function.
 */
double spmm_tiled_reuse(int m, int k, long long nnz, int n, int b_type);

/*
 * Column slabs the library uses by default for a product of algorithm alg
 * (a spmm_alg_t after selection) with k rows of B and n columns of b_type on
 * the current device: 2 when B is larger than twice the device's L2 and its
 * rows are wide (>= 512 bytes for merge, >= 256 bytes otherwise), else 1.
 * Each slab pass gathers that share of every row of B from a B slab that
 * much smaller.  Reads the L2 size of the current device (no device work).
 */
int spmm_default_column_slabs(int alg, int k, int n, int b_type);

/*
 * Longest row of A (max over i of row_ptr[i+1] - row_ptr[i]) computed on the
 * device and written to *max_row_len (host): the quantity behind the Type 1
 * imbalance of Section 3.2, which spmm_select_alg_gb300 takes.  Synchronises
 * `stream`.  The result words live in an 8-byte device buffer per host thread
 * and device, allocated at the first call and kept until exit.
 */
int spmm_csr_max_row_length(int m, const int *row_ptr, long long *max_row_len, void *stream);

/*
 * C = A B in float32 (vals, B, C all float32), the signature of the paper's
 * problem statement (Section 1).  alg is a spmm_alg_t.  For SPMM_ALG_AUTO the
 * heuristic needs nnz = row_ptr[m], which this call reads back from the device
 * (a 4-byte copy that synchronises `stream`); use spmm_csr_ex with a host nnz
 * to avoid it.  Merge-based launches take their workspace from a
 * stream-ordered allocation (cudaMallocAsync) released on the same stream.
 */
int spmm_csr(int m, int k, int n, const int *row_ptr, const int *col_ind, const float *vals,
             const float *B, long long ldb, float *C, long long ldc, int alg, void *stream);

/*
 * Full form of C = A B (Section 1; the algorithms of Sections 4.1 and 4.2,
 * chosen as in Section 5.4 for SPMM_ALG_AUTO).  Storage precision (16-bit
 * vals, B and C with float32 accumulation), the workspace, the launch shape
 * and the status word are this library's additions; the paper's kernels are
 * float32 throughout.  nnz is the host copy of row_ptr[m] (pass -1 to have it
 * read back, which synchronises `stream`).  vals_type / b_type / c_type are
 * spmm_dtype_t values; the supported combinations (vals, B, C) are
 * (f32,f32,f32), (bf16,bf16,bf16), (bf16,bf16,f32), (bf16,f16,f16),
 * (bf16,f16,f32), (f16,f16,f16) and (f16,f16,f32); others return
 * SPMM_ERR_UNSUPPORTED.  `tuning` may be NULL.
 * workspace: device memory of at least spmm_csr_workspace_size(...) bytes for
 * the merge-based algorithm (row split and SPMM_ALG_TILED need none); NULL
 * with workspace_bytes == 0 makes the call allocate it stream-ordered itself.
 * n == 1 (y = A x) runs the SpMV kernels of the chosen family: the row split
 * with tuning->lanes_per_row lanes per row (0: from the mean row length) and
 * the merge based with 4, 8 or 16 path items per thread
 * (tuning->items_per_subwarp; 0: 8).
 * ldb times the size of B's element type must be below 2^32 bytes
 * (SPMM_ERR_INVALID_VALUE otherwise): the kernels address rows of B with a
 * 32-bit byte stride.
 * The workspace must not be used by another call that may run concurrently.
 * d_status: optional device int; a bounded wait that runs out stores
 * SPMM_ERR_TIMEOUT there (the caller clears it).
 */
int spmm_csr_ex(int m, int k, int n, long long nnz, const int *row_ptr, const int *col_ind,
                const void *vals, int vals_type, const void *B, int b_type, long long ldb, void *C,
                int c_type, long long ldc, int alg, const spmm_tuning_t *tuning, void *workspace,
                size_t workspace_bytes, int *d_status, void *stream);

/* Semirings (+) . (x) of spmm_csr_semiring. */
typedef enum {
    SPMM_SEMIRING_PLUS_TIMES = 0, /* (+, x), identity 0: the ordinary product     */
    SPMM_SEMIRING_MIN_PLUS = 1,   /* (min, +), identity +inf: shortest-path step  */
    SPMM_SEMIRING_MAX_PLUS = 2,   /* (max, +), identity -inf: longest-path step   */
    SPMM_SEMIRING_MAX_TIMES = 3   /* (max, x), identity -inf: most reliable path  */
} spmm_semiring_t;

/*
 * C = A (+).(x) B over a semiring, float32 throughout: the GraphBLAS
 * matrix-matrix product that Section 1 names as a use of SpMM.
 * C[i][j] = (+) over the stored p of row i of (vals[p] (x) B[col_ind[p]][j]),
 * starting from the identity of (+), so an empty row gives the identity.
 * Both families (row split, merge based) and the selectors run unchanged;
 * the accumulate, the in-CTA combine and the fix-up use (+) and (x), and the
 * fix-up combines a split row's partial results in tile order as for the
 * ordinary product.  min and max are fminf / fmaxf (a NaN operand loses to a
 * number).  Arguments and workspace as in spmm_csr_ex (b_type float32);
 * semiring outside spmm_semiring_t returns SPMM_ERR_INVALID_VALUE.
 */
int spmm_csr_semiring(int m, int k, int n, long long nnz, const int *row_ptr, const int *col_ind,
                      const float *vals, const float *B, long long ldb, float *C, long long ldc, int semiring,
                      int alg, const spmm_tuning_t *tuning, void *workspace, size_t workspace_bytes,
                      int *d_status, void *stream);

/*
 * Bytes of workspace spmm_csr_ex needs for these sizes.  For the merge-based
 * algorithm this holds the merge-path coordinates of every tile boundary
 * (PARTITIONSPMM of Algorithm 1, Section 4.2) and each tile's carry-out and
 * head partial rows that FIXCARRYOUT combines; for the hybrid row split, its
 * queues of long rows and their segments' partial sums.  0 for row split.
 * alg SPMM_ALG_AUTO is resolved with the heuristic first.  Returns 0 for
 * invalid arguments.
 */
size_t spmm_csr_workspace_size(int m, int k, int n, long long nnz, int alg, int b_type,
                               const spmm_tuning_t *tuning);

/*
 * Merge-path partition (Section 4.2, PARTITIONSPMM of Algorithm 1; Section 4
 * item 2(b), Fig. 2(c)) on its own.  For t = 0 .. num_tiles, limits[2t] and
 * limits[2t + 1] receive (rows consumed, nonzeros consumed) where the merge of
 * the row end offsets row_ptr[1..m] with the nonzero indices 0..nnz-1 (row end
 * first on ties) crosses diagonal min(t * items_per_tile, m + nnz).
 * limits: device int array of 2 * (num_tiles + 1) entries.
 */
int spmm_merge_partition(int m, long long nnz, const int *row_ptr, int items_per_tile, int num_tiles,
                         int *limits, void *stream);

/*
 * C = A B with every array in HOST memory: the call copies A and B to the
 * device, computes, copies C back and synchronises `stream` before it returns.
 * Types and alg as in spmm_csr_ex; nnz is read from the host row_ptr[m]
 * (SPMM_ALG_AUTO_GB300 without tuning->max_row_len scans the host row_ptr for
 * the longest row).  Copies and compute are pipelined: B and C in column
 * slabs, A in up to four row chunks, so that the first block is computed as
 * soon as its pieces are on the device.  The uploads run on a copy stream of
 * the library's own, after all work queued on `stream` before the call, so a
 * host input that such work writes (a D2H copy, an earlier
 * spmm_csr_host_async) is read once it is written.  Device buffers come
 * stream-ordered from a memory pool of the library's own (one per device;
 * freed memory stays cached in it until exit) and are released before return.
 * Pinned (page-locked) host buffers make the copies asynchronous DMA.
 */
int spmm_csr_host(int m, int k, int n, const int *row_ptr, const int *col_ind, const void *vals,
                  int vals_type, const void *B, int b_type, long long ldb, void *C, int c_type,
                  long long ldc, int alg, const spmm_tuning_t *tuning, void *stream);

/*
 * spmm_csr_host without the final synchronisation (no counterpart in the
 * paper): the copies and kernels are queued and the call returns; C holds the
 * result once `stream` has been synchronised, or once an event recorded on
 * `stream` after the call has completed, and work queued on `stream` after the
 * call runs after C has arrived.  row_ptr is read on the host during the call; every
 * host buffer must stay valid, and A and B unmodified, until then.  Unlike
 * spmm_csr_host, the uploads are NOT ordered after work queued on `stream`
 * before the call: they start on the library's copy stream at once, so host
 * inputs must hold their final values when the call is made (the C of an
 * earlier asynchronous call becomes a valid input only after a
 * synchronisation of `stream`, or of an event recorded on it after that
 * call).  In exchange, with pinned host buffers, back-to-back calls overlap: a
 * call's uploads run while the previous call's last blocks of C are still
 * coming down.  Arguments, pipelining and errors as in spmm_csr_host; an error
 * of a queued copy or kernel is reported by the synchronisation, not by this
 * call.
 */
int spmm_csr_host_async(int m, int k, int n, const int *row_ptr, const int *col_ind, const void *vals,
                        int vals_type, const void *B, int b_type, long long ldb, void *C, int c_type,
                        long long ldc, int alg, const spmm_tuning_t *tuning, void *stream);

/*
 * Several host-buffer products with one sparse matrix (no counterpart in the
 * paper): C[i] = A B[i] for i < count, where B[i] is k x n[i] (leading
 * dimension ldb[i]) and C[i] is m x n[i] (ldc[i]), all in HOST memory, with
 * one vals / B / C type combination for all.  A goes up to the device once
 * for all of them, which is the saving over count calls of
 * spmm_csr_host_async.  The products run in the caller's order on the same
 * pipeline of column slabs and row chunks of A (a narrow product first lets
 * computing start soonest), and each block of every C[i] comes down as soon
 * as it is computed.  alg and tuning apply to every product; with
 * SPMM_ALG_AUTO_GB300 each product is selected for its own n[i] (the longest
 * row is found once).  Queued like spmm_csr_host_async, with the same rules:
 * the host inputs are read from call time on and must stay valid and
 * unmodified until `stream` has been synchronised (or an event recorded on
 * it after the call has completed), when every C[i] holds its result.
 * Products with n[i] == 0 are skipped.  n, B, ldb, C and ldc are host arrays
 * of count entries (they may be NULL when count == 0).  Argument errors of
 * any product return before any work is queued.
 */
int spmm_csr_host_multi(int m, int k, const int *row_ptr, const int *col_ind, const void *vals, int vals_type,
                        int count, const int *n, const void *const *B, int b_type, const long long *ldb,
                        void *const *C, int c_type, const long long *ldc, int alg, const spmm_tuning_t *tuning,
                        void *stream);

/*
 * Self-test of the bounded device-side wait used by the merge kernel's
 * shared-memory staging: one CTA waits on an mbarrier phase that nothing
 * completes, for at most limit_ns nanoseconds of device time (clamped to
 * [1e3, 2e9]), then stores SPMM_ERR_TIMEOUT to *d_status and returns.  The
 * context stays usable.  Not part of the paper; used by the failure tests.
 */
int spmm_debug_bounded_wait(int *d_status, long long limit_ns, void *stream);

/*
 * Gather-rate probe (measurement only; the paper has no counterpart, though
 * the access it times is the one Section 4.1 singles out: one row of B read
 * per nonzero with coalesced accesses).  Reads count rows of row_bytes bytes
 * (16, 32, 64, 128, 256 or 512) of the device array B (rows rows, row r at
 * byte offset r * row_bytes, B 16-byte aligned) at the row indices idx[0 ..
 * count) (device int array; an index outside [0, rows) is skipped), with
 * lane groups of row_bytes / 16 lanes and eight rows in flight per lane as in
 * the SpMM kernels, and XORs every 32-bit word read into *out (a device
 * word the caller initialises).  Timing it over B sizes and row widths gives
 * the gather ceilings and the effective L2 capacity that bound the SpMM
 * rooflines.  Asynchronous on `stream`.
 */
int spmm_gather_probe(const void *B, long long rows, int row_bytes, const int *idx, long long count,
                      unsigned *out, void *stream);

/* ------------------------------------------------------------------------
 * Backward of C = A B (not in the paper, which names SpMM_T only as future
 * work in Section 6): dB = A^T dC through spmm_csr_ex on A^T, and
 * dvals = SDDMM(dC, B) on A's pattern.
 * ---------------------------------------------------------------------- */

/* Bytes of workspace spmm_csr_transpose needs (0 for invalid sizes). */
size_t spmm_csr_transpose_workspace_size(int m, int k, long long nnz);

/*
 * A^T in CSR form by a stable sort of the nonzeros on their column index:
 * row c of A^T lists the nonzeros of column c of A in increasing original
 * position p; col_ind_t[q] is the row of A holding that nonzero and perm[q]
 * its position p, so vals_t[q] = vals[perm[q]] (spmm_gather_values).
 * row_ptr_t has k + 1 entries; col_ind_t and perm have nnz entries.  The
 * result is deterministic.  workspace as in spmm_csr_ex (NULL with 0 bytes
 * = stream-ordered allocation).
 */
int spmm_csr_transpose(int m, int k, long long nnz, const int *row_ptr, const int *col_ind, int *row_ptr_t,
                       int *col_ind_t, int *perm, void *workspace, size_t workspace_bytes, void *stream);

/* out[q] = vals[perm[q]] for q < nnz (vals_type: any spmm_dtype_t). */
int spmm_gather_values(long long nnz, const int *perm, const void *vals, int vals_type, void *out, void *stream);

/*
 * Sampled dense-dense product on A's pattern:
 * out[p] = sum_j dC[i][j] * B[col_ind[p]][j] for every nonzero p of row i,
 * the gradient of <dC, A B> with respect to the stored values.  dC is m x n
 * (leading dimension lddc), B is k x n (ldb); dC and B share one type;
 * (dc/b type, out type) in {(f32,f32), (bf16,bf16), (bf16,f32), (f16,f16),
 * (f16,f32)}.  Float32 accumulation.  Work is split into equal runs of
 * consecutive nonzeros (Section 4 item 2(a), nonzero split).
 */
int sddmm_csr(int m, int k, int n, long long nnz, const int *row_ptr, const int *col_ind, const void *dC,
              int dc_type, long long lddc, const void *B, int b_type, long long ldb, void *out, int out_type,
              void *stream);

/* ------------------------------------------------------------------------
 * Batched form (not in the paper): many independent float32 products
 * C_b = A_b B_b of uneven sizes in one persistent kernel launch plus one
 * fix-up launch, replayable as a CUDA graph.  Each matrix runs one of the
 * paper's two families: row split contributes chunks of consecutive rows,
 * merge based contributes merge-path tiles (Section 4.2) whose partition is
 * computed once, when the plan is made.
 * ---------------------------------------------------------------------- */

/* One product of a batch.  Device pointers, caller-owned, float32; n, ldb,
   ldc multiples of 4 and B, C 16-byte aligned (16-byte accesses only). */
typedef struct {
    int m, k, n;
    long long nnz; /* host copy of row_ptr[m] */
    const int *row_ptr;
    const int *col_ind;
    const float *vals;
    const float *B;
    long long ldb;
    float *C;
    long long ldc;
} spmm_batch_matrix_t;

typedef struct spmm_batched_plan spmm_batched_plan_t; /* opaque */

typedef enum {
    SPMM_BATCHED_MODEL = 0,     /* per matrix: merge based when the longest row trips the Type 1
                                   guard of spmm_select_alg_gb300 (longest rows read at plan
                                   time), row split otherwise: inside the batch the merge tiles
                                   run about 2x slower than the row chunks                      */
    SPMM_BATCHED_AUTOTUNE = 1,  /* per matrix: the autotuner's pick for its shape bucket            */
    SPMM_BATCHED_ROW_SPLIT = 2, /* every matrix row split                                            */
    SPMM_BATCHED_MERGE = 3,     /* every matrix merge based                                          */
    SPMM_BATCHED_ROW_SPLIT_X2 = 4 /* every matrix row split, read with two 16-byte vectors per lane
                                   where n, ldb and ldc are multiples of 8 (one elsewhere)        */
} spmm_batched_policy_t;

/*
 * Make a plan for `count` products (host array of descriptors; the pointed-to
 * device arrays must stay valid and keep their sparsity patterns while the
 * plan is used; values of vals and B may change between runs).  The plan owns
 * one device allocation (work list, merge partitions, carry buffers) and
 * synchronises `stream` once.  SPMM_BATCHED_AUTOTUNE times, for every shape
 * bucket (n, floor(log2 m), mean row length class) not yet in the process-wide
 * cache, row split with one and with two 16-byte vectors per lane (the latter
 * when n, ldb and ldc are multiples of 8), each with the full lane group of
 * the width and with a half and a quarter of it (twice and four times the
 * column slabs), and merge based with three tile sizes, on a sample of the
 * plan's matrices of that bucket (up to 64 matrices or 4M rows + nonzeros,
 * repeated to 32M rows + nonzeros so that it is timed on a busy GPU), and
 * keeps the fastest.  The row split of a plan runs as one persistent kernel
 * per access width that its matrices use.
 */
int spmm_batched_plan_create(int count, const spmm_batch_matrix_t *mats, int policy, void *stream,
                             spmm_batched_plan_t **plan);

/* Enqueue the batch: a persistent kernel over the row-split chunks of each
   access width the plan uses (on a stream of the plan's own, forked from and
   joined back to `stream`, when the plan also has merge tiles), a persistent
   kernel over the merge tiles and the fix-up (up to four launches, after a
   memset of the work counters).  Both
   persistent kernels take their work items from a counter, in the plan's
   order: row chunks of the largest matrices first.  Runs of one plan share its
   counters and carry buffers: they must not overlap on the GPU. */
int spmm_batched_run(const spmm_batched_plan_t *plan, void *stream);

/* Capture spmm_batched_run into a CUDA graph owned by the plan (replaces a
   previous one).  Capture happens on a private stream (the legacy default
   stream cannot be captured); `stream` is unused. */
int spmm_batched_capture_graph(spmm_batched_plan_t *plan, void *stream);

/* Launch the captured graph on `stream`. */
int spmm_batched_launch_graph(const spmm_batched_plan_t *plan, void *stream);

/* Baseline: the same per-matrix choices as one spmm_csr_ex call per matrix
   (partition, compute and fix-up launches for merge matrices). */
int spmm_batched_run_unfused(const spmm_batched_plan_t *plan, void *stream);

/* Per-matrix algorithm chosen (host array of count ints, may be NULL), work
   items of the persistent kernel and merge tiles (either may be NULL). */
int spmm_batched_plan_query(const spmm_batched_plan_t *plan, int *algs, long long *num_items, int *num_tiles);

int spmm_batched_plan_destroy(spmm_batched_plan_t *plan);

/* The autotuner's process-wide cache of per-bucket picks. */
long long spmm_autotune_cache_entries(void);
int spmm_autotune_cache_clear(void);

/*
 * Allocation-free form of spmm_csr_ex.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at call
 * time (plugins of a host that owns all device memory, real-time loops that
 * must not meet allocator latency or an out-of-memory failure mid-run) and
 * have no buffer to lend as a workspace.  Arguments are those of spmm_csr_ex
 * without the workspace; the caller still provides every input and output.
 *
 * The merge-based path keeps its scratch in one fixed array of
 * spmm_csr_static_scratch_bytes() bytes (16 MiB) in device global memory,
 * held until the process exits.  Problems whose merge scratch for the launch
 * shape the call picks exceeds it (at most spmm_csr_workspace_size(...), which
 * sizes for every shape) are rejected with SPMM_ERR_WORKSPACE before any
 * device work.  Row split needs no scratch.  The call itself makes no
 * cudaMalloc / cudaFree or other allocating call.
 *
 * The first merge-path call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  CUDA loads a library's device code lazily by
 * default, so that first call may also be the moment the library's code is
 * loaded on the device and the array reserved, and it can then fail for lack
 * of device memory: make it during set-up, and before any stream capture.
 * Every call shares the one array and leaves its contents behind; nothing in
 * it needs to start at zero, but calls that overlap on the GPU (on different
 * streams, or from several threads) race on it: serialise them.
 * nnz = -1 reads row_ptr[m] back (a 4-byte copy that synchronises `stream`).
 * alg SPMM_ALG_AUTO_GB300 is not accepted here (measuring the longest row
 * allocates); use SPMM_ALG_AUTO, SPMM_ALG_ROW_SPLIT or SPMM_ALG_MERGE.
 */
int spmm_csr_noalloc(int m, int k, int n, long long nnz, const int *row_ptr, const int *col_ind,
                     const void *vals, int vals_type, const void *B, int b_type, long long ldb, void *C,
                     int c_type, long long ldc, int alg, const spmm_tuning_t *tuning, int *d_status,
                     void *stream);

/* Size in bytes of the fixed scratch array used by spmm_csr_noalloc. */
size_t spmm_csr_static_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* SPMM_GB300_H */
