/*
 * spmv.h — C ABI of the GB300 (sm_103a) CRS sparse matrix-vector multiply.
 *
 * The operation is the CRS product of Sec. 1.2 of Schubert, Hager, Fehske and
 * Wellein, "Parallel sparse matrix-vector multiplication as a test case for
 * hybrid MPI+OpenMP programming" (arXiv 1101.0091):
 *
 *     C(i) = sum_{j = row_ptr(i)}^{row_ptr(i+1)-1} val(j) * B(col_idx(j))
 *
 * with 0-based indices.  The paper's loop accumulates into C; every apply call
 * here OVERWRITES C (C = A*B), except where stated.  All arithmetic is FP64
 * (products and row sums); the FP32-value option only changes how val is
 * stored (it is widened to FP64 exactly before each multiply).
 *
 * Conventions
 *  - Host pointers are plain host memory unless a name says _dev (device
 *    memory of the plan's device) or _pinned (page-locked host memory).
 *  - Index arrays are int32, values float64; row-major blocks of k right-hand
 *    sides are addressed as B[col * ldb + c] and C[row * ldc + c].
 *  - Streams are CUDA stream handles (cudaStream_t / CUstream) passed as
 *    void*; NULL is the legacy default stream.  Apply calls are asynchronous
 *    on the given stream and never synchronise the device.
 *  - Every call returns an spmv_status; no call throws or aborts.  The text of
 *    the last error of the calling thread is in spmv_last_error().
 *  - A plan owns all device memory it allocates; the caller keeps ownership
 *    of every array it passes.  A plan may be applied concurrently from
 *    several streams only if the output buffers differ.
 *  - Duplicate column indices inside a row are allowed (their products are
 *    summed); columns need not be sorted.
 */
#ifndef SPMV_GB300_H
#define SPMV_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmv_plan* spmv_handle;
typedef struct spmv_batch_plan* spmv_batch_handle;
typedef struct spmv_model* spmv_model_handle;

typedef enum {
  SPMV_OK = 0,
  SPMV_ERR_ARG = 1,         /* bad argument (null pointer, negative size, k out of range, ...) */
  SPMV_ERR_CSR = 2,         /* malformed CRS arrays (rejected on the host before any launch)   */
  SPMV_ERR_CUDA = 3,        /* a CUDA runtime call failed; message in spmv_last_error()        */
  SPMV_ERR_OOM = 4,         /* device or host allocation failed; nothing was leaked            */
  SPMV_ERR_TIMEOUT = 5,     /* a bounded wait ran out (host event wait or a device-side wait)  */
  SPMV_ERR_UNSUPPORTED = 6, /* the request needs a format or option the plan was not built for */
  SPMV_ERR_DEVICE = 7       /* a kernel reported an error through the plan's status word        */
} spmv_status;

/* Kernel variants.  All compute the same product with FP64 accumulation and
 * one fused multiply-add per stored entry (SYM: per stored off-diagonal entry
 * also one multiply for its mirror product). */
typedef enum {
  SPMV_VARIANT_AUTO = 0,   /* the plan's default, decided at creation from the matrix: SELL with  */
                           /* sigma 256 when more than 30 % of the entries of a sample of rows   */
                           /* are gathered at scattered addresses (entry (i, c) is regular when */
                           /* row i-1 holds column c-1 or row i+1 holds c+1) and SELL-32-256     */
                           /* stores at least 0.85 nonzeros per slot; CRS_L1 otherwise (a tuner  */
                           /* or the cost model may switch)                                      */
  SPMV_CRS_STAGED = 1,     /* thread per row; each CTA's contiguous val/col tile is brought     */
                           /* into shared memory by one bulk copy (cp.async.bulk + mbarrier);   */
                           /* rows longer than 64 go to warp-per-row blocks                      */
  SPMV_CRS_L1 = 2,         /* L lanes per row (L = 1, 2, 4, ..., 32), loads straight from HBM,   */
  SPMV_CRS_L2 = 3,         /* warp-shuffle reduction of the L partial sums                       */
  SPMV_CRS_L4 = 4,
  SPMV_CRS_L8 = 5,
  SPMV_CRS_L16 = 6,
  SPMV_CRS_L32 = 7,
  SPMV_SELL = 8,           /* SELL-C-sigma, C = 32, sigma from the options / set_variant         */
  SPMV_SYM = 9,            /* symmetric CRS (Sec. 1.3.1): only the entries on and above the      */
                           /* diagonal are stored and streamed; C is zeroed, then one thread    */
                           /* per row adds its own sum and, for each stored off-diagonal entry, */
                           /* the mirror product to the other row, with FP64 atomic adds.       */
                           /* Square, symmetric matrices only; the order in which a row's       */
                           /* contributions meet varies from call to call                       */
  SPMV_N_VARIANTS = 10
} spmv_variant;

typedef struct {
  int32_t variant;      /* spmv_variant; 0 = AUTO                                               */
  int32_t sell_sigma;   /* sigma of SPMV_SELL (sorting window); <= 1 means no sorting           */
  int32_t val_fp32;     /* 1: store val as float32 (exactly widened to FP64 before each FMA)    */
  int32_t max_k;        /* largest k for spmv_apply_block (1..16); 0 means 16                   */
  int32_t split;        /* 1: build the local/halo column split at column halo_begin (Sec. 3.1); */
                        /* 0: no split                                                           */
  int32_t reserved;     /* must be 0                                                             */
  int64_t halo_begin;   /* h of the split, 0 <= h <= n_cols (read only when split = 1)          */
                        /* A zero-initialised struct is the default (AUTO, no sorting, FP64     */
                        /* values, max_k 16, no split), the same as spmv_default_options().     */
} spmv_options;

typedef struct {
  int64_t n_rows, n_cols, nnz;
  int32_t variant;          /* active variant                                                   */
  int32_t sell_sigma;       /* sigma of the built SELL arrays (0 if none)                       */
  int64_t sell_slots;       /* stored SELL slots, sum of 32 * chunk_len (0 if none)             */
  int64_t sell_chunks;      /* number of SELL chunks                                            */
  int64_t n_halo_rows;      /* rows with at least one halo entry (split plans; else 0)          */
  int64_t halo_nnz;         /* entries with col >= halo_begin                                   */
  int64_t n_row_blocks;     /* CTAs of CRS_STAGED (row blocks)                                  */
  int32_t tile_nnz;         /* nonzero capacity of one CRS_STAGED tile                          */
  int32_t val_fp32;
  int64_t device_bytes;     /* device memory held by the plan                                   */
  int64_t sym_nnz;          /* stored entries of the SPMV_SYM triangle (0 if not built)         */
  double scattered;         /* share of the sampled entries gathered at scattered addresses     */
                            /* (the test of SPMV_VARIANT_AUTO: about 4096 evenly spaced rows    */
                            /* i = 1, 1 + s, ... with s = max(1, (n_rows - 2) / 4096), i <      */
                            /* n_rows - 1; entry (i, c) regular when row i-1 holds c-1 or row   */
                            /* i+1 holds c+1)                                                   */
  double sell256_fill;      /* nonzeros per stored slot of SELL-32-256 (from the row lengths)    */
} spmv_info;

/* Default options: AUTO, sigma 1, FP64 values, max_k 16, no split (a zero-initialised
 * spmv_options means the same). */
spmv_options spmv_default_options(void);

/* Thread-local text of the last error ("" if none). */
const char* spmv_last_error(void);

/* Create a plan on the current CUDA device from HOST CRS arrays (copied;
 * the caller keeps them).  row_ptr has n_rows+1 entries with row_ptr[0] = 0,
 * non-decreasing, row_ptr[n_rows] = nnz <= 2^31-1; col_idx and val have nnz
 * entries with 0 <= col_idx < n_cols.  nnz is the caller's count of stored
 * entries; it must equal row_ptr[n_rows] (a mismatch is SPMV_ERR_CSR).
 * Violations return SPMV_ERR_CSR before anything is allocated on the device.
 * Sec. 1.2 (CRS format).  opt may be NULL (defaults). */
spmv_status spmv_create(spmv_handle* out, int64_t n_rows, int64_t n_cols, int64_t nnz,
                        const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                        const spmv_options* opt);

/* Free all memory of a plan; NULL is accepted.  Synchronises the device first. */
spmv_status spmv_destroy(spmv_handle h);

/* C_dev[0:n_rows] = A * B_dev[0:n_cols] (overwrite), asynchronous on stream.
 * Sec. 1.2 listing. */
spmv_status spmv_apply(spmv_handle h, const double* B_dev, double* C_dev, void* stream);

/* Block of k right-hand sides (SpMM): C_dev[i*ldc + c] = sum_j val(j) * B_dev[col(j)*ldb + c]
 * for c < k; 1 <= k <= opt.max_k <= 16, ldb >= k, ldc >= k.  Same loop as
 * Sec. 1.2, applied to k vectors at once. */
spmv_status spmv_apply_block(spmv_handle h, const double* B_dev, int32_t k, int64_t ldb,
                             double* C_dev, int64_t ldc, void* stream);

/* Local/halo split product with overlapped halo copy (Sec. 3.1 and 3.2 recast
 * for one GPU): on copy_stream, B_halo_pinned[0 : n_cols - h] is copied into
 * B_dev[h : n_cols] while the local kernel (entries with col < h; the plan's
 * CRS variant, CRS_L1 for SELL and SYM plans) writes C on main_stream;
 * main_stream then waits for the copy and the halo kernel adds
 * the entries with col >= h into C.  B_dev[0:h] must already hold the local
 * part.  Requires a plan built with split = 1, halo_begin = h.  copy_stream may equal
 * main_stream (no overlap).  On return all work is enqueued; main_stream
 * carries the completion of both. */
spmv_status spmv_apply_split(spmv_handle h, double* B_dev, const double* B_halo_pinned,
                             double* C_dev, void* main_stream, void* copy_stream);

/* Same product, end to end from HOST buffers: B_host (n_cols*k) is copied to
 * plan-owned device buffers, multiplied, and C_host (n_rows*k, ldc = k) is
 * copied back; synchronises the stream before returning.  k = 1 uses
 * spmv_apply, k > 1 spmv_apply_block with ldb = ldc = k. */
spmv_status spmv_apply_host(spmv_handle h, const double* B_host, int32_t k, double* C_host,
                            void* stream);

/* Pipelined end-to-end products from PAGE-LOCKED host buffers.  Each call
 * enqueues one step and returns: the copy of B_host (n_cols*k) into one of two
 * plan-owned device buffer sets on an internal copy-in stream, the product on
 * `stream` once that copy is in, and the copy of the result into C_host
 * (n_rows*k, row-major, ldc = k) on an internal copy-out stream.  Steps
 * alternate between the two buffer sets, so the copy-in of step i+1 and the
 * copy-out of step i-1 run while step i multiplies (the paper's overlap of
 * transfers and computation, Sec. 3.2, applied to the host link).  B_host and
 * C_host must stay valid until spmv_host_sync returns. */
spmv_status spmv_apply_host_async(spmv_handle h, const double* B_host, int32_t k, double* C_host, void* stream);

/* Wait for every step enqueued by spmv_apply_host_async on this plan. */
spmv_status spmv_host_sync(spmv_handle h);

/* Switch the active variant (building its format on first use: the row
 * blocks of CRS_STAGED, SELL-C-sigma with the given sigma, or the upper
 * triangle of SPMV_SYM).  SPMV_SYM needs n_rows == n_cols and a symmetric
 * matrix: every entry strictly above the diagonal, (i, j, v), matched one to
 * one by an entry (j, i, v) strictly below it (values compared with
 * -0.0 == +0.0, so duplicates must mirror one to one); otherwise it returns
 * SPMV_ERR_UNSUPPORTED, names the first unmatched row, and the active variant
 * stays as it was. */
spmv_status spmv_set_variant(spmv_handle h, int32_t variant, int32_t sell_sigma);

spmv_status spmv_get_info(spmv_handle h, spmv_info* info);

/* Launch parameters a tuner may change without touching the result.
 * prefetch_distance: each CTA of the row and SELL kernels asks the TMA engine
 * to prefetch into L2 the matrix slice of the CTA this many positions ahead
 * (cp.async.bulk.prefetch.L2); 0 disables it.  Default: 456 (three per SM), and
 * 0 on matrices whose gathers are scattered (the test of SPMV_VARIANT_AUTO):
 * their product is bound by the SMs' requests to L2, which a prefetch adds
 * to. */
typedef struct {
  int32_t prefetch_distance;
  int32_t reserved[7];
} spmv_tuning;

spmv_status spmv_set_tuning(spmv_handle h, const spmv_tuning* t);
spmv_status spmv_get_tuning(spmv_handle h, spmv_tuning* t);

/* Wait for the plan's work on `stream`, then read and clear the plan's device
 * status word: SPMV_ERR_DEVICE (message names the failing step) if a kernel
 * reported a failed bounded wait, else SPMV_OK. */
spmv_status spmv_check(spmv_handle h, void* stream);

/* Host-side bounded wait: poll until the work on `stream` is done, giving up
 * after timeout_ms with SPMV_ERR_TIMEOUT (the work keeps running; call again).
 * The paper's codes wait on MPI requests; this is the host's deadline. */
spmv_status spmv_wait(void* stream, int32_t timeout_ms);

/* Self-test of the failure path of the bounded device wait (no fault, no
 * hang): one CTA waits on an mbarrier phase that nothing completes, with the
 * same bounded wait as CRS_STAGED's bulk copies but a limit of limit_us
 * microseconds (1 .. 1,000,000); it gives up, records the timeout in a status
 * word and exits.  Returns SPMV_ERR_TIMEOUT when the kernel reported the
 * timeout (the expected outcome), SPMV_OK if the wait completed.  Synchronous
 * on the current device. */
spmv_status spmv_selftest_wait_timeout(int32_t limit_us);

/* Copy the built SELL-C-sigma arrays to host arrays sized from spmv_info:
 * perm[n_rows], chunk_ptr[sell_chunks+1], chunk_len[sell_chunks],
 * sell_col[sell_slots], sell_val[sell_slots] (any may be NULL to skip).
 * Layout: chunks of C = 32 sorted rows, column-major inside a chunk. */
spmv_status spmv_sell_export(spmv_handle h, int32_t* perm, int64_t* chunk_ptr, int32_t* chunk_len,
                             int32_t* sell_col, double* sell_val);

/* Copy the SPMV_SYM triangle to host arrays sized from spmv_info:
 * row_ptr[n_rows+1], col[sym_nnz], val[sym_nnz] (any may be NULL).  Row i
 * holds the entries of row i with col_idx >= i, in their order in the row
 * (Sec. 1.3.1).  SPMV_ERR_UNSUPPORTED if the triangle was not built. */
spmv_status spmv_sym_export(spmv_handle h, int32_t* row_ptr, int32_t* col, double* val);

/* Copy the local/halo split arrays to host arrays sized from spmv_info:
 * loc_row_ptr[n_rows+1], loc_col/loc_val[nnz - halo_nnz], halo_rows[n_halo_rows],
 * halo_row_ptr[n_halo_rows+1], halo_col/halo_val[halo_nnz] (any may be NULL). */
spmv_status spmv_split_export(spmv_handle h, int32_t* loc_row_ptr, int32_t* loc_col, double* loc_val,
                              int32_t* halo_rows, int32_t* halo_row_ptr, int32_t* halo_col,
                              double* halo_val);

/* ----------------------------------------------------------------------------
 * Batched products: many uneven matrices, each with a block of k right-hand
 * sides, in ONE persistent kernel launch replayed from a CUDA graph.  Each
 * member computes C_m = A_m * B_m with the loop of Sec. 1.2 (row-major blocks,
 * ldb_m/ldc_m >= k).  The work list holds items (matrix, row range, lanes per
 * row L); warps of a grid of (SMs x resident CTAs) take items either in a fixed
 * round-robin order or from an atomic counter, and L lanes share a row (an
 * xor-shuffle tree adds their partial sums when L > 1).  The batch keeps
 * pointers to the members' device arrays: the plans must outlive the batch.
 * ------------------------------------------------------------------------- */

/* Per-matrix row policy of a batch member (the "variant" of a member). */
typedef enum {
  SPMV_BATCH_L1 = 0,      /* one lane per row                                        */
  SPMV_BATCH_L2 = 1,
  SPMV_BATCH_L4 = 2,
  SPMV_BATCH_L8 = 3,
  SPMV_BATCH_L32 = 4,     /* a warp per row                                          */
  SPMV_BATCH_ADAPT = 5,   /* rows binned by exact length (<= 32: one lane per row),   */
                          /* longer rows with about 32 entries per lane (L <= 32)     */
  SPMV_BATCH_SORTED = 6,  /* rows of <= 64 entries copied into a length-sorted       */
                          /* SELL-32 layout (coalesced, one lane per row); longer     */
                          /* rows as in ADAPT.  Costs a copy of those rows' entries.  */
  SPMV_BATCH_N_POLICIES = 7
} spmv_batch_policy;

typedef struct {
  int32_t item_nnz;       /* target nonzeros per work item (64 .. 1<<20)              */
  int32_t schedule;       /* 0 = static round-robin over warps, 1 = atomic counter     */
  int32_t ctas_per_sm;    /* persistent grid = SMs x ctas_per_sm CTAs of 128 threads (1 .. 8); at most 7
                             resident per SM for k <= 4, 5 for k = 5..8, 4 for k = 9..16 (the static
                             schedule runs the items of CTAs beyond that after the resident ones) */
  int32_t reserved[5];
} spmv_batch_config;

/* Default batch configuration: item_nnz 1024, atomic counter, 7 CTAs per SM. */
spmv_batch_config spmv_batch_default_config(void);

/* Build a batch over `count` plans (same device) with k right-hand sides each
 * (1 <= k <= 16).  policies[count] (NULL: all SORTED) picks each member's row
 * policy.  Uploads the work list and the member table; no product runs.  The
 * batch reads the plans' CRS arrays in place: the plans must outlive it. */
spmv_status spmv_batch_create(spmv_batch_handle* out, int32_t count, const spmv_handle* plans, int32_t k,
                              const int32_t* policies, const spmv_batch_config* cfg);

/* Set the members' operands: B_ptrs[m] (n_cols_m x ldb[m]) and C_ptrs[m]
 * (n_rows_m x ldc[m]) are DEVICE pointers held in host arrays; ldb/ldc NULL
 * means k.  B_ptrs[m] may be NULL only for a member without nonzeros, C_ptrs[m]
 * only for a member without rows (else SPMV_ERR_ARG).  The call first waits
 * until the batch's last enqueued replay (spmv_batch_apply or
 * spmv_batch_apply_host, on whatever stream) has finished, then copies the
 * pointers into the device member table; call again to move the batch to other
 * buffers.  Replays enqueued after it read the new operands. */
spmv_status spmv_batch_set_io(spmv_batch_handle b, const double* const* B_ptrs, const int64_t* ldb,
                              double* const* C_ptrs, const int64_t* ldc);

/* Enqueue the whole batch on `stream`: replays the batch's CUDA graph (counter
 * reset + persistent kernel).  Asynchronous. */
spmv_status spmv_batch_apply(spmv_batch_handle b, void* stream);

/* End to end from HOST buffers: each member's B_host[m] (n_cols_m x k, ld = k;
 * pinned memory for asynchronous copies) is copied into the device B set by
 * spmv_batch_set_io (overwriting it), the batch runs, and each member's C
 * (n_rows_m x k) is copied back to C_host[m] (ld = k); one cudaMemcpyAsync
 * per direction and run of consecutive members whose blocks follow one another
 * both on the host and on the device (one copy per member when they do not),
 * all on `stream`.  Needs set_io with ldb = ldc = k
 * (else SPMV_ERR_ARG).  Asynchronous: synchronise `stream` before reading
 * C_host.  Host arrays B_host[count], C_host[count] are read during the call. */
spmv_status spmv_batch_apply_host(spmv_batch_handle b, const double* const* B_host, double* const* C_host,
                                  void* stream);

/* Pipelined end-to-end batched products from PAGE-LOCKED host buffers (the
 * paper's overlap of transfers and computation, Sec. 3.2, applied to the host
 * link).  Each call enqueues one step and returns: every member's B_host[m]
 * (n_cols_m x k, ld = k) is copied into one of two batch-owned device buffer
 * sets on an internal copy-in stream, the batched launch runs on `stream` once
 * that copy is in, and every member's C (n_rows_m x k) is copied back to
 * C_host[m] (ld = k) on an internal copy-out stream.  Steps alternate between
 * the two sets (each with its own member table and graph), so the copy-in of
 * step i+1 and the copy-out of step i-1 run while step i computes.  Copies of
 * consecutive members whose host blocks follow one another are merged.  The
 * sets are allocated on the first call (the operands of spmv_batch_set_io are
 * not used or changed).  Host arrays B_host[count], C_host[count] are read
 * during the call; the buffers they point to must stay valid until
 * spmv_batch_host_sync returns. */
spmv_status spmv_batch_apply_host_async(spmv_batch_handle b, const double* const* B_host, double* const* C_host,
                                        void* stream);

/* Wait for every step enqueued by spmv_batch_apply_host_async on this batch. */
spmv_status spmv_batch_host_sync(spmv_batch_handle b);

/* Same work as separate launches: one kernel per member, in member order (the
 * baseline the batched launch replaces).  Asynchronous. */
spmv_status spmv_batch_apply_separate(spmv_batch_handle b, void* stream);

/* Change the configuration (rebuilds the work list and the graph). */
spmv_status spmv_batch_set_config(spmv_batch_handle b, const spmv_batch_config* cfg);
spmv_status spmv_batch_get_config(spmv_batch_handle b, spmv_batch_config* cfg);

/* Change the members' policies (rebuilds the work list and the graph). */
spmv_status spmv_batch_set_policies(spmv_batch_handle b, const int32_t* policies);

/* Autotuner: times every configuration of item_nnz in {256, 512, 1024, 2048,
 * 4096} x schedule in {static, atomic} x ctas_per_sm in {4, 7} (`reps` graph
 * replays each after one warm-up, CUDA events on `stream`; needs set_io
 * first), keeps the fastest, and returns it (best may be NULL).  times_ms
 * (NULL or 20 entries) receives the median time of each configuration in that
 * order.  Results do not depend on the configuration. */
spmv_status spmv_batch_autotune(spmv_batch_handle b, void* stream, int32_t reps, spmv_batch_config* best,
                                float* times_ms);

/* Number of work items in the current work list. */
spmv_status spmv_batch_info(spmv_batch_handle b, int64_t* n_items, int64_t* total_rows, int64_t* total_nnz);

spmv_status spmv_batch_destroy(spmv_batch_handle b);

/* Batched products without any device allocation.  The paper has no
 * counterpart: this entry exists for callers that may not call cudaMalloc
 * themselves or through a library -- applications that hand every byte of
 * device memory to their own pool under a fixed budget, and latency-critical
 * paths where an allocation's implicit device synchronisation and unbounded
 * cost are not acceptable.  Such callers cannot create plans (plan creation
 * allocates), so they pass their own device CRS arrays.
 *
 * Computes, for each member m < count, C_dev[m][i*ldc[m] + c] = sum over
 * j = row_ptr_dev[m][i] .. row_ptr_dev[m][i+1]-1 of
 * val_dev[m][j] * B_dev[m][col_dev[m][j]*ldb[m] + c], c < k (1 <= k <= 16),
 * with lanes[m] lanes per row (1, 2, 4, 8, 16 or 32; NULL: 1) in one launch of
 * the persistent batch kernel (atomic work counter).  All per-member arrays
 * are HOST arrays of `count` entries; the pointers in them are DEVICE pointers
 * of the current device; ldb/ldc NULL means k.  A member with rows needs
 * non-NULL row_ptr, col, val, B and C pointers (else SPMV_ERR_ARG; every
 * argument is checked before the first CUDA call).  Results are the same,
 * bit for bit, as spmv_batch_apply with the fixed policy of the same lanes
 * per row (there is none for 16 lanes).
 *
 * Scratch: one static 8 MiB device array per device that loads the library,
 * held until the process exits, holding the work counter, the member table and
 * the work list.  Limits: count <= 8192 members and at most 245,752 work
 * items (one item per 32 warp passes: 1024 rows at 1 lane per row), beyond
 * which the call returns SPMV_ERR_ARG without touching the device.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress).
 * Every call clears the counter and overwrites the table and the list in the
 * shared array, so calls that overlap on the GPU (other streams, other host
 * threads) race: order them on one stream.  Host calls are serialised by a mutex.  Asynchronous on
 * `stream`; calls no cudaMalloc, cudaFree or allocating library routine. */
spmv_status spmv_batch_apply_noalloc(int32_t count, const int64_t* n_rows, const int32_t* const* row_ptr_dev,
                                     const int32_t* const* col_dev, const double* const* val_dev,
                                     const double* const* B_dev, const int64_t* ldb, double* const* C_dev,
                                     const int64_t* ldc, int32_t k, const int32_t* lanes, void* stream);

/* ----------------------------------------------------------------------------
 * Cost model: an MLP predicting the log run time of each kernel variant from a
 * matrix's features (spmv_features), so that a plan or batch member runs the
 * variant with the smallest prediction.  The paper has no learned component
 * (its Sec. 1.2 model is analytic); the network and its training are
 * hand-written FP32 CUDA kernels:
 *   Xn = (X - mean) * inv_std; H1 = relu(Xn W1^T + b1); H2 = relu(H1 W2^T + b2);
 *   Y = H2 W3^T + b3; loss = sum(mask (Y - T)^2) / sum(mask); Adam updates.
 * Parameters (host and device layout, float32): W1[H*F], b1[H], W2[H*H], b2[H],
 * W3[V*H], b3[V].  X (M x F), T and mask (M x V) are row-major float32 DEVICE
 * arrays; masked-out targets may hold any value.  All reductions run in a
 * fixed order: results are deterministic.
 * ------------------------------------------------------------------------- */
spmv_status spmv_model_create(spmv_model_handle* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                              const float* params /* host */);
spmv_status spmv_model_info(spmv_model_handle m, int32_t* n_in, int32_t* n_hidden, int32_t* n_out,
                            int64_t* n_params, int32_t* adam_steps);
/* Replace the parameters (host array) and reset the Adam moments and step. */
spmv_status spmv_model_set_params(spmv_model_handle m, const float* params);
spmv_status spmv_model_get_params(spmv_model_handle m, float* params);
/* Feature normalisation (host arrays of n_in), applied inside the forward pass. */
spmv_status spmv_model_set_normalizer(spmv_model_handle m, const float* mean, const float* inv_std);
/* Y_dev (M x n_out) = network(X_dev); asynchronous on stream. */
spmv_status spmv_model_forward(spmv_model_handle m, const float* X_dev, int32_t M, float* Y_dev, void* stream);
/* Forward + backward: loss (1 float, device; NULL: internal) and the gradient
 * in the parameter layout (device; NULL: the model's own gradient buffer). */
spmv_status spmv_model_loss_grad(spmv_model_handle m, const float* X_dev, const float* T_dev, const float* mask_dev,
                                 int32_t M, float* loss_dev, float* grad_dev, void* stream);
/* One Adam step with the given gradient (NULL: the model's own buffer). */
spmv_status spmv_model_adam_step(spmv_model_handle m, const float* grad_dev, float lr, float beta1, float beta2,
                                 float eps, void* stream);
/* loss_grad + Adam (beta1 0.9, beta2 0.999, eps 1e-8). */
spmv_status spmv_model_train_step(spmv_model_handle m, const float* X_dev, const float* T_dev, const float* mask_dev,
                                  int32_t M, float lr, float* loss_dev, void* stream);
/* Predict for M HOST feature rows (float64, M x n_in) and return, per row, the
 * index of the smallest predicted log time (host int32[M]); predicted (host
 * float32[M x n_out]) may be NULL.  Synchronises the stream. */
spmv_status spmv_model_select(spmv_model_handle m, const double* features, int32_t M, int32_t* choice,
                              float* predicted, void* stream);
/* As spmv_model_select, with a guard for a known-good default: row i takes the
 * output of smallest prediction only if that prediction is below the
 * prediction of output `fallback` by more than `margin` (log-time units: 0.05
 * asks for a predicted gain above about 5 %); otherwise it takes `fallback`.
 * fallback < 0 turns the guard off; margin >= 0. */
spmv_status spmv_model_select_guarded(spmv_model_handle m, const double* features, int32_t M, int32_t fallback,
                                      float margin, int32_t* choice, float* predicted, void* stream);
/* Pick a plan's kernel with the cost model: the plan's 34 features for k
 * right-hand sides (spmv_features) go through the network (n_in must be 34),
 * output o stands for variant variants[o] with SELL sigma sigmas[o] (host
 * arrays of the network's n_out entries), and the plan switches to the
 * output with the smallest prediction as spmv_set_variant would.  *choice
 * (host) receives o.  Synchronises the stream. */
spmv_status spmv_select(spmv_handle h, spmv_model_handle m, int32_t k, const int32_t* variants,
                        const int32_t* sigmas, int32_t* choice, void* stream);

/* Exhaustive timed sweep, the fallback of the cost model and the measure of its
 * regret: for each candidate (variants[i], sigmas[i]), i < n, the product of
 * k right-hand sides B_dev -> C_dev (layout as spmv_apply_block) is run once
 * untimed and then `reps` times between CUDA events on `stream`; the plan
 * switches to the candidate with the smallest median time.  *best (host)
 * receives its index; times_ms[n] (host, may be NULL) the medians, +inf for
 * a candidate the plan cannot build (e.g. SYM on an unsymmetric matrix).
 * Returns SPMV_ERR_UNSUPPORTED if no candidate builds.  Synchronous. */
spmv_status spmv_autotune(spmv_handle h, int32_t k, const double* B_dev, int64_t ldb, double* C_dev, int64_t ldc,
                          const int32_t* variants, const int32_t* sigmas, int32_t n, int32_t reps, int32_t* best,
                          float* times_ms, void* stream);

/* Checkpoint with the normaliser, parameters and Adam state (binary file). */
spmv_status spmv_model_save(spmv_model_handle m, const char* path);
spmv_status spmv_model_load(spmv_model_handle* out, const char* path);
spmv_status spmv_model_destroy(spmv_model_handle m);

/* ----------------------------------------------------------------------------
 * Iterative consumers of the product.  Sec. 1.3.1 names Lanczos and
 * Jacobi-Davidson as the eigensolvers run on the Hamiltonian matrices, whose
 * run time the product dominates; conjugate gradients is the matching solver
 * for symmetric positive definite matrices such as the Poisson workload.
 * Both run on k independent columns, so each iteration's product is one
 * k-column spmv_apply_block through the plan (whatever its variant).
 *
 * A solver holds three n x k work blocks and per-column scalars on the
 * plan's device; it borrows the plan (destroy the solver first).  Vector
 * blocks are row-major n x k with ld = k (X[i*k + c]) and 16-byte aligned
 * (else SPMV_ERR_ARG).  Inner products are reduced in a fixed order: repeated
 * solves give identical results.
 * ------------------------------------------------------------------------- */
typedef struct spmv_solver* spmv_solver_handle;

typedef struct {
  int32_t iterations;   /* largest number of iterations run by a column               */
  int32_t converged;    /* columns with |r| <= rtol |b|                                */
  int32_t breakdown;    /* columns stopped because p.Ap <= 0 (A not positive definite) */
  int32_t reserved;
} spmv_cg_summary;

/* Square plans only; 1 <= k <= the plan's max_k. */
spmv_status spmv_solver_create(spmv_handle A, int32_t k, spmv_solver_handle* out);
/* Synchronises the device, frees the work blocks; NULL is accepted. */
spmv_status spmv_solver_destroy(spmv_solver_handle s);

/* Conjugate gradients (Hestenes-Stiefel) on the k columns of B_dev.  X_dev
 * holds the initial guess on entry and the iterate on return.  Per column:
 * R = B - A X, P = R; each iteration Q = A P, alpha = R.R / P.Q, X += alpha P,
 * R -= alpha Q, beta = R.R(new) / R.R(old), P = R + beta P.  A column stops
 * (exactly as it is) once |R| <= rtol |B|, or on breakdown (P.Q <= 0); the
 * call returns when every column has stopped or after max_iter iterations.
 * The host polls the device every check_every iterations (those iterations
 * run from a CUDA graph captured on first use for these B, X and check_every,
 * and captured again after the plan's variant or tuning changes).
 * iterations_host[k] and rr_host[k] (final R.R) may be NULL.  Synchronous. */
spmv_status spmv_cg_solve(spmv_solver_handle s, const double* B_dev, double* X_dev, int32_t max_iter,
                          double rtol, int32_t check_every, void* stream, int32_t* iterations_host,
                          double* rr_host, spmv_cg_summary* summary);

/* m steps of the Lanczos three-term recurrence (no reorthogonalisation) from
 * the k columns of V0_dev: v_1 = v0/|v0|; w = A v_j - beta_{j-1} v_{j-1};
 * alpha_j = w.v_j; w -= alpha_j v_j; beta_j = |w|; v_{j+1} = w / beta_j.  A
 * column whose beta reaches 0 stops (zeros from there on).  alpha_host and
 * beta_host are m x k row-major host arrays; the Ritz values are the
 * eigenvalues of the tridiagonal matrix with alpha_1..m on the diagonal and
 * beta_1..m-1 beside it.  Synchronous. */
spmv_status spmv_lanczos(spmv_solver_handle s, const double* V0_dev, int32_t m, double* alpha_host,
                         double* beta_host, void* stream);

/* ----------------------------------------------------------------------------
 * Reordering.  Sec. 1.3.1 applies reverse Cuthill-McKee (RCM) to the
 * Hamiltonian matrix to make the accesses to B more local.  The permutation
 * is computed on the host with fixed tie-breaking (unique result):
 *  - graph: the pattern of A + A^T without self loops; degree = number of
 *    distinct neighbours;
 *  - components in order of their smallest node; each starts at a
 *    pseudo-peripheral node: r = the node of minimum (degree, index), then
 *    repeatedly the node of minimum (degree, index) in the last level of r's
 *    breadth-first level structure replaces r while its structure is deeper;
 *  - Cuthill-McKee breadth-first order from r, each node appending its
 *    unvisited neighbours in ascending (degree, index); perm is the reverse
 *    of that order (perm[new] = old).
 * ------------------------------------------------------------------------- */
typedef struct spmv_reorder* spmv_reorder_handle;

/* RCM permutation of a square HOST CRS pattern (n x n): perm[n] (host). */
spmv_status spmv_rcm(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* perm);

/* A' = P A P^T for perm[new] = old (host arrays): row r of A' is row perm[r]
 * of A with every column c relabelled to inv[c] (inv[perm[r]] = r) and the
 * entries sorted by the new column (stable: duplicates keep their order).
 * out_row_ptr[n+1], out_col_idx / out_val [nnz].  perm must be a permutation
 * of 0..n-1 (else SPMV_ERR_ARG). */
spmv_status spmv_permute_csr(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                             const int32_t* perm, int32_t* out_row_ptr, int32_t* out_col_idx, double* out_val);

/* A validated permutation on the current device, to move k-column row-major
 * blocks between the original and the permuted row order:
 *   gather:  Y[r*ldy + c] = X[perm[r]*ldx + c]   (original -> permuted order)
 *   scatter: Y[perm[r]*ldy + c] = X[r*ldx + c]   (permuted -> original order)
 * for r < n, c < k; X and Y are distinct device blocks; asynchronous. */
spmv_status spmv_reorder_create(int64_t n, const int32_t* perm, spmv_reorder_handle* out);
spmv_status spmv_reorder_gather(spmv_reorder_handle h, int32_t k, const double* X_dev, int64_t ldx, double* Y_dev,
                                int64_t ldy, void* stream);
spmv_status spmv_reorder_scatter(spmv_reorder_handle h, int32_t k, const double* X_dev, int64_t ldx, double* Y_dev,
                                 int64_t ldy, void* stream);
spmv_status spmv_reorder_destroy(spmv_reorder_handle h);

/* ----------------------------------------------------------------------------
 * Measurement probes: the machine side of the balance model.  Sec. 2 sets the
 * code balance of Eq. 1 against the machine's measured memory bandwidth
 * (STREAM); on this GPU two more rates bound forms of the product, and these
 * probes measure them with kernels of their own (CUDA events on a private
 * stream, best of `reps` launches after one untimed launch; synchronous on the
 * current device; each allocates and frees its own device buffers).
 * ------------------------------------------------------------------------- */

/* FP64 fused multiply-add rate: every thread of a grid filling all SMs runs 8
 * independent FMA chains with register operands.  *gflops = 2 x FMAs / time
 * (1e9 flop/s); *ms the best launch time; *sm_count the device's
 * multiprocessors; *sm_mhz the SM clock during that launch (clock cycles over
 * %globaltimer nanoseconds, averaged over the CTAs), so that
 * gflops / (2 x sm_count x sm_mhz) is the FMA rate per SM and clock.  Any
 * output may be NULL.  Bounds the products with k >= 2 columns, where each
 * stored entry needs k FMAs (and the batch, the solvers). */
spmv_status spmv_probe_fp64(int32_t reps, double* gflops, double* ms, int32_t* sm_count, double* sm_mhz);

/* Random 8-byte read rate: a grid filling all SMs reads uniformly random
 * entries of a zero-filled buffer of n_elems doubles (1 <= n_elems <=
 * 2^31-1) with read-only loads, 8 independent reads in flight per thread.
 * *gathers_per_s = reads / time; *ms the best launch time; *sm_mhz the SM
 * clock during it (as for spmv_probe_fp64).  A buffer the size of B of the
 * eigenproblem-shaped workload (6,201,600 doubles, 50 MB) stays in L2; every
 * read of a sector that the SM's L1 does not hold costs one request from the
 * SM's L1 to the crossbar, and those requests, about one per SM and clock,
 * bound a product whose B gathers are scattered. */
spmv_status spmv_probe_gather(int64_t n_elems, int32_t reps, double* gathers_per_s, double* ms, double* sm_mhz);

/* ----------------------------------------------------------------------------
 * Matrix features read by the cost model (host computation, no device use).
 * out[34] (float64) for HOST CRS arrays and k right-hand sides:
 *   [0:13]  fraction of rows in length bin b: b(L) = 0 for L = 0, else
 *           min(1 + floor(log2 L), 12) (bin 12 holds L >= 2048)
 *   [13:26] fraction of nonzeros in the rows of bin b
 *   [26] log2(1 + n_rows)      [27] log2(1 + nnz)        [28] nnz / n_rows (Nnzr)
 *   [29] log2(1 + max L)       [30] std(L) / (1 + Nnzr)  [31] max |i - j| / n_cols
 *   [32] mean over non-empty rows of (max col - min col) / n_cols
 *   [33] log2(k)
 * Row-length statistics and the bandwidth follow the paper's discussion of
 * Nnzr and of B-access locality (Sec. 1.2, Sec. 2).  Malformed CRS -> SPMV_ERR_CSR.
 * ------------------------------------------------------------------------- */
spmv_status spmv_features(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                          int32_t k, double* out);

/* ----------------------------------------------------------------------------
 * Host-side format builders (no device use): the builders that spmv_create and
 * spmv_set_variant run, on HOST CRS arrays (validated as in spmv_create:
 * malformed CRS -> SPMV_ERR_CSR; val may be NULL only when nnz = 0).  Two-call
 * pattern: with the first output array NULL a call returns only the sizes; a
 * second call with arrays of those sizes (caller-owned) fills them.  The
 * arrays are the ones spmv_sell_export / spmv_split_export / spmv_sym_export
 * copy from a plan, byte for byte.
 *
 * SELL-C-sigma, C = 32 (Kreutzer et al. 2014; the CRS loop of Sec. 1.2 on a
 * sliced, sorted, column-major form): sigma >= 1 (else SPMV_ERR_ARG).
 *   perm int32[n_rows], chunk_ptr int64[n_chunks + 1], chunk_len int32[n_chunks],
 *   sell_col int32[n_slots], sell_val float64[n_slots].
 * Local/halo split at column h (Sec. 3.1): 0 <= h <= n_cols (else SPMV_ERR_ARG).
 *   loc_row_ptr int32[n_rows + 1], loc_col int32[loc_nnz], loc_val float64[loc_nnz],
 *   halo_rows int32[n_halo_rows], halo_row_ptr int32[n_halo_rows + 1],
 *   halo_col int32[halo_nnz], halo_val float64[halo_nnz].
 * Symmetric triangle (Sec. 1.3.1): the entries with col >= row of each row;
 *   SPMV_ERR_UNSUPPORTED (reason in spmv_last_error) unless the matrix is
 *   square and symmetric.  sym_row_ptr int32[n_rows + 1], sym_col int32[sym_nnz],
 *   sym_val float64[sym_nnz].
 * ------------------------------------------------------------------------- */
spmv_status spmv_sell_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                 const double* val, int32_t sigma, int64_t* n_chunks, int64_t* n_slots,
                                 int32_t* perm, int64_t* chunk_ptr, int32_t* chunk_len, int32_t* sell_col,
                                 double* sell_val);
spmv_status spmv_split_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                  const double* val, int64_t h, int64_t* loc_nnz, int64_t* n_halo_rows,
                                  int64_t* halo_nnz, int32_t* loc_row_ptr, int32_t* loc_col, double* loc_val,
                                  int32_t* halo_rows, int32_t* halo_row_ptr, int32_t* halo_col,
                                  double* halo_val);
spmv_status spmv_sym_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                const double* val, int64_t* sym_nnz, int32_t* sym_row_ptr, int32_t* sym_col,
                                double* sym_val);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_GB300_H */
