/*
 * zoomsvd.h - C ABI of the GB300 range-SVD library (Zoom-SVD, arXiv 1805.00754).
 *
 * The library keeps a compressed store of a growing T x n multi-series matrix
 * A (rows = time, columns = series; the paper's c is n here) and answers
 * "SVD of rows [t_s, t_e]" from it without the raw rows.
 *
 *   storage phase  (Section 3.2, Algorithm 1, Def. 1-2): A is cut into blocks
 *                  of b rows; block i is kept as its rank-k truncated SVD
 *                  U_i (rows_i x k), sigma_i (k), V_i (n x k).
 *   query phase    (Section 3.3, Algorithm 2-3, Def. 3-4, Eq. 5-9):
 *                  Partial-SVD of the two boundary blocks, SVD of the stacked
 *                  Sigma_i V_i^T slabs (Stitched-SVD), then the lift
 *                  U = diag(S:E) U_r.
 *
 * Conventions for every call:
 *   - Rows are 0-based; a range [t_s, t_e] is inclusive and holds
 *     t_e - t_s + 1 rows (Problem 1, Section 2.3).
 *   - Matrices are row-major.  "device" pointers are CUDA global-memory
 *     addresses on the store's device; "host" pointers are ordinary memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without waiting unless
 *     stated otherwise; results are ready when the stream reaches that point.
 *   - Every call returns a zs_status; nothing throws across the ABI.  On an
 *     error the store is unchanged unless stated otherwise, and
 *     zs_last_error() gives a one-line message for the calling thread.
 *   - Results are written in the store's factor type: double for a ZS_F64
 *     store, float for ZS_F32 and ZS_BF16 stores.
 */
#ifndef ZOOMSVD_H
#define ZOOMSVD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZS_OK = 0,
    ZS_EINVAL = 1,      /* bad argument (null pointer, size, config)        */
    ZS_ERANGE = 2,      /* t_s < 0, t_s > t_e, or t_e >= rows appended      */
    ZS_ENOMEM = 3,      /* device or host allocation failed / capacity full */
    ZS_EBUSY = 4,       /* serving queue full; try again                    */
    ZS_ETIMEDOUT = 5,   /* a bounded wait ran out                           */
    ZS_EDTYPE = 6,      /* unsupported dtype combination                    */
    ZS_ECUDA = 7,       /* a CUDA runtime call failed                       */
    ZS_EINTERNAL = 8,   /* invariant violated inside the library            */
    ZS_ENOTFOUND = 9,   /* unknown ticket / block index                     */
    ZS_ENOCONV = 10     /* a truncated SVD did not pass its accuracy test
                           within the iteration cap (results are the last
                           iterate; see zs_store_status)                    */
} zs_status;

typedef enum { ZS_F64 = 0, ZS_F32 = 1, ZS_BF16 = 2 } zs_dtype;

/* Store flags. */
enum {
    /* Re-solve each small eigen core (k x k, Rayleigh-Ritz m x m) in FP64
     * after the FP32 Jacobi sweeps: FP64-accumulated Rayleigh quotient and one
     * FP64 Jacobi refinement sweep.  No effect on ZS_F64 stores (all FP64).  */
    ZS_FLAG_FP64_REFINE = 1,
    /* Compute every Gram matrix exactly in FP32 on the CUDA cores (slower)
     * instead of the default for float stores with n >= 64: a bf16
     * tensor-core Gram that only locates the dominant subspace, followed by a
     * split-bf16 (~FP32) projection and Rayleigh-Ritz that sets the accuracy. */
    ZS_FLAG_EXACT_GRAM = 2,
    /* Algorithm 1 as printed (Section 3.2, Eq. 2-3): every appended row
     * updates its block's rank-k SVD through the SVD of the (k+1) x n matrix
     * [Sigma V^T; a] and U <- blockdiag(U, 1) U~, truncated back to rank k
     * after every row - O(k^2 (rows + n)) per row (Theorem 1) instead of
     * recompressing the open block on each append.  The stored factors are
     * then the paper's row-by-row approximation, which equals the block's
     * truncated SVD when the block's rank is at most k and otherwise keeps
     * less energy (each row drops the (k+1)-th singular value of its stacked
     * matrix).  Needs (k+1)(2n + k + 1) factor elements of shared memory
     * (<= 227 KB); not combined with zs_store_set_xi.                     */
    ZS_FLAG_ROW_APPEND = 4
};

typedef struct zs_store zs_store;
typedef struct zs_server zs_server;

typedef struct {
    int64_t n;              /* series (columns), 1..1024                     */
    int64_t b;              /* block rows (Def. 1), >= 1                     */
    int32_t k;              /* stored rank per block, 1..64, <= n            */
    int32_t in_dtype;       /* zs_dtype of the rows given to zs_store_append */
    int64_t capacity_rows;  /* most rows the store will ever hold; the store
                               preallocates its factor arrays for this many */
    int32_t device;         /* CUDA device ordinal                           */
    int32_t flags;          /* ZS_FLAG_*                                     */
} zs_store_config;

/* Caller-owned device buffers for one query result (factor type). */
typedef struct {
    void* U;          /* (t_e - t_s + 1) x k_out, row stride ldu (elements) */
    int64_t ldu;      /* >= k_out                                            */
    void* S;          /* k_out singular values, descending                   */
    void* V;          /* n x k_out, row stride ldv (elements)               */
    int64_t ldv;      /* >= k_out                                            */
    int32_t* rank;    /* device int32: number of nonzero singular values;
                         may be NULL                                          */
} zs_result;

/* ------------------------------------------------------------------------
 * Store (Def. 2: the sets U, S, V).
 * ------------------------------------------------------------------------ */

/* Create an empty store on cfg->device.  Allocates the factor arrays for
 * cfg->capacity_rows rows (ceil(capacity_rows / b) blocks of
 * b*k + k + k*n factor elements each) plus the open-block staging buffer.
 * *out receives the handle (owned by the caller; free with
 * zs_store_destroy).  ZS_EINVAL on a bad config, ZS_EDTYPE on an unknown
 * dtype, ZS_ENOMEM if the device allocation fails.                         */
zs_status zs_store_create(const zs_store_config* cfg, zs_store** out);

/* Destroy a store and free its device memory.  Waits for work the library
 * enqueued on its own streams; the caller must not use the handle after.   */
void zs_store_destroy(zs_store* st);

/* Storage phase (Algorithm 1, Def. 1; Theorem 1 cost model).
 * Append nrows rows (row stride ld >= n elements of cfg.in_dtype; bf16 as
 * raw 16-bit patterns) to the matrix.  rows_on_device selects whether `rows`
 * is a device pointer (1) or a host pointer (0; copied before the call
 * returns, so the caller may reuse it).  Every block completed by these
 * rows is compressed to its rank-k truncated SVD; the rows of the still-open
 * last block are kept on the device and that block is (re)compressed as it
 * stands, so a query may touch every appended row (reading: a short block is
 * the paper's "current block" of Def. 1).  Work is enqueued on `stream`;
 * other streams must order after it before querying the new rows.
 * ZS_ENOMEM if capacity_rows would be exceeded (nothing appended).          */
zs_status zs_store_append(zs_store* st, const void* rows, int64_t nrows, int64_t ld,
                          int32_t rows_on_device, void* stream);

/* Forget every appended row (the factor arrays stay allocated), so the store
 * can be refilled.  Waits for the store's outstanding work to finish.      */
zs_status zs_store_reset(zs_store* st);

/* Host-side counters: rows appended, blocks (closed + open), and device
 * bytes held by the compressed factors (Theorem 3).  Any pointer may be
 * NULL.                                                                     */
zs_status zs_store_info(const zs_store* st, int64_t* rows, int64_t* nblocks,
                        int64_t* factor_bytes);

/* Energy rule (Eq. 1) for the blocks compressed from now on: xi in (0, 1]
 * gives block i the rank k_i = the smallest rank whose leading singular
 * values hold a fraction >= xi of ||X_i||_F^2 (the sum of all the block's
 * sigma_j^2), capped at the store's k; columns k_i.. of its U, sigma and V
 * are stored as zeros (the arrays keep width k).  While xi > 0, queries on
 * float stores with n >= 64 stack only the live rows (nonzero sigma) of each
 * interior block (ragged stacks); other stores treat the zero rows as rank
 * deficiency.  xi = 0 restores the fixed rank k.  Costs one more read of each
 * block's rows per append.  ZS_EINVAL for xi outside [0, 1], ZS_ENOMEM if the
 * per-block scratch (12 bytes per block of capacity) cannot be allocated.   */
zs_status zs_store_set_xi(zs_store* st, double xi);

/* Per-block ranks and energies (Eq. 1; Theorem 3; the reconstruction error
 * of Section 5.4).  Synchronises the device.  For blocks 0 .. nblocks-1
 * (host arrays, any may be NULL): ranks[i] = k_i, the energy rule's rank in
 * xi mode (its columns are the nonzero ones) or min(k, rows_i, n) at fixed
 * rank; kept[i] = sum_{j < k_i} sigma_ij^2, the energy the block keeps;
 * energy[i] = ||X_i||_F^2 as measured when the block was compressed in xi
 * mode, else -1.  The paper's space for the store is
 * sum_i k_i (b + n + 1) values, and 1 - sum kept / sum energy is the
 * stored blocks' relative squared reconstruction error (Eckart-Young).
 * ZS_ENOTFOUND if nblocks exceeds the store's blocks.                      */
zs_status zs_store_block_stats(const zs_store* st, int64_t nblocks, int32_t* ranks, double* kept, double* energy);

/* Device fault word of the store (failure detection): 1 once a kernel of
 * this store gave up a bounded wait on the device (the tensor-core
 * projection waits on its MMA completions with an iteration limit, then
 * drains its copies, releases its TMEM and returns, leaving its results
 * undefined); 0 otherwise.  Synchronises the device.  *flag (host) receives
 * the word; a non-zero word persists until the store is destroyed.        */
zs_status zs_store_fault(const zs_store* st, int32_t* flag);

/* Accuracy status of the store (Section 2.1: each stored block is the
 * rank-k truncated SVD of its rows; Algorithm 2: each answer the truncated
 * SVD of the stacked matrix).  On float stores every block and every
 * query's Stitched-SVD is tested on the device after it is computed: with
 * R = X^T U from the factors as written, rho_j = |X^T u_j - sigma_j v_j|
 * and the bound beta_j = min(rho_j, rho_j^2 / (sigma_j - s_m)) on the
 * error of sigma_j (s_m the smallest Ritz value of the subspace), an item
 * passes when beta_j <= 1e-5 max(sigma_j, 1e-2 sigma_1) for every kept
 * pair (relative, and 1e-7 sigma_1 absolute for singular values below 1% of
 * sigma_1, where FP32 arithmetic on the rows bounds what can be certified).
 * Items that fail
 * are refined by subspace iteration (64 directions, at most 12 passes over
 * their rows); one that still fails keeps its last iterate and is counted
 * here.  Synchronises the device.  *unconverged_blocks and
 * *unconverged_queries (host, may be NULL) receive the counts since the
 * store was created, *refined_blocks and *refined_queries (may be NULL)
 * how many items needed refinement at all.  Returns ZS_ENOCONV if an
 * unconverged count is nonzero, ZS_ETIMEDOUT if the fault word of
 * zs_store_fault is set, else ZS_OK.  FP64 stores use an exact Gram
 * eigen-solver and never count here.                                       */
zs_status zs_store_status(const zs_store* st, int64_t* unconverged_blocks, int64_t* unconverged_queries,
                          int64_t* refined_blocks, int64_t* refined_queries);

/* Copy block i's stored factors into caller device buffers: U (rows_i x k,
 * ld k), sigma (k), Vt (k x n, ld n), on `stream`.  *rows_i and *k_i (host)
 * receive the block's row count and kept rank min(k, rows_i, n); columns
 * past k_i are zero.  ZS_ENOTFOUND for i outside [0, nblocks).            */
zs_status zs_store_export_block(const zs_store* st, int64_t i, void* U, void* sigma, void* Vt,
                                int32_t* rows_i, int32_t* k_i, void* stream);

/* Storage-phase compression that allocates nothing (the paper has no
 * counterpart; it serves callers that cannot allocate device memory: code
 * running while a CUDA graph is being captured, plug-ins whose host program
 * owns every device allocation through its own pool, or loops that must
 * never enter the allocator).  Compresses nrows device rows (row stride
 * ld >= n elements of in_dtype) into ceil(nrows / b) blocks exactly as
 * zs_store_append does, without a store: block j's factors go to caller
 * device buffers U + j*b*k (b x k, ld k; rows past a short last block are
 * zero), sigma + j*k (k) and Vt + j*k*n (k x n, ld n), in the factor type
 * (double for ZS_F64 input, else float).  flags takes ZS_FLAG_FP64_REFINE.
 * Its scratch is one fixed 32 MiB device array inside the library (held on
 * every device that loads the library until the process exits), worked
 * through in chunks of blocks.  One block's scratch must fit it: the n x n
 * Gram matrix (8 n^2 bytes for ZS_F64, 4 n^2 otherwise) and, for float
 * factors with n >= 64, a subspace basis (about 8 n m bytes, m = k + 16
 * rounded up to 8, at most 64) plus b x m projections and Rayleigh-Ritz
 * data (about 4 m (b + m (b / 128 + 2)) bytes); sizes over that are rejected
 * with ZS_EINVAL, whose message gives the bytes asked for.  The call makes
 * no cudaMalloc, cudaFree or other allocating call.  Every call uses the
 * same array and overwrites the parts it reads before reading them (nothing
 * has to start at zero), so calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and must be serialised by the
 * caller.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture, and do not call it again on a
 * device after cudaDeviceReset (the cached address is then stale).  Work is
 * enqueued on `stream`; zs_noalloc_status reports how the last call went.  */
zs_status zs_compress_noalloc(const void* rows, int64_t nrows, int64_t ld, int32_t in_dtype, int64_t n,
                              int64_t b, int32_t k, int32_t flags, void* U, void* sigma, void* Vt,
                              void* stream);

/* Status of the last zs_compress_noalloc call on the current device, read
 * from two words in the same fixed device array (cleared by each call, so it
 * allocates nothing either).  Synchronises the device.  *fault (host, may be
 * NULL) is 1 if a bounded wait of a tensor-core kernel gave up (the factors
 * are then undefined; returns ZS_ETIMEDOUT); *unconverged_blocks (may be
 * NULL) counts blocks that did not pass the accuracy test of
 * zs_store_status within its pass cap (returns ZS_ENOCONV); else ZS_OK.    */
zs_status zs_noalloc_status(int32_t* fault, int32_t* unconverged_blocks);

/* ------------------------------------------------------------------------
 * Query phase (Algorithm 2 with Partial-SVD Algorithm 3; Eq. 5-9).
 * ------------------------------------------------------------------------ */

/* SVD of rows [t_s, t_e] of the stored (rank-k per block) matrix, truncated
 * to k_out = 1..64 columns: U ((t_e-t_s+1) x k_out), S (k_out), V (n x
 * k_out) into *res.  Columns past the range's rank are zero.  Each pair
 * (u_j, v_j) is signed so that the largest-|.| entry of v_j is positive
 * (lowest index on ties).  ZS_ERANGE for a bad range.  Enqueued on stream;
 * the library's scratch is reused by the next call on the same store, so
 * calls on one store are serialised by the library.                        */
zs_status zs_query(zs_store* st, int64_t t_s, int64_t t_e, int32_t k_out,
                   const zs_result* res, void* stream);

/* nq queries in one batch (host arrays ts[nq], te[nq], results[nq]), all
 * with width k_out.  Planning is done on the host; the device work is a
 * fixed set of persistent work-list kernels (replayed as one CUDA graph
 * when the batch shape fits the captured capacity).  Each result equals
 * the one zs_query gives for the same range.  ZS_ERANGE if any range is
 * bad (nothing enqueued).                                                  */
zs_status zs_query_batch(zs_store* st, const int64_t* ts, const int64_t* te, int32_t nq,
                         int32_t k_out, const zs_result* results, void* stream);

/* The same batch with U returned factored (Algorithm 2's last step, Eq. 9,
 * left to the caller): results[q].S, .V and .rank are filled as by
 * zs_query_batch (.U is not used and may be NULL), and U_{S:E} stays as
 * diag(S:E) U_r in the form of one coefficient matrix per covered block.
 * coef (device, factor type, coef_rows x k_out, row-major) receives, for
 * query q with blocks S_q..E_q (S = t_s / b, E = t_e / b), the k x k_out
 * matrices C_{q,S}..C_{q,E} stacked from row k * sum_{p<q} (E_p - S_p + 1):
 * the answer's rows that fall in block i are the store's U_i rows for them
 * (zs_store_export_block) times C_{q,i}.  ZS_EINVAL if coef_rows is smaller
 * than k * sum_q (E_q - S_q + 1); otherwise as zs_query_batch.             */
zs_status zs_query_batch_factored(zs_store* st, const int64_t* ts, const int64_t* te, int32_t nq,
                                  int32_t k_out, const zs_result* results, void* coef, int64_t coef_rows,
                                  void* stream);

/* Similar-range search (Section 6, case study).  L = base_te - base_ts + 1;
 * the windows are the ranges [t, t + L - 1] with t = base_ts - j * stride
 * >= 0, j = 1 .. nwin, nwin = min(max_windows, base_ts / stride).  Each is
 * scored by the cosine <u_1, u_1^base> / (|u_1| |u_1^base|) of its first
 * left singular vector (as zs_query gives it with k_out = 1, so with the
 * same sign rule) with the base range's; a zero vector scores 0.  starts
 * (host int64, >= max_windows entries) receives the window starts in that
 * order, cos (host double, >= max_windows) their scores, *nwin (host) the
 * count.  The windows run through zs_query_batch in chunks; the call
 * allocates its scratch (the base's and one chunk's first vectors), works
 * on `stream`, synchronises it and frees the scratch before it returns.
 * ZS_ERANGE for a bad base range, ZS_EINVAL for stride < 1 or a null
 * pointer, ZS_ENOMEM if the scratch cannot be allocated.                   */
zs_status zs_similar_ranges(zs_store* st, int64_t base_ts, int64_t base_te, int64_t stride, int32_t max_windows,
                            int64_t* starts, double* cos, int32_t* nwin, void* stream);

/* Autotuner (no counterpart in the paper): times the query launch set on
 * nq deterministic ranges of the store's current rows under candidate grid
 * shapes (persistent CTAs per SM of the slab work-list and projection
 * kernels), keeps the fastest for this store and, if the environment
 * variable ZS_TUNE_CACHE names a file, records it there keyed by
 * (n, b, k, dtype, flags, SM count); stores created later with the same key
 * start from the cached choice.  Results do not depend on the choice.  Needs
 * appended rows; allocates temporary result buffers; synchronises `stream`. */
zs_status zs_store_autotune(zs_store* st, int32_t nq, void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of range queries (no counterpart in the
 * paper; it serves the paper's query phase to concurrent callers).
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t max_batch;        /* most queries launched in one batch          */
    int32_t max_inflight;     /* batches on the device at once (streams)     */
    int32_t queue_capacity;   /* pending requests before submit says EBUSY   */
    int64_t memory_budget;    /* device scratch bytes all in-flight batches
                                 may hold; requests wait until it frees up   */
} zs_serve_config;

typedef struct {
    int64_t completed;
    int64_t rejected;         /* submits refused with ZS_EBUSY              */
    int64_t batches;
    double p50_ms, p99_ms, max_ms, mean_ms;   /* submit -> result ready     */
    double wall_s;            /* start -> stop                               */
    double queries_per_s;     /* completed / wall_s                          */
    double mean_batch;
} zs_serve_stats;

/* Start a serving thread on the store's device.  The store must outlive the
 * server.  Appends may continue on other streams; a request sees the rows
 * whose append call returned before the request was submitted.            */
zs_status zs_serve_start(zs_store* st, const zs_serve_config* cfg, zs_server** out);

/* Queue one range query; dst holds caller device buffers that must stay
 * valid until the request is done.  Non-blocking.  *ticket identifies it.
 * ZS_EBUSY when the queue is full, ZS_ERANGE for a bad range.             */
zs_status zs_serve_submit(zs_server* sv, int64_t t_s, int64_t t_e, int32_t k_out,
                          const zs_result* dst, uint64_t* ticket);

/* *done = 1 once the request's results are on the device (and *req_status
 * holds its status), else 0.  ZS_ENOTFOUND for an unknown ticket.          */
zs_status zs_serve_poll(zs_server* sv, uint64_t ticket, int32_t* done, int32_t* req_status);

/* Block until the request is done or timeout_ms passes (ZS_ETIMEDOUT).     */
zs_status zs_serve_wait(zs_server* sv, uint64_t ticket, int64_t timeout_ms, int32_t* req_status);

/* Drain queued requests, stop the thread, fill *stats (may be NULL) and
 * free the server.                                                        */
zs_status zs_serve_stop(zs_server* sv, zs_serve_stats* stats);

/* ------------------------------------------------------------------------
 * Misc.
 * ------------------------------------------------------------------------ */
const char* zs_status_str(zs_status s);
const char* zs_last_error(void);

/* Number of kernel launches the library has issued in this process (all
 * stores), for launch accounting.                                          */
int64_t zs_launch_count(void);

/* Kernel profiler (tracing).  While enabled, every kernel launch is
 * bracketed by CUDA events recorded on its launch stream; zs_profile_get
 * synchronises on those events and reports, for the i-th kernel name seen,
 * its launch count and summed device time.  zs_profile_reset clears the
 * table.  Off by default; costs two event records per launch when on.     */
void zs_profile_enable(int32_t on);
void zs_profile_reset(void);
int32_t zs_profile_count(void);
zs_status zs_profile_get(int32_t i, const char** name, int64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif
#endif /* ZOOMSVD_H */
