/*
 * spin.h -- C ABI of the GB300 (sm_103a) library for Strassen's
 * block-recursive matrix inversion (Misra, Haldar, Bhattacharya, Ghosh,
 * "SPIN: A Fast and Scalable Matrix Inversion Method in Apache Spark",
 * ICDCN'18, arXiv 1801.04723).
 *
 * Problem statement (Sec. 3.1, Algorithm 1; Sec. 3.3, Algorithm 2): given a
 * square n x n matrix A and a threshold (block size), return C = A^-1.  A is
 * split into quadrants A11, A12, A21, A22 and
 *     I = A11^-1, II = A21 I, III = I A12, IV = A21 III, V = IV - A22,
 *     VI = V^-1, C12 = III VI, C21 = VI II, VII = III C21, C11 = I - VII,
 *     C22 = -VI,
 * recursing on A11 and V until the block order reaches the threshold, where
 * the block is inverted directly.  The method has no pivoting across blocks:
 * A11 and every Schur complement must be invertible (Sec. 2.1 restricts the
 * method to positive definite invertible matrices; strictly diagonally
 * dominant matrices qualify as well).
 *
 * Conventions shared by every call:
 *   - Matrices are FP64, row-major, with a leading dimension (elements
 *     between consecutive rows) >= the number of columns.  The paper stores
 *     blocks column-major (Sec. 3.2); since (A^T)^-1 = (A^-1)^T a column-major
 *     caller passes its buffers unchanged and reads a column-major inverse.
 *   - Device pointers are CUDA device (or managed) memory of the current
 *     device, 8-byte aligned.  The caller owns A and X; A is never written.
 *     A and X must not overlap (the paper's inversion is out of place).
 *   - Work is enqueued on the given stream (0 = legacy default stream).
 *   - Return values are spin_status codes.  Argument errors are detected on
 *     the host before anything is enqueued.  Numerical failure (a zero or
 *     non-finite pivot in a leaf, i.e. a singular A11 or Schur complement
 *     somewhere in the recursion) is detected on the device and reported
 *     through the info record; X is then undefined, but the call never
 *     returns SPIN_OK with a result it knows to be wrong.
 *   - Split rule for orders that are not powers of two (the paper treats
 *     n = 2^p only, Sec. 4): n1 = 32*ceil(n/64) when n > 64, else ceil(n/2);
 *     n2 = n - n1.  A block is a leaf when its order is <= the leaf size.
 */
#ifndef SPIN_H
#define SPIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* spin_stream_t; /* == cudaStream_t */

typedef enum {
    SPIN_OK = 0,
    SPIN_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or option          */
    SPIN_ERR_SINGULAR = 2,      /* zero or non-finite leaf pivot (A11 or a Schur complement) */
    SPIN_ERR_NOT_CONVERGED = 3, /* refinement did not reach the requested residual           */
    SPIN_ERR_OOM = 4,           /* device memory for the workspace could not be obtained      */
    SPIN_ERR_CUDA = 5,          /* a CUDA call failed (launch, copy, event)                   */
    SPIN_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                         */
    SPIN_ERR_BUSY = 7,          /* serving: the request is not finished yet                   */
    SPIN_ERR_NOT_IMPLEMENTED = 8
} spin_status;

typedef enum {
    SPIN_FP64 = 0,         /* every product in FP64 (plain method)                           */
    SPIN_MIXED_BF16X3 = 1, /* products on BF16 tensor cores with 3-term splits, FP32 accumulate,
                              then Newton-Schulz refinement to opts.tol                       */
    /* 2 is not a precision (a call passing it gets SPIN_ERR_INVALID_ARG)                     */
    SPIN_MIXED_DIGITS = 3  /* products on BF16 tensor cores as 4-slice fixed-point digit
                              products with exact FP32 runs (~2^-30 relative), then the same
                              refinement -- which usually stops at its first, certifying
                              residual                                                    */
} spin_precision;

/* How spin_invert_batched runs a plain batch (spin_opts.schedule). */
typedef enum {
    SPIN_SCHEDULE_DEFAULT = 0,
    SPIN_SCHEDULE_LOCKSTEP = 1,
    SPIN_SCHEDULE_PERSISTENT = 2
} spin_batch_schedule;

/* Options of spin_invert_ex.  Zero-initialise and set what you need;
 * spin_opts_default() returns the defaults. */
typedef struct spin_opts {
    int32_t precision;         /* spin_precision; default SPIN_FP64                            */
    int32_t leaf;              /* leaf block order; 0 = library choice for this n and precision */
    double tol;                /* mixed modes: target ||AX-I||_F/(||A||_F||X||_F); default 1e-10 */
    int32_t max_refine;        /* mixed modes: Newton-Schulz iteration cap; default 6          */
    int32_t fp64_levels;       /* mixed modes: top recursion levels whose Schur complement
                                  V = IV - A22 is formed FP64-accurately; default 2            */
    int32_t blocking;          /* 1: synchronise the stream and fill *info before returning    */
    int32_t residual_slices;   /* mixed modes: 8-bit digit slices of the FP64-class refinement
                                  residual, 1..7 (every round); 0 (default) = chosen per order
                                  from the residual's error model (about 0.6 sqrt(n)
                                  2^-(8s-1) of ||A||_F ||X||_F): certifying residuals keep it
                                  within 1 % of tol, the first one, which only feeds the
                                  update, within 20 % (6 slices for tol = 1e-10 up to
                                  n = 32768; 7 for tol = 1e-13)                              */
    void* workspace;           /* optional caller device buffer (>= spin_workspace_bytes);
                                  NULL: the library uses its own cached per-device buffer     */
    size_t workspace_bytes;
    int32_t pretransform;      /* for matrices whose leading blocks may be singular (the
                                  recursion does not pivot across blocks):
                                  0 (default) none;
                                  1 random butterfly transform of depth 2: X = V (U^T A V)^-1 U^T
                                    with U, V recursive butterflies (A padded with the identity
                                    to a multiple of 4); the mixed modes then refine X against A;
                                  2 the plain recursion first, and on a zero or non-finite pivot
                                    the transform (the call then waits for the first attempt)  */
    int32_t schedule;          /* launch schedule (spin_batch_schedule).
                                  spin_invert_batched, plain form: 0 (default) the persistent
                                  kernel -- one launch that walks a device-side task list --
                                  unless leaf > 64; 1 lockstep launches per order bucket on a
                                  pool of streams; 2 the persistent kernel (leaf > 64 refused).
                                  The persistent kernel inverts leaves of order <= 64 on one
                                  CTA each: a larger leaf chosen by the library (n for
                                  n <= 128, or an autotuned one) becomes 64.  The mixed batch
                                  ignores it.
                                  spin_invert_ex and the calls built on it: 0 (default) each
                                  level's II = A21 I and C21 run on a second stream beside the
                                  recursion on S up to order 8192 (plain) or 16384 (mixed);
                                  1 one stream, in Algorithm 1's order; 2 the second stream at
                                  every order.  The same products on the same operands either
                                  way, so the same results bit for bit; the second stream
                                  needs II's slab and (mixed) a second split arena in the
                                  workspace (spin_workspace_bytes takes the schedule)        */
    uint64_t rbt_seed;         /* seed of the butterflies' random diagonals (splitmix64)      */
} spin_opts;

/* Result record of one inversion. */
typedef struct spin_info {
    int32_t status;            /* spin_status of the numerical work                            */
    int32_t refine_iters;      /* Newton-Schulz iterations taken (mixed modes)                 */
    int64_t fail_leaf;         /* leaf index (execution order) whose pivot failed, else -1     */
    int64_t fail_col;          /* pivot column inside that leaf, else -1                       */
    double rel_residual;       /* last computed ||AX-I||_F/(||A||_F||X||_F); -1 if none        */
    int32_t pretransformed;    /* 1 if the result came through the random butterfly transform */
    int32_t reserved;
} spin_info;

spin_opts spin_opts_default(void);

/*
 * spin_invert: X = A^-1 by the plain method (Algorithm 1, every product in
 * FP64; leaves by Gauss-Jordan with partial pivoting, the direct leaf
 * inversion that Alg. 1 and Alg. 2 leave open).
 *   A    device, n x n, leading dimension lda >= n, read only.
 *   X    device, n x n, leading dimension n, written.
 *   n    order, >= 1.
 *   leaf leaf block order, 1 <= leaf; 0 = library choice.  leaf >= n inverts
 *        A directly.
 * Blocking: returns after the stream has finished the inversion, with the
 * numerical status (SPIN_OK or SPIN_ERR_SINGULAR) as the return value.
 * Workspace: the library's cached per-device buffer (grown on demand).
 */
int spin_invert(const double* A, double* X, int64_t n, int64_t lda, int leaf, spin_stream_t stream);

/*
 * spin_invert_ex: the general form.  X (n x n, leading dimension ldx >= n).
 * opts may be NULL (defaults).  With opts->blocking, or when info is not
 * NULL, the call synchronises the stream and fills *info; otherwise it
 * returns once the work is enqueued and spin_sync() reads the status later.
 * Mixed precisions refine until opts->tol or opts->max_refine: rounds
 * 0 .. max_refine of Newton-Schulz are all enqueued and the stopping
 * decision is taken on the device after each residual (a converged matrix
 * skips the remaining rounds' work), so they do not synchronise the stream
 * unless blocking or info asks for it; pretransform = 2 waits once for the
 * first attempt's status.  The caller-provided workspace (opts->workspace)
 * must be 256-byte aligned.
 * Schedule: the recursion (Algorithm 2's driver) is a DAG of product and
 * leaf launches over views of X, A and the workspace, on the stream and, up
 * to order 8192 in FP64, a second library stream (II, then C21, beside the
 * main chain).  A call whose arguments (pointers, leading dimensions,
 * order, options, workspace) equal the previous call's on the same stream
 * captures that DAG into a CUDA graph, and later calls with the same
 * arguments replay it (one graph launch; the dependencies are resolved on
 * the device, and the graph reads A's current contents).  Calls made while
 * spin_profile_start is active, and pretransform = 2, launch directly.
 */
int spin_invert_ex(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n,
                   const spin_opts* opts, spin_info* info, spin_stream_t stream);

/*
 * spin_invert_batched: X[i] = A[i]^-1 for `count` independent matrices of
 * any orders (the paper inverts one matrix at a time; the batch is this
 * library's form of its many-block parallelism, Sec. 3.3).
 *   A, X     host arrays of `count` device pointers (X[i] has leading
 *            dimension n[i]); lda, n: host arrays.  Matrices may not overlap.
 *   opts     NULL or spin_opts: precision SPIN_FP64 (plain method) or
 *            SPIN_MIXED_BF16X3 (tensor-core level products, FP64 leaves,
 *            FP64-class Schur complements at the top fp64_levels levels,
 *            Newton-Schulz refinement of every matrix to tol); leaf (0 = the
 *            leaf spin_autotune_batched_leaf recorded for the order, else n
 *            for n <= 128 and 64 above), blocking, and for the mixed form tol,
 *            max_refine, fp64_levels and residual_slices are used.
 *   info_dev device int32[count] (may be NULL): status of each matrix
 *            (SPIN_OK, SPIN_ERR_SINGULAR, or SPIN_ERR_NOT_CONVERGED for the
 *            mixed form), written when the work ends.
 * Matrices of equal order form a bucket whose recursion runs in lockstep
 * (batched products, one leaf cluster per matrix); buckets run concurrently
 * on streams forked from `stream`.  The launch sequence is captured into a
 * CUDA graph on the first call and replayed while the arguments (pointers,
 * orders, leading dimensions, options) stay the same; the
 * workspace is library-owned.  The mixed form's refinement is part of the
 * graph: each matrix's stopping decision is taken on the device, so the
 * result of a matrix does not depend on the others in the batch, and the
 * call returns once the graph is enqueued (with opts->blocking, once it has
 * run).  count <= 65535, n[i] <= 65536.
 */
int spin_invert_batched(const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
                        int count, const spin_opts* opts, int* info_dev, spin_stream_t stream);

/* The random diagonals of the butterfly transform for order n (padded to
 * np, a multiple of 2^depth): 2 * depth * np doubles written to out_dev,
 * U's levels then V's, level k entry i = exp((u - 1/2) / 10) with u the
 * 53-bit uniform of splitmix64(seed) at counter (b * depth + k) * np + i.
 * For tests and for callers that apply the transform themselves. */
int spin_rbt_diagonals(uint64_t seed, int64_t n, int depth, double* out_dev, spin_stream_t stream);

/*
 * spin_autotune_batched_leaf: the block-size trade-off of Sec. 5.3 (the
 * U-shaped running time against the number of splits) per order bucket of
 * a batch.  orders: host array of the batch's `count` orders (repeats give
 * the bucket sizes); for every distinct order one lockstep run of its bucket
 * (seeded strictly diagonally dominant matrices, the same count) per
 * candidate leaf (host array of ncand orders; candidates above the order
 * are clamped to it), after a warm-up run, CUDA events around each; the
 * fastest leaf is recorded for (precision, order) and spin_invert_batched
 * with opts.leaf = 0 uses it (plans captured before are rebuilt).
 * precision: SPIN_FP64 or SPIN_MIXED_BF16X3.  leaf_out (host, count): the
 * chosen leaf for each entry of orders; ms_out (host, count, optional): its
 * time per bucket run.  Allocates the buckets' matrices and workspaces for
 * the duration of the call; synchronises the stream.  ncand = 0 (candidates
 * may be NULL) forgets the records of the listed orders instead and returns
 * the default leaves in leaf_out.  Errors: SPIN_ERR_INVALID_ARG (null
 * arrays, count < 1, an order outside [1, 65536], another precision),
 * SPIN_ERR_OOM (nothing is recorded).
 */
int spin_autotune_batched_leaf(const int64_t* orders, int count, int precision, const int* candidates, int ncand,
                               int* leaf_out, double* ms_out, spin_stream_t stream);

/* The persistent schedule a plain spin_invert_batched would run for these
 * orders (host only, no device work; count entries, leaf as opts.leaf,
 * 0..64): order buckets become stage lists (Algorithm 1's leaf inversions
 * and its six level products per node), merged into one task order.
 * Writes the stages, the tasks (matrix x output tile), the leaf inversions
 * and the products over all matrices, and their flops (2 L^3 per leaf,
 * 2 m n k per product; the method's total is 2 n^3 per matrix, Sec. 4).
 * Any output pointer may be NULL.  SPIN_ERR_INVALID_ARG for bad orders or
 * leaf; SPIN_ERR_CUDA if the task order breaks one of its invariants (each
 * bucket's stages in recursion order, every stage's dependency count equal
 * to the tasks of the bucket's earlier stages). */
int spin_batch_schedule_info(const int64_t* n, int count, int leaf, int64_t* stages, int64_t* tasks,
                             int64_t* leaves, int64_t* products, double* flops);

/*
 * spin_autotune_batched_persistent: the block-size trade-off of Sec. 5.3
 * for the persistent schedule of plain batches, per order bucket: leaf
 * size and product tile shape.  orders: host array of the batch's `count`
 * orders (repeats give the bucket sizes).  A batch of these orders (seeded
 * strictly diagonally dominant matrices) runs on the persistent kernel once
 * per candidate pair of leaf (host array of nleaf orders, each 1..64;
 * clamped to the order) and largest product tile (host array of ntile
 * values, each 16, 32 or 64; every product of a bucket then takes the
 * cheapest allowed tile by the schedule's cost rule), the pair applied to
 * every bucket, after a warm-up run.  The kernel adds the SM clocks of each
 * task to its bucket's counter (two counted runs, the smaller count kept),
 * and each bucket is given the pair under which its tasks took the fewest
 * clocks -- its share of the whole launch, measured beside the other
 * buckets -- when that beats the library's own pair (leaf 64, tile 64, or
 * the first candidate pair if that one is not among them) by 2 %.  The pairs are recorded per order:
 * plain spin_invert_batched calls with opts.leaf = 0 on the persistent
 * schedule use them (plans captured before are rebuilt).  leaf_out,
 * tile_out (host, count): the chosen pair per entry of orders; ms_out
 * (host, count, optional): the bucket's task time under it, in SM
 * milliseconds at the maximum SM clock.  Allocates the batch (two copies of
 * its matrices and its workspace) for the duration of the call;
 * synchronises the stream.  spin_autotune_batched_leaf with precision
 * SPIN_FP64 and ncand = 0 forgets both records.  Errors:
 * SPIN_ERR_INVALID_ARG (null arrays, count outside 1..65535, nleaf or
 * ntile < 1, an order outside [1, 65536], a leaf outside 1..64, a tile not
 * 16, 32 or 64), SPIN_ERR_OOM (nothing is recorded).
 */
int spin_autotune_batched_persistent(const int64_t* orders, int count, const int* leaves, int nleaf,
                                     const int* tiles, int ntile, int* leaf_out, int* tile_out, double* ms_out,
                                     spin_stream_t stream);

/* The persistent task list itself (host only, for checks of the device-side
 * schedule): per stage, in task order, five int64 -- kind (0 leaf
 * inversion, 1 level product), first matrix of its bucket (matrices sorted
 * by order, stable), matrices of the bucket, tasks per matrix, and the
 * dependency count (tasks of the matrix's earlier stages that must be done
 * before any of this stage's tasks starts) -- written to out (5 * max_stages
 * entries); *stages gets the stage count.  SPIN_ERR_INVALID_ARG for bad
 * orders or leaf (as spin_batch_schedule_info), or when the list has more
 * than max_stages stages (*stages is then set, out untouched). */
int spin_batch_schedule_stages(const int64_t* n, int count, int leaf, int64_t* out, int64_t max_stages,
                               int64_t* stages);

/* Shape of the graph the latest spin_invert_batched on `stream` replays:
 * kernel launches per call and order buckets.  SPIN_ERR_INVALID_ARG if none. */
int spin_batched_stats(spin_stream_t stream, int* kernels, int* buckets);

/* Mixed-form refinement of the latest spin_invert_batched on `stream`
 * (synchronises the stream): Newton-Schulz steps taken (the most over the
 * matrices) and the largest ||A X - I||_F / (||A||_F ||X||_F) over the
 * batch; -1 for a plain batch. */
int spin_batched_refine_info(spin_stream_t stream, int* refine_iters, double* worst_rel);

/* ---------------------------------------------------------------------
 * Serving: inversion requests admitted continuously by device-memory
 * footprint (the paper runs one job at a time; Sec. 5.1 sizes the Spark
 * executors so that no task fails for lack of memory -- here requests wait
 * for memory instead).  A request waits in a FIFO queue until one of
 * max_slots slots is free and its footprint (device copy of A when A is in
 * host memory, the result X, the workspace) fits hbm_budget_bytes; it then
 * runs on that slot's stream while other requests run on theirs.  The
 * result stays on the device, counted against the budget, until polled.
 * Continuous batching (the many-block parallelism of Alg. 2, Sec. 3.3, over
 * requests): a request of order n <= batch_max_order (precision SPIN_FP64
 * or SPIN_MIXED_BF16X3) is padded with the identity to the next multiple of
 * 32, and the slot that takes it also takes every queued request of the same
 * padded order, precision and tolerance (up to max_batch, within the
 * budget); the group runs as one lockstep batched recursion (one launch per
 * product and per leaf for all of it).  Such a request takes this path even
 * alone, and every decision in it is per matrix, so its result is the same
 * bit for bit whatever it is batched with.
 * ------------------------------------------------------------------- */
typedef struct spin_serve_cfg {
    size_t hbm_budget_bytes;  /* device memory the server may hold for requests       */
    int32_t max_slots;        /* requests running at once (one stream and thread each) */
    int32_t priority_order;   /* 0: off; else requests of order <= this run on
                                 high-priority streams, so that their kernels are
                                 scheduled ahead of a large request's pending blocks */
    size_t max_queued_bytes;  /* load shedding: 0 = unbounded queue; else a submit whose
                                 A (n*n*8 bytes) would take the bytes of A held by
                                 queued, not yet admitted, requests above this is
                                 refused with SPIN_ERR_BUSY and counted as shed (an
                                 empty queue accepts any request)                    */
    int32_t max_batch;        /* requests per batched launch group: 0 = 64; 1 = no
                                 batching (every request alone on the single path)  */
    int32_t batch_max_order;  /* orders above this are never batched: 0 = 1024; at most
                                 4096                                                 */
} spin_serve_cfg;

typedef struct spin_result {
    int32_t status;           /* spin_status of the inversion                          */
    int32_t refine_iters;
    int32_t precision;        /* spin_precision the request asked for                  */
    int32_t batch;            /* requests in the batched launch group it ran in (1: a
                                 group of its own); 0: the single-matrix path         */
    double rel_residual;      /* -1 for SPIN_FP64 (not computed)                       */
    double queue_ms;          /* submit -> admitted                                    */
    double run_ms;            /* admitted -> finished                                  */
    double latency_ms;        /* submit -> finished                                    */
} spin_result;

typedef struct spin_serve_stats_t {
    uint64_t submitted, completed, rejected, queued;
    int32_t running, peak_running;
    size_t bytes_in_use;
    uint64_t shed;            /* submits refused by max_queued_bytes                   */
    uint64_t deferred;        /* admissions put back in the queue because device memory
                                 could not be allocated (retried after another request
                                 completed; a request fails with SPIN_ERR_OOM only when
                                 it cannot be allocated while running alone)          */
    uint64_t groups;          /* batched launch groups run                             */
    uint64_t grouped;         /* requests those groups held                            */
    int32_t max_group;        /* largest group                                         */
    int32_t reserved;
} spin_serve_stats_t;

typedef struct spin_server spin_server;

/* Create a server on the current device.  SPIN_ERR_INVALID_ARG if
 * max_slots is outside 1..64 or the budget is 0. */
int spin_serve_create(const spin_serve_cfg* cfg, spin_server** out);

/* Queue X = A^-1.  A (host or device memory, n x n, leading dimension lda)
 * must stay valid and unchanged until the request is polled.  precision:
 * SPIN_FP64, SPIN_MIXED_BF16X3 or SPIN_MIXED_DIGITS (tol applies to the
 * mixed modes).  Returns a ticket; SPIN_ERR_OOM if the request alone
 * exceeds the budget; SPIN_ERR_BUSY (nothing queued, A may be released) if
 * cfg.max_queued_bytes would be exceeded. */
int spin_serve_submit(spin_server* sv, const double* A, int64_t lda, int64_t n, int precision, double tol,
                      uint64_t* ticket);

/* SPIN_ERR_BUSY while the request is queued or running.  When finished:
 * copies X (host or device memory, leading dimension ldx; NULL to drop the
 * result), fills *r, releases the request and returns SPIN_OK (the
 * numerical status is r->status). */
int spin_serve_poll(spin_server* sv, uint64_t ticket, double* X, int64_t ldx, spin_result* r);

/* Counters: submitted, completed, rejected, queued, running, peak running,
 * bytes held, shed, deferred, batched groups, requests in them, largest. */
int spin_serve_stats(spin_server* sv, spin_serve_stats_t* st);

/* Stop the slots (running requests finish), free everything. */
int spin_serve_destroy(spin_server* sv);

/*
 * spin_invert_noalloc: spin_invert for callers that must not allocate device
 * memory (the paper has no counterpart; it is a deployment variant).  A
 * process whose device memory is reserved up front by another allocator, or
 * code that cannot pay for the device-wide synchronisation of cudaMalloc /
 * cudaFree, can call this instead: it calls neither, and no allocating
 * library routine either.  Its workspace and status record live in one
 * fixed 8 MB array in device global memory that every GPU loading the
 * library keeps until exit, so the order is limited to problems whose
 * workspace fits it (n <= 1024 at any leaf <= 512; larger n, or a leaf whose
 * scratch does not fit, returns SPIN_ERR_INVALID_ARG before any work).
 *   A, X, n, lda, leaf, stream: as spin_invert (X has leading dimension n).
 * Blocking: the call synchronises `stream`, copies the 16-byte status
 * record into a host variable and returns the numerical status.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  CUDA loads a library's device code lazily, so
 * that first call is also when the driver places this library's kernels and
 * the 8 MB array on the device: a caller whose device memory will later be
 * reserved by another allocator makes one call (any small n) before that
 * happens; later calls add nothing to the device's memory use.  All calls on
 * a device share the one array, which keeps the previous call's contents
 * (each call clears the status record itself): calls that may overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller.
 */
int spin_invert_noalloc(const double* A, double* X, int64_t n, int64_t lda, int leaf, spin_stream_t stream);

/* Graph replays of spin_invert_ex on `stream` so far, and the node count
 * of its captured schedule (0 if none).  Host values; no synchronisation. */
int spin_schedule_stats(spin_stream_t stream, int64_t* replays, int64_t* nodes);

/* Synchronise the stream and fill *info with the status of the latest
 * non-blocking spin_invert_ex enqueued on it by this thread. */
int spin_sync(spin_stream_t stream, spin_info* info);

/* Device workspace, in bytes, that spin_invert_ex needs for this order and
 * these options (the value to pass as opts->workspace_bytes); it depends on
 * opts->schedule (the two-stream schedule keeps II per level and, in the
 * mixed forms, a second split arena).  0 for an order below 1, a leaf out
 * of range or a schedule outside 0..2. */
size_t spin_workspace_bytes(int64_t n, const spin_opts* opts);

/* The leaf order the library picks for n and a precision when leaf = 0:
 * n itself for n <= 128, else the autotuned choice for n's size class
 * (ceil(log2 n); a class above the largest tuned one reuses it), else a
 * built-in default (plain: 512 for n >= 16384, else 256; mixed: 128). */
int spin_default_leaf(int64_t n, int precision);

/* Predicted time (seconds) of one plain FP64 inversion of order n with the
 * given leaf on one GB300: the paper's cost analysis (Sec. 4, Table 2)
 * restated for this GPU -- six products per node priced by tile waves over
 * 152 SMs at the FP64 rate, leaves priced per pivot step on one thread-block
 * cluster.  spin_default_leaf uses its optimum for untuned FP64 orders.
 * -1 for other precisions or bad arguments. */
double spin_model_seconds(int64_t n, int leaf, int precision);

/*
 * spin_autotune_leaf: time one inversion (after a warm-up) per candidate
 * leaf order on a synthetic strictly diagonally dominant matrix of order n,
 * and record the fastest for n's size class and this precision; later calls
 * with leaf = 0 use it.  This is the block-size trade-off the paper studies
 * (Sec. 5.3, the U-shaped running time against the number of splits): many
 * small leaves leave the level products small and inefficient, few large
 * leaves make the serial leaf inversions dominate.  candidates: host array
 * of ncand orders (orders >= n are skipped); ms_out (optional, host, ncand)
 * receives each time (-1 if skipped).  Allocates two n x n matrices.
 */
int spin_autotune_leaf(int64_t n, int precision, const int* candidates, int ncand, int* leaf_out, double* ms_out,
                       spin_stream_t stream);

/*
 * spin_invert_host: X_host = A_host^-1 with both matrices in host memory
 * (pinned memory gives full copy bandwidth).  Copies A to the device, runs
 * spin_invert_ex on `stream`, copies X back, synchronises.  Device buffers
 * are the library's (cached per device).  lda/ldx as above.
 */
int spin_invert_host(const double* A_host, int64_t lda, double* X_host, int64_t ldx, int64_t n,
                     const spin_opts* opts, spin_info* info, spin_stream_t stream);

/* Human-readable name of a spin_status. */
const char* spin_status_string(int status);

/* Library version, major*10000 + minor*100 + patch. */
int spin_version(void);

/* Text of the last CUDA failure seen by this thread (SPIN_ERR_CUDA), or "". */
const char* spin_last_error(void);

/* ---------------------------------------------------------------------
 * Building blocks, exposed for testing and for callers that compose the
 * recursion themselves.  All are asynchronous on `stream`.
 * ------------------------------------------------------------------- */

/*
 * spin_leaf_inverse: X = A^-1 for one leaf block by Gauss-Jordan with
 * partial pivoting (largest |a_ik|, lowest row position on ties), the
 * paper's direct leaf inversion (Alg. 1, which leaves the method open;
 * Alg. 2 locInverse).  A: device n x n (lda), X: device n x n (ldx).
 * info_dev: device int32[4] {status, leaf_index, column, 0}; the first
 * failure is recorded (status 0 -> SPIN_ERR_SINGULAR) and later ones are
 * ignored; pass NULL to use the library's slot.  n <= 4096.
 */
int spin_leaf_inverse(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n,
                      int32_t* info_dev, spin_stream_t stream);

/*
 * spin_gemm_f64: D = beta*C + alpha*(A B) in FP64 (the paper's `multiply`
 * and `subtract` fused, Sec. 3.3), A m x k (lda), B k x n (ldb),
 * C and D m x n (ldc, ldd).  alpha in {+1,-1}; beta in {0, 1}; with beta = 0
 * C is not read (may be NULL).  D may equal C (in-place update) but must not
 * overlap A or B.
 */
int spin_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, const double* C, int64_t ldc, double* D, int64_t ldd,
                  spin_stream_t stream);

/*
 * spin_gemm_bf16x3: D = beta*C + alpha*(A B) on the BF16 tensor cores with
 * each FP64 operand split as hi + lo (hi = bf16(x), lo = bf16(x - hi)) and
 * the three leading products A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated
 * in FP32: the mixed method's level product (relative error ~2^-16 of
 * |A||B| plus FP32 accumulation).  Shapes, alpha/beta and aliasing rules as
 * spin_gemm_f64.  Split planes use a library-owned device arena.
 */
int spin_gemm_bf16x3(int64_t m, int64_t n, int64_t k, double alpha,
                     const double* A, int64_t lda, const double* B, int64_t ldb,
                     double beta, const double* C, int64_t ldc, double* D, int64_t ldd,
                     spin_stream_t stream);

/*
 * spin_gemm_ozaki: D = beta*C + alpha*(A B) (+ I when add_identity) with
 * FP64-class accuracy on the BF16 tensor cores: every row of A and column
 * of B is scaled by a power of two and cut into `slices` (1..7) fixed-point
 * digit slices of 8 bits (balanced digits of magnitude <= 128, exact in
 * BF16; 8 * slices - 1 bits in all); digit products (<= 2^14) are summed
 * exactly in FP32 runs of 1024, the runs in int32, and each slice-pair group
 * is scaled into the FP64 result (slice pairs (t, u) with t + u < slices).  The refinement residual
 * R = I - A X of the mixed method is this call with alpha = -1, beta = 0,
 * add_identity = 1.  sumsq_dev (device double, optional) receives
 * += sum of squares of D.
 */
int spin_gemm_ozaki(int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb,
                    double beta, const double* C, int64_t ldc, double* D, int64_t ldd,
                    int slices, int add_identity, double* sumsq_dev, spin_stream_t stream);

/* Synchronise `stream` and return (and clear) the device error word of the
 * building-block tensor-core calls: SPIN_OK, or SPIN_ERR_TIMEOUT if a
 * bounded device-side wait gave up. */
int spin_take_device_error(spin_stream_t stream);

/* Test hook for the leaf's bounded exchange waits: inverts the identity of
 * order L (2..256, the pushed-row leaf form on its widest cluster) with the
 * CTA of rank mute_rank sending nothing and every wait limited to limit_ms
 * (0 < limit_ms <= 4000).  The waits run out, the kernel leaves without a
 * fault or a hang, and the leaf's status is returned: SPIN_ERR_TIMEOUT.
 * SPIN_ERR_INVALID_ARG for a bad order, rank or limit. */
int spin_test_leaf_timeout(int64_t L, int mute_rank, double limit_ms);

/* Test hook for the persistent batch kernel's bounded dependency waits: a
 * plain batch of two matrices 2I of order 128 (leaf 64) in which the first
 * level product waits for a task count that nothing reaches, every wait
 * limited to limit_ms (0 < limit_ms <= 4000).  The wait runs out, the
 * kernel records SPIN_ERR_TIMEOUT, the remaining tasks skip their work, and
 * the launch ends without a fault or a hang; *status0 and *status1 get the
 * two matrices' statuses (both SPIN_ERR_TIMEOUT).  Synchronises the device.
 * SPIN_ERR_INVALID_ARG for a bad limit or a NULL pointer. */
int spin_test_persistent_timeout(double limit_ms, int* status0, int* status1);

/* ---------------------------------------------------------------------
 * Instrumentation: the paper times each method of the recursion
 * separately (Sec. 5, Table 3: leafNode, multiply, subtract, ...).  With
 * profiling on, every kernel the library enqueues on the stream is
 * bracketed by CUDA events and described by one record.
 * ------------------------------------------------------------------- */
typedef enum {
    SPIN_KERNEL_LEAF = 0,      /* Gauss-Jordan leaf inversion                     */
    SPIN_KERNEL_GEMM_F64 = 1,  /* FP64 fused level product                        */
    SPIN_KERNEL_GEMM_TC = 2,   /* tensor-core level product (mixed precisions)    */
    SPIN_KERNEL_SPLIT = 3,     /* FP64 -> low-precision operand split             */
    SPIN_KERNEL_RESIDUAL = 4,  /* refinement residual R = I - A X                 */
    SPIN_KERNEL_UPDATE = 5,    /* refinement update X <- X + X R                  */
    SPIN_KERNEL_OTHER = 6
} spin_kernel_kind;

typedef struct spin_prof_record {
    int32_t kind;     /* spin_kernel_kind                                          */
    int32_t depth;    /* recursion depth of the issuing node (root 0), -1 if none  */
    int64_t m, n, k;  /* GEMM m x n x k; leaf: m = n = order, k = 0                */
    double flops;     /* algorithmic flops: 2 m n k per product, 2 L^3 per leaf    */
    double bytes;     /* algorithmic bytes: operands read once, result written once */
    double ms;        /* device time between the bracketing events                 */
} spin_prof_record;

/* Start recording launches on `stream` (up to max_records; older ones are
 * kept, later ones dropped).  Host-side only; no device work. */
int spin_profile_start(spin_stream_t stream, int max_records);

/* Synchronise `stream`, stop recording, copy up to `max` records into out
 * (may be NULL) and the number recorded into *count. */
int spin_profile_stop(spin_stream_t stream, spin_prof_record* out, int max, int* count);

/* Measure the FP64 FMA throughput of this GPU with a DFMA-bound kernel on
 * every SM (about 0.1 s); *tflops receives 2 * FMAs / s / 1e12. */
int spin_probe_fp64_peak(double* tflops, spin_stream_t stream);

/* The same measurement on the FP64 tensor path: every warp issues
 * independent mma.sync m8n8k4 f64 (DMMA) chains on every SM (about 0.1 s);
 * *tflops receives 2 * FMAs / s / 1e12.  Sec. 4 prices the method by its
 * products, so the faster of the two FP64 forms is the one the plain path's
 * level products use (on GB300: DFMA, which this lets anyone re-check). */
int spin_probe_fp64_mma_peak(double* tflops, spin_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPIN_H */
