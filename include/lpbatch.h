/*
 * lpbatch.h -- C ABI of the GB300 batched dense simplex solver.
 *
 * The solver runs the simplex method of Gurung & Ray, "Simultaneous Solving
 * of Batched Linear Programs on a GPU" (arXiv 1802.08557), on many
 * independent LPs at once.  Each LP is
 *
 *     maximize   c^T x                    (Section 3, Eq. 1)
 *     subject to A x <= b                 (Eq. 2)
 *                x >= 0                   (Eq. 3)
 *
 * with A of size m x n.  The solve starts from the slack basis (Eq. 4) and
 * runs the two-phase method (Section 3) when some b_i < 0.  Each iteration is
 * Step 1 (entering variable: most negative reduced cost), Step 2 (leaving
 * variable: minimum ratio) and Step 3 (pivot: divide the pivot row by the
 * pivot element, rank-1 update of every other row), Section 3.1.  LPs of
 * different sizes may share a batch (the paper's Section 4 batches LPs of one
 * size only).
 *
 * Conventions (identical in every entry point):
 *  - All floating-point data is IEEE binary64.  A is row-major per LP.
 *  - Ties: the entering variable is the LOWEST variable index whose reduced
 *    cost lies within tau*max(1,|d*|) of the minimum d*; the leaving row is
 *    the LOWEST row index whose ratio lies within tau*max(1,|r*|) of the
 *    minimum r*.  Variables are numbered 0..n-1 (structural), n..n+m-1
 *    (slack of row i = n+i), n+m.. (artificials of the rows with b_i < 0).
 *  - A row takes part in the ratio test when its entry in the entering
 *    column is > eps_piv.  An LP is optimal when no eligible reduced cost is
 *    < -eps_opt, and infeasible when the phase-I optimum exceeds
 *    eps_feas*max(1, max_i |b_i|).
 *  - Error codes (lpb_err) report call failures; the outcome of each LP is
 *    an lp_status value, not an error.  No entry point aborts or exits.
 *  - Thread safety: distinct handles may be used from distinct threads; one
 *    handle must not be used by two threads at once.
 */
#ifndef LPBATCH_H
#define LPBATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Outcome of one LP (Section 3.1 halt conditions; Section 3 two-phase test). */
typedef enum {
    LP_OPTIMAL = 0,     /* no entering variable: the basis is optimal          */
    LP_INFEASIBLE = 1,  /* phase-I optimum > 0: Ax <= b, x >= 0 has no point    */
    LP_UNBOUNDED = 2,   /* Step 2 found no admissible ratio in phase II         */
    LP_ITER_LIMIT = 3,  /* max_iters pivots done without reaching a halt        */
    LP_NUMERICAL = 4    /* breakdown (non-finite pivot, unbounded phase I)      */
} lp_status;

/* Result of a call. */
typedef enum {
    LPB_OK = 0,
    LPB_EINVAL = 1,     /* bad argument (null pointer, size < 1, non-finite data, bad offset) */
    LPB_ENOMEM = 2,     /* device or host allocation failed                     */
    LPB_ECUDA = 3,      /* a CUDA runtime call failed (text in lpb_last_error)  */
    LPB_ETOOBIG = 4,    /* an LP exceeds the supported size                     */
    LPB_ENOTSOLVED = 5  /* results requested before any lp_batch_solve          */
} lpb_err;

/* Arithmetic of the tableau.
 *  LP_PREC_FP64: FP64 tableau (the paper's double precision, Section 5).
 *  LP_PREC_FP32_REFINE: FP32 tableau pivots; the basis it ends on is then
 *    certified in FP64 (refined x_B = B^-1 b and duals from the original A, b,
 *    c; primal and dual feasibility to 1e-9, duality gap, or a refined
 *    unbounded ray).  LPs that are not certified, or that end infeasible, at
 *    the iteration limit or in breakdown, are solved again with the FP64
 *    tableau.  Reported x, y, obj of certified LPs are FP64 values of the
 *    certified basis; iters counts the FP32 pivots.  No counterpart in the
 *    paper. */
enum { LP_PREC_FP64 = 0, LP_PREC_FP32_REFINE = 1 };

/* Tolerances and limits.  Fill with lpb_default_opts() and then override. */
typedef struct {
    int32_t precision;   /* LP_PREC_FP64 (default) or LP_PREC_FP32_REFINE         */
    int32_t max_iters;   /* pivots per LP, both phases; <= 0: 50*(m+n)             */
    double eps_opt;      /* default 1e-9                                          */
    double eps_piv;      /* default 1e-9                                          */
    double eps_feas;     /* default 1e-9                                          */
    double tau;          /* relative tie window, default 1e-12                    */
    int32_t block_threads; /* threads per LP (one CTA per LP); 0 = from the LP size;
                              with LP_PREC_FP32_REFINE, 32 = one warp per LP       */
    int32_t schedule;    /* LPB_SCHED_AUTO or LPB_SCHED_STREAMED                   */
} lp_batch_opts;

/* Kernel choice.  AUTO: shared-memory-resident tableau when it fits in one
 * CTA, else a global workspace slot per LP (persistent CTAs, many LPs at
 * once).  With LP_PREC_FP32_REFINE the FP32 tableau is in one CTA's shared
 * memory when it fits, else in a global workspace; the FP64 re-solve of an
 * uncertified LP runs in one CTA when its FP64 tableau fits, else on a
 * thread-block cluster (one LP's latency matters there).
 * STREAMED: global workspace for every LP (FP32_REFINE: the FP32 tableau of
 * every LP).  CLUSTER: as AUTO, but an FP64 tableau above one CTA is split by
 * rows over the shared memory of a thread-block cluster of 2-16 CTAs (the
 * smallest that holds it; all CTAs take the same decisions).  SINGLE: the
 * whole batch in one persistent launch -- CTAs (512 threads for LP_PREC_FP64,
 * 256 for LP_PREC_FP32_REFINE) take the LPs, longest work first, from one work
 * queue and keep each tableau in their shared memory when it fits 110 KB,
 * else in their global workspace slot; with LP_PREC_FP32_REFINE the LPs that
 * AUTO solves on one warp come last and are solved one per warp (each warp
 * of a CTA takes its own from the queue), and the FP64 re-solves of
 * uncertified LPs follow as separate launches (they need the whole pass's
 * queues).  Results are bit-identical under every schedule. */
enum { LPB_SCHED_AUTO = 0, LPB_SCHED_STREAMED = 1, LPB_SCHED_CLUSTER = 2, LPB_SCHED_SINGLE = 3 };

typedef struct lp_batch lp_batch;   /* opaque; owned by the library */

/* Where a pointer argument lives. */
enum { LPB_HOST = 0, LPB_DEVICE = 1 };

/* Largest LP (m and n each) the library accepts. */
#define LPB_MAX_DIM 16384

void lpb_default_opts(lp_batch_opts *opts);

/*
 * Create a batch of `num_lps` LPs and upload / copy their data to the current
 * CUDA device.  (Section 4.1 and Algorithm 1: the host gathers the LPs and
 * copies them to device memory; here the library also plans the launches.)
 *
 *  m, n          [host, num_lps]  sizes of each LP, 1 <= m,n <= LPB_MAX_DIM.
 *  a_off         [host, num_lps]  element offset of LP k's A (row-major m x n)
 *                                 in `A`; NULL = packed back to back.
 *                                 Offsets may repeat (LPs sharing A).
 *  b_off, c_off  [host, num_lps]  same for b (m entries) and c (n entries).
 *  A, b, c       [ptr_kind]       data; must hold every offset + size.
 *  a_len, b_len, c_len            number of elements of A, b and c.
 *  ptr_kind      LPB_HOST or LPB_DEVICE (A, b, c only; the size and offset
 *                arrays are always host memory).
 *  opts          NULL = defaults.
 *  stream        cudaStream_t used for the copies (NULL = legacy default).
 *
 * Ownership: every argument is only read during the call; the library keeps
 * its own copies and retains no caller pointer.  The call returns after the
 * data has been copied and checked.  Non-finite entries give LPB_EINVAL.
 * On error *out is set to NULL and nothing is leaked.
 */
lpb_err lp_batch_create(lp_batch **out, int32_t num_lps,
                        const int32_t *m, const int32_t *n,
                        const int64_t *a_off, const double *A, int64_t a_len,
                        const int64_t *b_off, const double *b, int64_t b_len,
                        const int64_t *c_off, const double *c, int64_t c_len,
                        int32_t ptr_kind, const lp_batch_opts *opts, void *stream);

/*
 * Solve every LP of the batch on `stream` (cudaStream_t; NULL = legacy
 * default stream).  Asynchronous: returns after the kernels are enqueued.
 * Builds each tableau on the device from the uploaded A, b, c and runs
 * Steps 1-3 until every LP halts (Section 3.1).  Tableaux that fit in one
 * CTA's shared memory stay there for the whole solve; larger ones are kept
 * in a library-owned global workspace (allocated by lp_batch_create).  May be
 * called again (each call solves from scratch); calls on one handle must not
 * overlap on the GPU (they share the workspace).
 */
lpb_err lp_batch_solve(lp_batch *h, void *stream);

/*
 * Copy results of the last solve out (waits for that solve to finish).
 *  status [num_lps] int32 lp_status, iters [num_lps] int32 pivots of both
 *  phases, obj [num_lps] objective value of the final tableau,
 *  x [sum n] final basic solution, LP k at offset sum_{j<k} n_j,
 *  y [sum m] reduced costs of the slack variables (LP duals; for
 *  LP_INFEASIBLE the Farkas multipliers of the phase-I optimum), LP k at
 *  offset sum_{j<k} m_j.
 * Any output pointer may be NULL (not copied).  ptr_kind says whether the
 * outputs are host or device memory.  For LPs that are not LP_OPTIMAL, x, obj
 * and y describe the last basis reached.
 */
lpb_err lp_batch_results(lp_batch *h, int32_t *status, int32_t *iters, double *obj,
                         double *x, double *y, int32_t ptr_kind);

/* Largest `chunks` of lp_solve_host. */
#define LPB_MAX_HOST_CHUNKS 64

/*
 * One call from host buffers to host results, with the copy of the inputs
 * overlapped with the solve: the batch is split into `chunks` contiguous
 * ranges of LPs (0 = one per 256 MiB of A, b and c, at most 8), each created and solved
 * as its own batch on its own internal stream.  The ranges' input copies run
 * one after another, each range's solve starts when its copy and input check
 * end, and the host waits for nothing until every solve is enqueued; then the
 * input checks and the results are read.  Section 4.3 of the paper splits a
 * batch over CUDA streams so that copies overlap kernels; this is the same
 * idea inside one call.
 *
 *  num_lps, m, n, a_off, A, a_len, b_off, b, b_len, c_off, c, c_len, opts:
 *                 as for lp_batch_create, all in HOST memory.  Each range
 *                 copies the smallest spans of A, b and c that hold its LPs
 *                 (shared data is copied once per range).  The overlap needs
 *                 page-locked (pinned) A, b, c; with pageable memory the call
 *                 still works, with less overlap.
 *  status, iters, obj [num_lps], x [sum of n], y [sum of m] or NULL: HOST
 *                 buffers, filled as by lp_batch_results.
 * Each LP's results are the same, bit for bit, as those of lp_batch_create +
 * lp_batch_solve + lp_batch_results on the whole batch with the same opts (an
 * LP's arithmetic does not depend on the batch it is solved in).  Synchronous:
 * returns when the results are in the host buffers.  Errors: LPB_EINVAL for
 * bad arguments (nothing launched); LPB_EINVAL for a non-finite entry of A, b
 * or c, found after the solves (the device copy of such an entry is zeroed
 * before any solve reads it) and then no result buffer is written; every
 * error of lp_batch_create / lp_batch_solve / lp_batch_results.  All device
 * memory is released on return.
 */
lpb_err lp_solve_host(int32_t num_lps, const int32_t *m, const int32_t *n,
                      const int64_t *a_off, const double *A, int64_t a_len,
                      const int64_t *b_off, const double *b, int64_t b_len,
                      const int64_t *c_off, const double *c, int64_t c_len,
                      const lp_batch_opts *opts, int32_t chunks,
                      int32_t *status, int32_t *iters, double *obj, double *x, double *y);

/* Launch plan of a batch (filled by lp_batch_plan_info). */
typedef struct {
    int32_t num_groups;        /* kernel launches per solve                         */
    int32_t num_resident;      /* LPs whose tableau stays in one CTA's shared memory */
    int32_t num_streamed;      /* LPs whose tableau lives in a global workspace (FP64 or FP32) */
    int32_t num_phase1;        /* LPs with some b_i < 0                              */
    int32_t num_mixed;         /* LPs on the FP32 tableau + FP64 certificate path    */
    int32_t num_fallback;      /* of those, re-solved in FP64 by the last solve      */
    int32_t internal_errors;   /* internal-consistency failures seen by the kernels in
                                  the last solve (0 in a correct run; the LP concerned
                                  gets LP_NUMERICAL or is re-solved)                  */
    int32_t internal_error_code; /* code of the first such failure (0 if none)       */
    int32_t internal_error_lp;   /* its LP index (-1 if none)                        */
    int32_t internal_error_detail[5]; /* kernel state at that failure (diagnostics)   */
    int32_t num_warm_certified;/* last lp_batch_solve_warm: LPs certified from the
                                  network's proposal (the rest: num_fallback)     */
    int32_t num_warm_rounds;   /* last lp_batch_solve_warm: restricted LPs solved    */
    int32_t num_cluster;       /* LPs solved on a thread-block cluster (tableau split
                                  over the CTAs' shared memory)                   */
    int32_t num_warm_retried;  /* last lp_batch_solve_warm: LPs whose restricted LP
                                  outgrew the first pass's 16 rows and went to the
                                  second pass (up to 32 rows)                     */
    int64_t max_smem_bytes;    /* largest shared-memory footprint of a launch        */
    int64_t workspace_bytes;   /* global workspace of the streamed LPs (and of the
                                  streamed FP64 re-solve of large mixed LPs)      */
} lp_batch_plan;

/* Report the launch plan made by lp_batch_create (and, for num_fallback, the
 * outcome of the last solve: this waits for that solve). */
lpb_err lp_batch_plan_info(lp_batch *h, lp_batch_plan *plan);

/* The same solve as lp_batch_solve, captured once into a CUDA graph (on an
 * internal stream, the first time it is called) and replayed on `stream`
 * afterwards: one graph launch instead of the memsets, event records and
 * kernel launches of every solve.  Stage timing does not apply to it.
 * lp_batch_autotune drops the captured graph (the launch forms change). */
lpb_err lp_batch_solve_graph(lp_batch *h, void *stream);

/* Launch-form tuner.  For every launch group of the plan (LPs of one kernel,
 * thread count and shared-memory size), time the group alone on `stream` with
 * every candidate thread count (FP64: 32, 64, 128, 256, 512; mixed precision:
 * 32, 64, 128, 256) in both forms -- one CTA per LP, or persistent CTAs over an atomic
 * work queue with the LPs in descending order of work (groups that need the
 * whole 227 KB of a CTA's shared memory: one CTA per LP only) -- `rounds` times each,
 * and keep the fastest.  No counterpart in the paper.  Results of a solve do
 * not depend on these choices.  The trial launches overwrite the outputs, so
 * call lp_batch_solve again before lp_batch_results.  Waits for the GPU. */
lpb_err lp_batch_autotune(lp_batch *h, int32_t rounds, void *stream);

/* One launch group of the plan: index 0 .. lp_batch_plan.num_groups-1 (the
 * FP64 re-solve launches of the mixed path are not listed). */
typedef struct {
    int32_t kind;        /* 0 mixed precision, 1 FP64 shared-memory resident, 2 FP64 streamed,
                            3 FP64 on a thread-block cluster, 4 mixed precision
                            with the FP32 tableau in a global workspace, 5 single
                            launch (LPB_SCHED_SINGLE, FP64 or mixed) */
    int32_t count;       /* LPs in the group                                  */
    int32_t threads;     /* threads per CTA                                   */
    int32_t persistent;  /* 1: persistent CTAs over a work queue              */
    int64_t smem_bytes;  /* dynamic shared memory per CTA of the current form */
    float tuned_ms;      /* group time of the chosen form (-1: not tuned)     */
    int32_t cluster_ctas;/* kind 3: CTAs per cluster (else 0)                 */
} lp_batch_group;
lpb_err lp_batch_group_info(lp_batch *h, int32_t index, lp_batch_group *out);
/* Set a group's form by hand (threads a multiple of 32, at most 512; for a
 * mixed-precision group 32 without persistent selects one warp per LP;
 * persistent 0 or 1, and 0 for groups that need more than 226 KB of shared
 * memory).  Streamed groups are fixed. */
lpb_err lp_batch_set_group_form(lp_batch *h, int32_t index, int32_t threads, int32_t persistent);

/* Device timing of the stages of lp_batch_solve, off by default.  enable != 0
 * creates CUDA events (timing-capable) that every later solve records on the
 * caller's stream; enable == 0 waits for the last solve and frees them.  No
 * counterpart in the paper (which times whole runs, Section 5). */
lpb_err lp_batch_set_timing(lp_batch *h, int32_t enable);

/* Mean device time, in ms, of the solves recorded since timing was enabled
 * or since the previous call (at most the last 64 of them):
 *   stage_ms[0]  every launch group of the solve, from the fork off the
 *                caller's stream to the join back onto it;
 *   stage_ms[1]  the FP64 re-solve of the LPs the mixed-precision kernel did
 *                not certify (about 0 without LP_PREC_FP32_REFINE).
 * Waits for the last recorded solve.  *num_solves = how many solves the means
 * cover (0: nothing recorded, stage_ms untouched).  LPB_EINVAL when timing is
 * not enabled. */
lpb_err lp_batch_stage_times(lp_batch *h, float *stage_ms, int32_t *num_solves);

/*
 * Solve a batch of LPs that all have the same size m x n without allocating
 * any memory.  There is no counterpart in the paper: it is for callers that
 * must not allocate while they run -- code that hands all device memory to its
 * own pool, loops that cannot afford cudaMalloc/cudaFree (both can stall the
 * whole device), or hosts where no allocator is reachable.  Such a caller
 * allocates the inputs and outputs once and then calls this as often as it
 * wants; every call gives the same results as lp_batch_create + lp_batch_solve
 * + lp_batch_results on the same data.
 *
 *  num_lps, m, n  batch size and the common LP size (host values).
 *  A, b, c        [device] packed: LP k's A (row-major m x n) at k*m*n, its b
 *                 at k*m, its c at k*n.  Finite values (not checked here).
 *  status, iters, obj [device, num_lps]; x [device, num_lps*n]; y [device,
 *                 num_lps*m] or NULL: the outputs of lp_batch_results, packed
 *                 the same way.
 *  opts           NULL = defaults (opts->schedule and block_threads are ignored;
 *                 opts->precision must be LP_PREC_FP64, else LPB_EINVAL: only
 *                 the FP64 streamed kernel runs here).
 *  stream         cudaStream_t (NULL = legacy default); the call is
 *                 asynchronous and returns once the work is enqueued.
 *
 * Scratch: a fixed 64 MiB array inside the library, present on every GPU that
 * loads the library until the process exits.  It holds ~52 bytes per LP plus
 * at least one tableau workspace of about 8*(m+2)*(n+m+4) bytes; a batch that
 * does not fit returns LPB_ETOOBIG before any GPU work (e.g. up to ~1.2
 * million 50 x 50 LPs per call).  Every call looks up the array's device
 * address in the current context (a lookup, no allocation), so a call after
 * cudaDeviceReset or under another context uses that context's copy; the
 * first call on a device may load the library's device code, so make it
 * before capturing any stream.  All calls share the array, so
 * calls that overlap on the GPU race and give wrong results: serialise them
 * (one stream, or wait for the previous call).  Errors are reported by the
 * return code only (LPB_EINVAL, LPB_ETOOBIG, LPB_ECUDA); lpb_last_error is not
 * updated, since recording a message would allocate.
 */
lpb_err lp_solve_uniform_noalloc(int32_t num_lps, int32_t m, int32_t n,
                                 const double *A, const double *b, const double *c,
                                 int32_t *status, int32_t *iters, double *obj, double *x, double *y,
                                 const lp_batch_opts *opts, void *stream);

/* Largest dimension lp_hyperbox_solve accepts. */
#define LPB_MAX_HYPERBOX_DIM (1 << 20)

/*
 * Hyperbox LPs (Section 4.4, Eq. 7): for each direction l_k, k < num_lps,
 *
 *     obj[k] = max  l_k . x   over the box  lo <= x <= hi
 *            = sum_i l_ki h_ki,   h_ki = lo_i where l_ki < 0, hi_i otherwise,
 *
 * and x[k] = h_k, a maximiser (the hi bound where l_ki is 0 or -0).
 *
 *  num_lps, dim   number of directions (>= 0) and their dimension
 *                 (1 <= dim <= LPB_MAX_HYPERBOX_DIM).
 *  lo, hi         the box: dim values each when box_per_lp == 0 (one box for
 *                 every direction), num_lps*dim values laid out like L when
 *                 box_per_lp != 0.  lo_i <= hi_i is the caller's to ensure.
 *  L              num_lps*dim directions, row-major (direction k at k*dim).
 *  obj            [num_lps] output; x [num_lps*dim] output or NULL.
 *  ptr_kind       LPB_DEVICE: every array is memory of the current device and
 *                 the call is asynchronous on `stream` (returns once the work
 *                 is enqueued); LPB_HOST: host arrays, copied through device
 *                 buffers; the call returns when the results are in obj / x.
 *  stream         cudaStream_t (NULL = legacy default).
 *
 * All values must be finite.  The sum is taken in FP64 with a fused
 * multiply-add per term, in ascending i for dim <= 64 and as 32 lane sums
 * combined by a fixed tree above: within dim * 2^-53 * sum_i |l_ki h_ki| of the
 * exact value.  Arrays that are 16-byte aligned are staged with bulk
 * asynchronous copies; others are read with plain loads (same results).
 * If the GPU fails to complete a staged copy within about one second (a
 * hardware or driver fault, not an input condition), the affected outputs are
 * NaN.  Errors: LPB_EINVAL (bad argument, a LPB_DEVICE pointer that is not
 * device memory), LPB_ETOOBIG, LPB_ENOMEM, LPB_ECUDA.  No counterpart of the
 * host/device choice in the paper (which solves these LPs inside its tool).
 */
lpb_err lp_hyperbox_solve(int32_t num_lps, int32_t dim, const double *lo, const double *hi, int32_t box_per_lp,
                          const double *L, double *obj, double *x, int32_t ptr_kind, void *stream);

/*
 * Warm-start network.  No counterpart in the paper (whose solver always
 * starts from the slack basis): a perceptron n_in -> n_h1 -> n_h2 -> n_out with
 * ReLU hidden layers that maps an LP's data to one logit per constraint ("is
 * this constraint active at the optimum"), trained on LPs this library has
 * solved (lp_batch_solve_warm uses it).
 *
 * Precision: every matrix product has BF16 operands (round to nearest even)
 * and FP32 accumulation on the tensor cores; biases, pre-activations, the loss
 * and all gradients are FP32; master weights and Adam moments FP32.  Inputs are
 * scaled as (x - mean) * inv_std before the first product.  The loss is the
 * mean over the batch and the outputs of the weighted binary cross entropy
 * (weight pos_weight on targets 1, 1 on targets 0).
 *
 * Parameters travel as one FP32 array: W1 (n_h1 x n_in, row-major), b1, W2
 * (n_h2 x n_h1), b2, W3 (n_out x n_h2), b3.  Device arrays must belong to the
 * device that was current at lp_mlp_create; a host pointer is refused
 * (LPB_EINVAL) before any launch.
 */
#define LPB_MAX_MLP_WIDTH 8192
#define LPB_MAX_MLP_BATCH (1 << 20)

typedef struct lp_mlp lp_mlp;   /* opaque; owned by the library */

/* Create a network with He-uniform weights (rounded to BF16 values; splitmix64
 * stream from `seed`), zero biases, identity input scaling; max_batch = the
 * largest batch of lp_mlp_train_step / lp_mlp_gradients (lp_mlp_forward takes
 * any batch, in chunks of max(max_batch, 131072) rows).  Allocates on the
 * current device, for the 300-512-512-200 network: about 2.7 KB per
 * inference-chunk row and 23 KB per max_batch row. */
lpb_err lp_mlp_create(lp_mlp **out, int32_t n_in, int32_t n_h1, int32_t n_h2, int32_t n_out, int32_t max_batch,
                      uint64_t seed);
lpb_err lp_mlp_num_params(const lp_mlp *net, int64_t *count);
/* Host copies of the parameters (layout above).  Setting them restarts Adam. */
lpb_err lp_mlp_set_params(lp_mlp *net, const float *params);
lpb_err lp_mlp_get_params(lp_mlp *net, float *params);
/* Input scaling (host arrays of n_in values). */
lpb_err lp_mlp_set_scaling(lp_mlp *net, const float *mean, const float *inv_std);
lpb_err lp_mlp_get_scaling(lp_mlp *net, float *mean, float *inv_std);
/* Set the input scaling from data: mean and 1/std (population) of each of the
 * n_in features over x [rows x n_in] (device, FP32), summed in FP64 in a
 * fixed order (the same result on every call); a constant feature gets
 * inv_std = 1.  Waits for the GPU. */
lpb_err lp_mlp_fit_scaling(lp_mlp *net, const float *x, int64_t rows, void *stream);
/* logits [batch x n_out] (device, FP32) of x [batch x n_in] (device, FP32,
 * unscaled); asynchronous on stream. */
lpb_err lp_mlp_forward(lp_mlp *net, const float *x, int64_t batch, float *logits, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * batch (x [batch x n_in], targets y [batch x n_out] in {0,1}, device FP32).
 * loss (host, may be NULL) receives the batch loss before the step; asking
 * for it waits for the step. */
lpb_err lp_mlp_train_step(lp_mlp *net, const float *x, const float *y, int32_t batch, float lr, float pos_weight,
                          double *loss, void *stream);
/* Forward + backward without an update: the gradient of the loss (host,
 * parameter layout) and the loss; waits for the GPU. */
lpb_err lp_mlp_gradients(lp_mlp *net, const float *x, const float *y, int32_t batch, float pos_weight,
                         float *grads, double *loss, void *stream);
/*
 * The backward pass at given forward values: like lp_mlp_gradients, but the
 * forward products are not run; the pre-activations a1 [batch x n_h1], a2
 * [batch x n_h2] and the logits z [batch x n_out] (device, FP32) are taken
 * from the caller, and h1 = relu(a1), h2 = relu(a2) are rounded to BF16 from
 * them exactly as the forward pass rounds its own.  x, y as for
 * lp_mlp_gradients.  Used to check the backward kernels layer by layer on the
 * same inputs as a reference implementation; waits for the GPU.
 */
lpb_err lp_mlp_gradients_at(lp_mlp *net, const float *x, const float *a1, const float *a2, const float *z,
                            const float *y, int32_t batch, float pos_weight, float *grads, double *loss,
                            void *stream);
lpb_err lp_mlp_destroy(lp_mlp *net);

/* Epilogues of the network's product kernel (lp_mlp_gemm_bf16). */
enum {
    LPB_EPI_STORE = 0,      /* C = acc                                                   */
    LPB_EPI_BIAS_RELU = 1,  /* v = acc + bias[col]; C = v (if C); h = hT^T = bf16(max(v, 0)) */
    LPB_EPI_BIAS = 2,       /* C = acc + bias[col]                                       */
    LPB_EPI_MASK_GRAD = 3   /* v = pre > 0 ? acc : 0 (pre at C's index); C = v; h = hT^T = bf16(v) */
};
/* Kernel forms of the product: AUTO picks as the network does; MMA64 and
 * MMA128 are warp-level mma.sync kernels (64 x 64 and 128 x 128 tiles, the
 * same results bit for bit); TC is the tcgen05 kernel (TMA-staged 128 x 128
 * tiles, FP32 accumulator in tensor memory; another accumulation order, so
 * equal to the others within the FP32 accumulation bound). */
enum { LPB_GEMM_AUTO = 0, LPB_GEMM_MMA64 = 1, LPB_GEMM_MMA128 = 2, LPB_GEMM_TC = 3 };

/*
 * The network's matrix product on caller buffers: acc[M x N] = A[M x K] .
 * B[N x K]^T with BF16 operands (bit patterns as uint16_t, row-major, K
 * contiguous; lda, ldb >= K and multiples of 8; A and B 16-byte aligned; K a
 * multiple of 32 -- pad with zeros), FP32 accumulation on the tensor cores,
 * then the epilogue above: C FP32 [M x ldc], h BF16 [M x ldh], hT BF16 [N x
 * ldt] (the transposed copy; may be NULL for LPB_EPI_BIAS_RELU).  Every
 * array is device memory of the current device; asynchronous on `stream`.
 * This is the building block of lp_mlp_forward / lp_mlp_train_step, exposed
 * so that each product can be checked on its own.  Errors: LPB_EINVAL (bad
 * sizes, alignment, missing array, host memory), LPB_ETOOBIG, LPB_ECUDA.
 */
lpb_err lp_mlp_gemm_bf16(int32_t epilogue, int32_t form, int32_t M, int32_t N, int32_t K, const uint16_t *A,
                         int32_t lda, const uint16_t *B, int32_t ldb, float *C, int32_t ldc, const float *bias,
                         const float *pre, uint16_t *h, int32_t ldh, uint16_t *hT, int32_t ldt, void *stream);

/* Tiles of the tcgen05 product kernel that gave up on a wait (for a copy or
 * the tensor cores) since the library was loaded: 0 in a correct run.  Such a
 * tile's outputs are NaN.  Its waits are bounded at about two seconds. */
lpb_err lp_mlp_tc_faults(int32_t *count);

/*
 * Solve the batch from the warm-start network's proposal.  For every LP the
 * network scores the constraints from (b, c); the LP restricted to the rows
 * scored above `threshold` (a probability in (0, 1); at most 32 rows) is
 * solved by the simplex method and its optimum checked on the full LP in FP64
 * from the original data (every row feasible to 1e-9*max(1,|b|_inf), duals >=
 * 0 and every reduced cost >= 0 to 1e-9*max(1,|c|_inf), c^T x = b_R^T y to
 * 1e-9 relative).  Violated rows are added and the restricted LP solved again
 * (up to 8 rounds).  A certified LP is reported LP_OPTIMAL with that x, the
 * duals y (0 off the restricted rows), obj = c^T x and iters = the restricted
 * pivots; every other LP is solved cold by the FP64 path (same results as
 * lp_batch_solve with LP_PREC_FP64).  The restricted LP holds at most 16 rows
 * in a first pass (a smaller tableau: more LPs per SM); an LP whose rows
 * outgrow that is tried again in a second pass with up to 32 rows before it
 * goes to the cold solve.  Requirements: all LPs of one size m x n,
 * a network with m + n inputs (b then c) and m outputs on the batch's device,
 * and every LP's FP64 tableau within one CTA's shared memory (LPB_ETOOBIG
 * otherwise).  Asynchronous like lp_batch_solve; lp_batch_plan_info reports
 * num_warm_certified, num_warm_rounds, num_warm_retried and num_fallback. */
lpb_err lp_batch_solve_warm(lp_batch *h, lp_mlp *net, float threshold, void *stream);

/* Training data from a batch of equal-size LPs (device arrays):
 * features x [num_lps x (m+n)] = (b, c) as FP32 (the network's input), and,
 * after a solve, labels [num_lps x m] = 1.0 where the LP is optimal and its
 * dual y_i > 0 (constraint i active), else 0.0.  Asynchronous on stream. */
lpb_err lp_batch_features(lp_batch *h, float *x, void *stream);
lpb_err lp_batch_active_labels(lp_batch *h, float *labels, void *stream);

/* Throughputs of the units the solver's kernels are bound by, measured on the
 * current device by microbenchmarks (CUDA events, best of 5 launches over
 * every SM): FP64 and FP32 fused multiply-add (2 flops each), and shared
 * memory (16-byte loads plus stores, bytes moved both ways).  They are the
 * denominators of the roofline fractions the benchmark reports.  Waits for
 * the GPU; allocates a small temporary buffer.  No counterpart in the paper. */
typedef struct {
    double fp64_gflops;
    double fp32_gflops;
    double smem_gbs;
    int32_t num_sms;
} lpb_peaks;
lpb_err lpb_measure_peaks(lpb_peaks *out, void *stream);

/* Free the batch (waits for its pending work).  NULL is accepted. */
lpb_err lp_batch_destroy(lp_batch *h);

/* Static text of an error code. */
const char *lpb_strerror(lpb_err err);

/* Detail of the last failing call on this thread ("" if none). */
const char *lpb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LPBATCH_H */
