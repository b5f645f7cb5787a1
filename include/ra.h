/*
 * ra.h -- C ABI of the GB300 price-discovery library (libra.so).
 *
 * The library solves the fungible resource-allocation problem of
 * "Allocation of Fungible Resources via a Fast, Scalable Price Discovery
 * Method" (arXiv 2104.00282), Section 2.4, problem (e-res-alloc):
 *
 *     maximize    sum_i u_i(a_i^T x_i)
 *     subject to  x_i >= 0,  1^T x_i <= 1   (per-job cap; optional),
 *                 sum_i x_i <= R,
 *
 * by minimising the dual function over resource prices lambda >= 0
 * (Section 3, problem (e-dual); the paper writes the prices as p).
 *
 * Conventions for every entry point:
 *  - All array arguments are DEVICE pointers unless the comment says
 *    "host".  They are borrowed: the caller keeps them alive and unchanged
 *    until the work has completed on the problem's stream.
 *  - Work is enqueued on the CUDA stream given to ra_problem_create and is
 *    asynchronous unless the comment says the call synchronises.
 *  - Matrices are row-major; the efficiency matrix A is n x m FP32 with row i
 *    equal to a_i^T.  A, kind, w and param must be 16-byte aligned.
 *  - No exception crosses the ABI.  A non-RA_OK status leaves outputs
 *    unspecified; ra_last_error() returns a thread-local message.
 *  - Utility kinds (per job, uint8):
 *      RA_U_LOG     u(t) = w log t                 (Eq. e-log-util, weighted)
 *      RA_U_POWER   u(t) = w t^p, 0 < p < 1, or    (Section 2.2, power utility;
 *                   u(t) = -w t^p, -64 <= p < 0     alpha-fair with alpha = 1 - p)
 *      RA_U_LINCAP  u(t) = w min(t, T)             (target-priority + w T)
 *      RA_U_TARGET  u(t) = w min(t - T, 0)         (Eq. e-target-priority-util)
 *    param[i] holds p (power) or T (lincap, target) and is ignored for log.
 */
#ifndef RA_H
#define RA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RA_OK = 0,
    RA_EINVAL = 1,      /* invalid argument or problem data                  */
    RA_ENOMEM = 2,      /* device allocation failed                          */
    RA_ECUDA = 3,       /* a CUDA runtime call failed                        */
    RA_ENOTCONV = 4,    /* solve stopped at max_evals above the tolerance    */
    RA_ETIMEOUT = 5,    /* a bounded device wait expired (kernel gave up)    */
    RA_EUNBOUNDED = 6   /* a zero price with no per-job cap: demand unbounded */
} ra_status;

enum { RA_U_LOG = 0, RA_U_POWER = 1, RA_U_LINCAP = 2, RA_U_TARGET = 3 };

/* Flags for ra_problem_create. */
#define RA_JOB_CAP      0x0u /* default: keep the per-job cap 1^T x_i <= 1 (Eq. e-res-alloc) */
#define RA_NO_JOB_CAP   0x1u /* drop the per-job cap: c_i(t) = t min_j lambda_j / A_ij        */
#define RA_FP64_JOBMATH 0x2u /* per-job arithmetic in FP64 instead of FP32                     */
#define RA_VALIDATE     0x4u /* check the data at create time (copies it to the host; syncs)  */

typedef struct ra_problem ra_problem; /* opaque; owns its device workspace */

/* Maximum number of resources m handled by the kernels. */
#define RA_MAX_M 32

/*
 * ra_problem_create -- bind problem data (Section 2.4) and allocate the
 * workspace (per-block partial sums, two n-length compact allocation
 * buffers of 10 bytes per job, solver state; about 20 n bytes).
 *   n      number of jobs, n >= 1
 *   m      number of resources, 1 <= m <= RA_MAX_M
 *   A      n*m FP32 efficiencies, A_ij >= 0                       (borrowed)
 *   kind   n uint8 utility kinds                                   (borrowed)
 *   w      n FP32 weights, w > 0                                   (borrowed)
 *   param  n FP32 utility parameters (p in (0,1) or [-64,0), or T > 0) (borrowed)
 *   R      m FP64 resource limits, R_j >= 0                        (borrowed)
 *   flags  RA_JOB_CAP or RA_NO_JOB_CAP, | RA_FP64_JOBMATH, | RA_VALIDATE
 *   stream cudaStream_t used by every call on this problem (NULL = legacy)
 *   out    host: receives the problem handle
 * Errors: RA_EINVAL on bad sizes, misaligned pointers or (with RA_VALIDATE)
 * invalid data; RA_ENOMEM / RA_ECUDA on allocation failure.
 */
ra_status ra_problem_create(int64_t n, int32_t m, const float *A, const uint8_t *kind,
                            const float *w, const float *param, const double *R, uint32_t flags,
                            void *stream, ra_problem **out);

/* Release the workspace (synchronises the problem's stream first). */
void ra_problem_destroy(ra_problem *prob);

/*
 * ra_eval_dual -- dual function and subgradient at prices lambda
 * (Section 3, "Evaluating the dual function" and eq. e-g-subgrad):
 *     g(lambda) = lambda^T R + sum_i max_{x_i} [u_i(a_i^T x_i) - lambda^T x_i],
 *     q         = R - sum_i x_i(lambda).
 * Each job's subproblem (Algorithm 1) is solved in closed form on the lower
 * convex hull of (0,0), (A_ij, lambda_j) (Section 4).
 *   lambda  m FP64 prices >= 0
 *   g       1 FP64 output (may be NULL)
 *   q       m FP64 output (may be NULL)
 *   U_lb    1 FP64 output or NULL: utility of the column-scaled feasible
 *           allocation (Section 5); costs a second, lighter pass over the
 *           jobs.  With the per-job cap the scaling is the paper's
 *           X diag(min(1, R/r)).  Without it the columns are scaled to use
 *           exactly R (up as well as down), except that jobs with a linear
 *           utility keep their allocation while they use less than R_j and
 *           the other jobs share what is left of it.
 * Deterministic: identical inputs give bitwise identical outputs on the
 * same GPU.  Per-thread sums are compensated FP32; the block and grid stages
 * add float-float pairs (about 44 significant bits) in a fixed order and the
 * totals are converted to FP64 (with RA_FP64_JOBMATH every stage is FP64).
 * If a bounded device wait gave up (RA_ETIMEOUT, see ra_set_wait_timeout),
 * g, q and U_lb are NaN.
 */
ra_status ra_eval_dual(ra_problem *prob, const double *lambda, double *g, double *q, double *U_lb);

/*
 * ra_eval_records -- the per-job allocation chosen inside the last
 * ra_eval_dual call made with U_lb != NULL (the compact record the lower
 * bound is formed from): for job i, resources j12[2i], j12[2i+1] (-1 = none,
 * lower efficiency first) and the throughput A_ij x_ij each delivers,
 * t12[2i], t12[2i+1] (FP32).  Both outputs are 2n device arrays.
 */
ra_status ra_eval_records(ra_problem *prob, int32_t *j12, float *t12);

/*
 * ra_init_prices -- initial prices of Section 5, Eq. e-initialization:
 *     x_i = R / (kappa n), kappa = max(1, 1^T R / n) (kappa = 1 without the cap),
 *     lambda^1 = (1/n) sum_i u_i'(a_i^T x_i) a_i.
 *   lambda1  m FP64 output.
 */
ra_status ra_init_prices(ra_problem *prob, double *lambda1);

typedef struct {
    double tol_rel;       /* target relative gap (g_best - U_best)/max(|U_best|,|g_best|,1);
                             with FP32 per-job arithmetic the loop stops at tol_rel / 2, leaving
                             room for the FP32 rounding of its own estimate of the gap           */
    int32_t max_evals;    /* cap on dual evaluations (line-search trials included)             */
    int32_t lbfgs_mem;    /* L-BFGS memory, 1..16 (Section 6.1 uses 10)                         */
    int32_t update;       /* price update (Section 5):
                             0 = projected L-BFGS, initial inverse Hessian chosen by the problem
                                 (default): diagonal without the per-job cap, scalar with it;
                             1 = projected subgradient;
                             2 = projected L-BFGS, scalar initial matrix s^T y / y^T y;
                             3 = projected L-BFGS, diagonal initial matrix diag(lambda_j / r_j)
                                 scaled by s^T y / y^T D y                                    */
    int32_t use_graph;    /* 1 = run the loop as one CUDA graph with a device-side while node   */
    double lam_floor;     /* lower bound on prices; <0 selects 0 (cap) / 1e-12 max(lambda^1)    */
    int32_t master_lb;    /* 1 = also bound U* by the master LP over evaluated allocations      */
    int32_t repair_window;/* > 0: when the gap has not halved in this many evaluations, leave the
                             device loop, re-mix the jobs at ties at the best prices (as
                             ra_recover_feasible) and resume; also tried once at max_evals.
                             0 = off.  -1 (default) = automatic: 4 when the problem has fewer
                             than 4096 jobs per resource (ties stall its column-scaled bound
                             early), else 16                                                    */
    double init_step;     /* length of the first price step (and of a restarted gradient step)
                             as a fraction of |lambda|; default 0.05, smaller from a close start */
    int32_t init_scale;   /* without the per-job cap and lambda0: 1 (default) scales the prices
                             of Eq. e-initialization by the minimiser of g along their ray (one
                             pass); 0 starts from Eq. e-initialization itself                  */
    int32_t pad_;
} ra_solve_opts;

typedef struct {
    int32_t status;       /* ra_status of the solve                                            */
    int32_t iters;        /* accepted price updates                                            */
    int32_t evals;        /* dual evaluations                                                  */
    int32_t ls_fail;      /* line searches that gave up (then a gradient step is used)          */
    double g;             /* best dual value (upper bound on U*)                                */
    double U_lb;          /* best feasible utility (lower bound on U*)                          */
    double rel_gap;       /* relative duality gap at exit                                      */
    double gap_per_job;   /* (g - U_lb) / n, the paper's absolute measure (Algorithm 2)         */
    int32_t repairs;      /* repairs of the lower bound run (see repair_window)                 */
    int32_t n_flex;       /* jobs the last repair re-mixed                                      */
    double eval_ms;       /* device time (global timer) in dual evaluations, from the end of one
                             price update to the start of the next (launch gaps included)      */
    double step_ms;       /* device time in the solver steps (master LP and price update);
                             neither counts the host-side repairs                               */
} ra_solve_info;

/* Fill *opts with the defaults (tol 1e-6, 500 evals, memory 10, L-BFGS, graph,
 * first step 0.05 |lambda|). */
void ra_solve_opts_default(ra_solve_opts *opts);

/*
 * ra_solve -- price discovery, Algorithm 2 of Section 5: from lambda0 (or
 * Eq. e-initialization when lambda0 is NULL) repeat {dual evaluation,
 * column-scaled lower bound, gap test, price update} on the device until the
 * relative duality gap is <= tol_rel or max_evals is reached.  The loop runs
 * without host round trips.  With the per-job cap the lower bound of an
 * evaluation is formed from a 10-byte-per-job record in a pass beside the
 * next price update, so it costs no second read of A.  Without the cap it is
 * formed from the evaluation's own sums as soon as the evaluation ends:
 * U(X) + sum_j lambda_j (r_j - r_lin_j) ln s_j (t u'(t) = lambda_j x_ij at
 * each job's optimum), less a Taylor remainder for powers p < 0 -- a lower
 * bound on the utility of the column-scaled allocation that ra_eval_dual's
 * U_lb describes; where a column would scale its linear-utility jobs down,
 * the records and that pass serve instead.
 *   opts        host, may be NULL for defaults
 *   lambda0     m FP64 start prices or NULL
 *   lambda_out  m FP64 output: prices with the best dual value
 *   lambda_lb   m FP64 output or NULL: prices whose (column-scaled) allocation
 *               gave the best lower bound U_lb
 *   info        host output (may be NULL)
 * Synchronises the problem's stream.  Returns RA_ENOTCONV when max_evals
 * was reached above the tolerance (lambda_out and info are still valid).
 */
ra_status ra_solve(ra_problem *prob, const ra_solve_opts *opts, const double *lambda0,
                   double *lambda_out, double *lambda_lb, ra_solve_info *info);

/*
 * ra_solve_certificate -- the allocation behind the lower bound U_lb of the
 * last ra_solve, as a convex combination of subproblem allocations: entry k
 * has weight theta[k] (summing to 1), prices lam[k*m .. k*m+m) and scaled[k]
 * = 1 when that allocation was column-scaled (Section 5) before mixing: to
 * X diag(min(1, R/r)) with the per-job cap, as ra_eval_dual's U_lb describes
 * without it.  The mixture meets sum_i x_i <= R, and since every u_i is
 * concave its utility is at least U_lb.  A single entry with scaled[0] = 2
 * means the bound came from a repair (see repair_window): the allocation is
 * the one ra_recover_feasible returns at lam[0] with default options.  theta, scaled: host arrays of
 * RA_MAX_CERT entries; lam: host array of RA_MAX_CERT * m doubles.  Returns
 * the number of entries written, or -1 on error.  Synchronises.
 */
#define RA_MAX_CERT 64
int32_t ra_solve_certificate(ra_problem *prob, double *theta, double *lam, int32_t *scaled);

/*
 * ra_solve_history -- per-evaluation log of the last ra_solve (the paper's
 * verbose output, Section 6.1): rows of RA_HIST_COLS doubles (evaluation, g,
 * best U_lb, relative gap, master-LP bound of that evaluation or -inf, its
 * simplex pivots).  hist: host buffer of RA_HIST_COLS*cap doubles.  Returns
 * the number of rows written (<= cap) or -1 on error.  Synchronises.
 */
#define RA_HIST_COLS 6
int32_t ra_solve_history(ra_problem *prob, double *hist, int32_t cap);

/*
 * ra_recover_primal -- allocation at prices lambda (Section 3, "Recovering an
 * optimal allocation from optimal prices"): each job's subproblem solution,
 * which uses at most two resources (Section 4.1).
 *   jstar     n int32 output or NULL: argmin_j lambda_j / A_ij (-1 if none)
 *   j12       2n int32 output or NULL: resources used, -1 = none, lower-A first
 *   x12       2n FP32 output or NULL: their time fractions
 *   t         n FP32 output or NULL: throughput a_i^T x_i
 *   X_dense   n*m FP32 output or NULL: dense allocation matrix
 *   U         1 FP64 output or NULL: sum_i u_i(t_i) of this (unscaled) allocation
 *   near_tie  n uint8 output or NULL: 1 where the two best effective prices
 *             lambda_j/A_ij are within 1e-6 relative
 *   n_near_ties host output or NULL: count of such jobs (synchronises)
 */
ra_status ra_recover_primal(ra_problem *prob, const double *lambda, int32_t *jstar, int32_t *j12,
                            float *x12, float *t, float *X_dense, double *U, uint8_t *near_tie,
                            int64_t *n_near_ties);

/*
 * ra_recover_feasible -- an allocation that meets the resource limits, at
 * prices lambda (Section 3, "Recovering an optimal allocation from optimal
 * prices").  Every job gets its subproblem's optimum (as ra_recover_primal);
 * the jobs whose optimum is within tie_rel of a tie -- two effective prices
 * lambda_j / A_ij, two hull segments, or (linear utilities) w and a segment
 * slope -- are re-mixed: each job's optimal extreme allocations are listed and
 * a small LP (FP64, on the host) picks convex weights that maximise the
 * weighted utility minus the overuse max(r_j - R_j, 0) priced at lambda_j
 * (about the utility that scaling it away would cost).  Overuse the LP leaves
 * is taken out by the column
 * scaling of Section 5 (without the per-job cap, under-used columns are also
 * scaled up).  The paper is silent on this step; at optimal prices the
 * re-mixed allocation closes the duality gap that column scaling alone
 * leaves when few jobs share a resource.
 *   lambda   m FP64 prices
 *   opts     host or NULL: tie_rel (default 1e-3), max_flex jobs re-mixed at
 *            most (default 512, <= 4096; the jobs closest to a tie are taken)
 *   jk, xk   4n int32 / 4n FP32 outputs or both NULL: per job up to four
 *            (resource, time fraction) pairs, resource -1 = unused slot;
 *            RA_EINVAL if a re-mixed job uses more than four (then use X)
 *   X_dense  n*m FP32 output or NULL
 *   info     host output (required): the utility U of the allocation, taken
 *            in FP64 before the outputs round it to FP32 (feasible to FP64
 *            rounding, so U is a lower bound on the optimum), the worst
 *            usage_j / R_j of the FP32 outputs, the jobs re-mixed and the LP's
 *            outcome
 * Synchronises.  Overwrites the records that ra_eval_records returns.
 * Allocates about 4n bytes of workspace on its first call.
 */
typedef struct {
    double tie_rel;        /* margin below which a job's optimum counts as tied (0, 1]      */
    int32_t max_flex;      /* jobs re-mixed at most, 1..4096                                 */
    int32_t pad_;
} ra_repair_opts;

typedef struct {
    int64_t n_flex;           /* jobs re-mixed by the LP                                      */
    int32_t n_alt;            /* optimal extreme allocations offered to the LP               */
    int32_t lp_status;        /* 0 optimal; 1 iteration limit; -1 no LP was needed           */
    double tie_cut;           /* the re-mixed jobs have tie margins below this              */
    double overuse;           /* sum_j max(r_j - R_j, 0) / R_j left by the LP (then scaled)  */
    double U;                 /* utility of the allocation in FP64 (lower bound on U*)       */
    double max_usage_over_R;  /* worst usage_j / R_j of the returned allocation            */
} ra_repair_info;

void ra_repair_opts_default(ra_repair_opts *opts);
ra_status ra_recover_feasible(ra_problem *prob, const double *lambda, const ra_repair_opts *opts,
                              int32_t *jk, float *xk, float *X_dense, ra_repair_info *info);

/*
 * ra_eval_dual_static -- g(lambda) and q = R - r exactly as ra_eval_dual
 * computes them (the same kernel, launch shape and reduction order, so the
 * same bits), but without creating a problem and without allocating any
 * device memory.  (The paper has no counterpart; this is a deployment aid.)
 *
 * For callers that must not allocate: latency-bound serving loops with a
 * no-allocation rule (cudaMalloc can synchronise the device and its latency
 * is unbounded), and hosts whose framework owns all device memory through
 * its own pool allocator and forbids allocations behind its back.
 *
 * Arguments are those of ra_problem_create plus lambda (m FP64 device prices)
 * and the outputs g (1 FP64, device) and q (m FP64, device); flags may only
 * be RA_JOB_CAP or RA_NO_JOB_CAP (FP32 per-job arithmetic).  All pointers are
 * device pointers; A, kind, w, param must be 16-byte aligned.  Work is
 * enqueued on `stream`.
 *
 * Scratch: one static device array of about 546 KB in this library, which
 * every GPU that loads libra.so keeps until the process exits.  It holds the
 * per-CTA partial sums of at most 1024 CTAs; a GPU whose evaluation would use
 * more CTAs is refused with RA_EINVAL.  Any n and 1 <= m <= RA_MAX_M are
 * accepted.  The first call on a device (per m and cap mode) does the
 * set-up with that device current: it looks up the array's device address
 * (cudaGetSymbolAddress) and sets the kernels' launch attributes; make that
 * first call before any stream capture.  All calls share the array and it
 * keeps the previous call's contents (the kernel's ticket and status word
 * are cleared on the stream before each launch): calls whose work overlaps
 * on the GPU -- on different streams or devices sharing a context -- race
 * and must be serialised by the caller.
 *
 * The call returns before the work is done, so it cannot return
 * RA_ETIMEOUT: when a bounded device wait gives up (ra_set_wait_timeout),
 * g and q receive NaN instead.
 */
ra_status ra_eval_dual_static(int64_t n, int32_t m, const float *A, const uint8_t *kind,
                              const float *w, const float *param, const double *R,
                              const double *lambda, uint32_t flags, void *stream, double *g,
                              double *q);

/*
 * One problem split by job range across devices or processes (shards).  Given
 * the prices the jobs are independent (Section 3, "Evaluating the dual
 * function"), so each shard evaluates its own jobs and only m-sized sums
 * cross between shards; a shard is a problem created with ra_problem_create
 * over a contiguous range of the jobs (the pointers offset to the range's
 * first job -- a range starting at a multiple of 16 jobs keeps them 16-byte
 * aligned) and the whole problem's R.  (Not in the paper.)
 *
 * Exchanged per shard: RA_SHARD_WIDTH(m) FP64 values [sum_i h_i, sum_i
 * u_i(t_i), lagged lower bound, status word, r_0..r_{m-1}, r_lin_0..]; shards
 * are always added in shard (rank) order, so every shard computes the same
 * bits.
 */
#define RA_SHARD_WIDTH(m) (4 + 2 * (m))

/* ra_eval_partial -- this shard's sums at lambda: part (device,
 * RA_SHARD_WIDTH(m) FP64) as laid out above (the lagged bound is 0). */
ra_status ra_eval_partial(ra_problem *shard, const double *lambda, double *part);

/* ra_combine_partials -- g = lambda^T R + sum_s h_s and q = R - sum_s r_s from
 * S shards' parts (device, S x RA_SHARD_WIDTH(m), shard order); g (1) and q
 * (m) are device outputs (either may be NULL); enqueued on `stream`. */
ra_status ra_combine_partials(int32_t S, int32_t m, const double *parts, const double *lambda,
                              const double *R, double *g, double *q, void *stream);

/*
 * ra_solve_sharded -- ra_solve for one shard of a problem of n_total jobs
 * split across `world` shards; shard `rank` of them.  Every shard calls it
 * with the same options and start prices.  Once per evaluation (and once for
 * Eq. e-initialization) the library writes `count` FP64 values into send
 * (device, >= RA_SHARD_WIDTH(m)) and calls fn(ctx, count, stream): fn must
 * all-gather every shard's send into recv (device, world x count, shard
 * order), enqueued on `stream` (for example an NCCL all-gather), and return
 * 0.  The price update then runs on every shard on the same combined values,
 * so the prices agree bit for bit.  Host-driven loop (no CUDA graph, no
 * repair of the lower bound); synchronises every evaluation.
 */
typedef int32_t (*ra_allgather_fn)(void *ctx, int32_t count, void *stream);
ra_status ra_solve_sharded(ra_problem *shard, int64_t n_total, int32_t rank, int32_t world,
                           double *send, double *recv, ra_allgather_fn fn, void *ctx,
                           const ra_solve_opts *opts, const double *lambda0, double *lambda_out,
                           ra_solve_info *info);

/*
 * Batched price discovery (a throughput mode; the paper solves one problem at
 * a time, Algorithm 2 of Section 5): P independent problems of the form
 * (e-res-alloc), each with its own n_p, m_p, data and capacities, solved
 * together on one GPU.  Each loop trip evaluates the dual of every problem
 * still iterating in one streaming pass per width class (m <= 4, 8, 16, 32),
 * then runs each problem's master LP and price update (one CTA per problem);
 * a problem whose relative gap has met tol_rel, or that has reached
 * max_evals, drops out of all three.  Per problem the arithmetic is that of
 * ra_solve.
 */
typedef struct ra_batch ra_batch; /* opaque; owns its device workspace */

/*
 * ra_batch_create -- describe P problems.  n, m: host arrays of P sizes
 * (1 <= n_p <= 2^31, 1 <= m_p <= RA_MAX_M).  A, kind, w, param, R: host arrays
 * of P DEVICE pointers laid out as in ra_problem_create (A row-major n_p x
 * m_p, A/kind/w/param 16-byte aligned); the data is not copied and must stay
 * valid until ra_batch_destroy.  flags: RA_JOB_CAP or RA_NO_JOB_CAP.
 * Allocates about 20 bytes per job (two generations of the 10-byte
 * lower-bound record) plus about 100 KB of solver state per problem.
 * Returns RA_EINVAL on bad sizes, NULL pointers or misalignment (naming the
 * problem), RA_ENOMEM when the workspace does not fit.
 */
ra_status ra_batch_create(int32_t P, const int64_t *n, const int32_t *m, const float *const *A,
                          const uint8_t *const *kind, const float *const *w,
                          const float *const *param, const double *const *R, uint32_t flags,
                          void *stream, ra_batch **out);

/*
 * ra_batch_create_shaped -- ra_batch_create with the launch shape of the
 * batched evaluation given (chosen by the package's autotuner): a problem of
 * at most whole_tiles 256-job tiles is one chunk (one CTA visits all of it
 * in an evaluation, so small problems never wait for other CTAs), a larger
 * one is cut into chunks of chunk_tiles tiles; the persistent grid of each
 * width class runs ctas_per_sm CTAs per SM (0: as many as fit).  shape NULL
 * gives the defaults {16, 0, 0}.
 */
typedef struct {
    int32_t chunk_tiles;  /* 1..4096, default 16 */
    int32_t whole_tiles;  /* >= 0, default 0 */
    int32_t ctas_per_sm;  /* 0..8, default 0 */
    int32_t pad_;
} ra_batch_shape;
ra_status ra_batch_create_shaped(int32_t P, const int64_t *n, const int32_t *m, const float *const *A,
                                 const uint8_t *const *kind, const float *const *w,
                                 const float *const *param, const double *const *R, uint32_t flags,
                                 const ra_batch_shape *shape, void *stream, ra_batch **out);

/* Waits for the batch's stream, then frees its workspace. */
void ra_batch_destroy(ra_batch *b);

/* Length of the concatenated price vector, sum_p m_p (problem p's prices
 * follow those of problems 0 .. p-1), or -1 for NULL. */
int64_t ra_batch_prices(const ra_batch *b);

/*
 * ra_batch_solve -- solve every problem of the batch.
 *   opts        host, may be NULL (defaults of ra_solve; one set for all)
 *   lambda0     device, sum_p m_p FP64 start prices (concatenated), or NULL
 *               for Eq. e-initialization of each problem
 *   lambda_out  device, sum_p m_p FP64: each problem's prices with the best
 *               dual value
 *   infos       host, P records as ra_solve returns them
 *   seconds     host, P doubles or NULL: device time from the start of the
 *               call's GPU work until problem p stopped (its time to
 *               tolerance)
 * Synchronises.  RA_ENOTCONV / RA_EUNBOUNDED when at least one problem ended
 * that way (its infos entry says which); RA_ETIMEOUT when a device wait gave
 * up (all results are then unreliable).
 */
ra_status ra_batch_solve(ra_batch *b, const ra_solve_opts *opts, const double *lambda0,
                         double *lambda_out, ra_solve_info *infos, double *seconds);

/*
 * ra_batch_rebalance -- price coordination of M shards of one problem
 * (Section 7: shards solved independently with budgets R_k, resources then
 * moved from shards with lower prices to shards with higher prices; it
 * converges to the solution of the whole problem).  The batch's problems
 * are the shards (every one with the same m); their R arrays are the budgets
 * and are overwritten in place:
 *     R_kj <- Pi( R_kj + step (lambda_kj - pbar_j) / pbar_j * R_total_j / M ),
 * pbar_j the mean price of resource j over the shards and Pi the Euclidean
 * projection onto {R_kj >= f_j, sum_k R_kj = R_total_j} with the floor
 * f_j = 1e-3 R_total_j / M: a shard with none of a resource would price it
 * at infinity without the per-job cap (and its jobs that only use it would
 * get no throughput).
 *   lambda   device, the shards' prices concatenated (as ra_batch_solve returns)
 *   R_total  device, m FP64: the whole problem's limits
 * Enqueued on the batch's stream; allocates nothing.
 */
ra_status ra_batch_rebalance(ra_batch *b, const double *lambda, const double *R_total, double step);

/*
 * Learned warm start (not in the paper; the cold start it competes with is
 * the paper's Eq. e-initialization).  A problem is summarised per resource j
 * by RA_MLP_STATS = 13 statistics taken over a strided sample of at most
 * 16384 rows (rows floor(k n / S), S = min(n, 16384)): the order statistics
 * of A[:, j] at levels (2l+1)/16, l = 0..7, as logarithms; log(R_j / n); the
 * fractions of log, power and linear (lin-cap and target) utilities; the mean
 * of log w.  The network input of resource j (RA_MLP_IN = 26 floats) is its
 * 13 statistics followed by their mean over the problem's resources.  A
 * shared per-resource MLP 26 -> 256 -> 256 -> 1 with GELU maps each input row
 * to log(lambda_j).
 *
 * Parameters: one FP32 vector of RA_MLP_PARAMS entries laid out as W1 (26 x
 * 256, row-major, input-major), b1 (256), W2 (256 x 256), b2 (256), W3 (256),
 * b3 (1).  Training minimises the mean squared error against log(lambda*)
 * with Adam (Kingma and Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8).
 */
#define RA_MLP_STATS 13
#define RA_MLP_IN 26
#define RA_MLP_HIDDEN 256
#define RA_MLP_PARAMS 72961
/* The network is trained on log(lambda* + RA_MLP_PRICE_OFFSET), so that zero
 * prices (resources left with slack) have a finite target; its prices are
 * lambda_j = max(exp(y_j) - RA_MLP_PRICE_OFFSET, 0). */
#define RA_MLP_PRICE_OFFSET 1e-3

typedef struct ra_mlp ra_mlp; /* opaque; owns parameters, Adam moments, activations */

/* theta: host, RA_MLP_PARAMS floats, or NULL for zeros.  Kernels of the
 * network run on `stream`, except inside ra_warmstart_prices (the problem's
 * stream); the object is not safe for concurrent use. */
ra_status ra_mlp_create(const float *theta, void *stream, ra_mlp **out);
void ra_mlp_destroy(ra_mlp *net);
/* Host copies of the parameters / the gradient of the last training step
 * (RA_MLP_PARAMS floats each; synchronise).  set_params also clears Adam's
 * moments and step count. */
ra_status ra_mlp_get_params(ra_mlp *net, float *theta);
ra_status ra_mlp_set_params(ra_mlp *net, const float *theta);
ra_status ra_mlp_get_grads(ra_mlp *net, float *grad);
/* log_lambda[r] = MLP(feats[r, 0..26)) for rows r < rows (device arrays). */
ra_status ra_mlp_forward(ra_mlp *net, const float *feats, int32_t rows, float *log_lambda);
/* One Adam step on L = (1/rows) sum_r (MLP(feats_r) - target_r)^2 at
 * learning rate lr; loss (device, 1 float) receives L before the step, or
 * NULL. */
ra_status ra_mlp_train_step(ra_mlp *net, const float *feats, const float *target, int32_t rows,
                            float lr, float *loss);

/* Network input of every resource of a problem: feats (device) m x 26. */
ra_status ra_warmstart_features(ra_problem *prob, float *feats);
/* The same for every problem of a batch: (sum_p m_p) x 26, problem order. */
ra_status ra_batch_features(ra_batch *b, float *feats);

/*
 * ra_warmstart_prices -- start prices for ra_solve: lambda_w = max(exp(MLP(x_j))
 * - RA_MLP_PRICE_OFFSET, 0) and the cold start lambda_c of Eq.
 * e-initialization are both evaluated,
 * and lambda0 (device, m FP64) receives lambda_w when g(lambda_w) is finite
 * and g(lambda_w) <= g(lambda_c), else lambda_c.  used_warm (host, or NULL
 * to stay asynchronous) receives 1 when the network's prices were kept.
 * The statistics and the network run on a stream of the problem's own
 * (created on the first call) joined back to the problem's stream, beside
 * the cold start's pass; both g values come from one pass over the data.
 * That pass is also a complete evaluation at lambda_w: when ra_solve is the
 * next call on this problem and is given this lambda0 buffer (unchanged), a
 * solve that starts from the network's prices uses it as its first
 * evaluation instead of repeating it (any other call on the problem in
 * between drops it).
 */
ra_status ra_warmstart_prices(ra_problem *prob, ra_mlp *net, double *lambda0, int32_t *used_warm);
/* The choice of the problem's last ra_warmstart_prices call: *used_warm (host)
 * receives 1 when the network's prices were kept, 0 when the cold start was,
 * after the problem's stream has finished that call (synchronises the
 * stream).  RA_EINVAL when the problem has made no such call. */
ra_status ra_warmstart_used(ra_problem *prob, int32_t *used_warm);

/*
 * ra_scale_by_demand -- per-job demands (Section 7.1, "Extensions and
 * variations"): a job may hold several units of a resource while it runs, so
 * the resource constraint becomes sum_i d_i o x_i <= R, with d_i a positive
 * scalar per job or a positive m-vector per job (o the elementwise product).
 * Without the per-job cap this is the plain problem in resource units
 * y_ij = d_ij x_ij with efficiencies a_ij / d_ij: a_i^T x_i = sum_j
 * (a_ij / d_ij) y_ij and sum_i y_i <= R.  This call writes
 *     A_out[i, j] = A[i, j] / d[i]          (per_resource = 0: d has n entries)
 *     A_out[i, j] = A[i, j] / d[i * m + j]  (per_resource = 1: d is n x m)
 * (IEEE FP32 division).  Create the problem on A_out with RA_NO_JOB_CAP; its
 * solution y gives x_ij = y_ij / d_ij and the same prices, dual value and
 * utility.  (With the per-job cap the cap would become sum_j y_ij / d_ij <= 1,
 * which this transformation does not express.)
 *   A, d, A_out  device arrays (A_out may equal A); 16-byte aligned
 * Enqueued on `stream`.  RA_EINVAL on bad sizes or NULL pointers; a demand
 * that is not positive gives an infinite or NaN efficiency, which
 * ra_problem_create with RA_VALIDATE rejects.
 */
ra_status ra_scale_by_demand(int64_t n, int32_t m, const float *A, const float *d,
                             int32_t per_resource, float *A_out, void *stream);

/*
 * ra_set_wait_timeout -- bound of every device-side wait of the library's
 * kernels (a CTA waiting for its bulk copies), in seconds of device time; 2
 * by default, process-wide, read when work is enqueued (or captured).  A
 * kernel whose wait expires records it and returns instead of hanging: the
 * solvers then report RA_ETIMEOUT and the evaluations' outputs are NaN.  0
 * makes every such wait give up at once (for testing a caller's handling of
 * RA_ETIMEOUT).  RA_EINVAL unless 0 <= seconds <= 60.  (Not in the paper.)
 */
ra_status ra_set_wait_timeout(double seconds);

/* Static strings; ra_last_error() is thread-local and valid until the next call. */
const char *ra_status_string(ra_status s);
const char *ra_last_error(void);

/* Library build information, e.g. "libra sm_103a". */
const char *ra_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RA_H */
