// Internal declarations shared by the libra translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ra.h"

struct ra_batch;
struct ra_mlp;

namespace ra {

constexpr int kTile = 256;          // jobs per tile == threads per CTA of the streaming kernels
constexpr int kMaxStages = 8;
constexpr int kMaxLbfgsMem = 16;
constexpr int kHist = 512;          // solver history length
constexpr int kHistCols = 6;        // eval, g, best U_lb, gap, master-LP value, LP pivots
constexpr int kPartW = 2 * RA_MAX_M + 4; // doubles per block partial: h, U(X), U_lb(prev), spare, r[m], r_lin[m]
constexpr int kCand = 64;           // master-LP candidates kept (two per evaluation)
constexpr size_t kWarmBytes = 8192; // per-problem warm-start scratch

// Status word bits written by kernels (never trap: a kernel that gives up
// records why and returns).
constexpr int kStatusTimeout = 1;

// Column scaling of Section 5 that makes the evaluated allocation feasible,
// for one column with usage r, of which r_lin by jobs with a linear utility.
// With the per-job cap both factors are min(1, R / r): the over-used column
// is scaled down.  Without the cap nothing bounds a job's x_i, so the column
// is scaled to use exactly R: while the linear-utility jobs (at t = T, where
// more throughput is worth nothing) use less than R they keep their
// allocation, s_lin = 1, and the other jobs get the capacity left,
// s = (R - r_lin) / (r - r_lin); a column that the linear jobs alone fill, or
// nearly alone use (others below 1e-3 r, where r - r_lin would lose its
// digits to rounding), is scaled uniformly, s = s_lin = R / r.  s stays
// below 1e30 so that FP32 products cannot overflow.
__host__ __device__ inline void column_scales(double R, double r, double r_lin, int cap, double &s,
                                              double &s_lin)
{
    if (cap) {
        s = r > R ? R / r : 1.0;
        s_lin = s;
        return;
    }
    const double r_oth = r - r_lin;
    if (r_lin < R && r_oth > 1e-3 * r) {
        s_lin = 1.0;
        s = fmin((R - r_lin) / r_oth, 1e30);
    } else {
        s = r > 0.0 ? fmin(R / r, 1e30) : 1.0;
        s_lin = s;
    }
}

// Result slots of one dual evaluation (device, FP64).
struct EvalOut {
    double g;        // lambda^T R + sum h_i
    double Ux;       // sum_i u_i(t_i) of the unscaled allocation
    double Ulb_prev; // utility of the column-scaled allocation of the previous evaluation
    double sumh;     // sum_i h_i
    double s2neg;    // sum of p_i^2 |u_i(t_i)| over power jobs with p_i < 0, the
                     // remainder term of the solver's own bound; NaN when not reduced
    double q[RA_MAX_M];
    double r[RA_MAX_M];
    double r_lin[RA_MAX_M];  // part of r used by linear-utility jobs (kinds 2, 3; no-cap mode)
    int32_t rec_buf;         // solver mode: record buffer this evaluation wrote (-1 = none)
    int32_t pad_;
};

// Projected L-BFGS state of one solve, entirely in device memory.
struct SolverState {
    int32_t phase;       // 0: first evaluation pending; 1: line-search trial pending
    int32_t done;
    int32_t status;
    int32_t k;           // accepted iterations
    int32_t evals;
    int32_t ls_iter;
    int32_t ls_fail;
    int32_t mem_count;
    int32_t mem_head;
    int32_t have_lb_prev; // the evaluation just finished carried a lagged lower bound
    int32_t m;
    int32_t mem;
    int32_t max_evals;
    int32_t update;       // 0 L-BFGS, 1 subgradient
    int32_t hist_len;
    int32_t cap;          // per-job cap 1^T x_i <= 1 (selects the column scaling)
    double tol;
    double lam_floor;
    double g_cur;
    double step;
    double g_best;
    double U_best;
    double gap;
    double sg_a0;         // subgradient step scale
    // device time (globaltimer) of the loop: evaluations (from the end of one
    // solver step to the start of the next, launch gaps included) and steps;
    // here so that one copy of the state's first 144 bytes reads the results
    double eval_ns, step_ns;
    double init_step;     // first step length / |lambda|
    double g_bt;          // best trial value of the current line search
    double last_step;     // norm of the last accepted price step
    int32_t sg_pending;   // the evaluation in flight is a fallback subgradient step
    int32_t pad2_;
    double lam_bt[RA_MAX_M];
    double q_bt[RA_MAX_M];
    // master-LP lower bound: candidates (utility, usage) of evaluated
    // allocations, unscaled and column-scaled, with the prices that made them
    int32_t cand_count;
    int32_t cand_head;
    int32_t use_master;
    int32_t master_ok;      // the best lower bound came from the master LP
    double U_master;        // value of the last master LP (-inf if none)
    int32_t lp_iters;       // pivots of the last master LP
    int32_t lb_stall;       // evaluations since the scaled bound last closed 10 % of the gap
    int32_t mu_ok;          // mu_lp holds the LP's resource duals
    int32_t pad3_;
    double mu_lp[RA_MAX_M]; // minimiser of the cutting-plane model of g (LP duals)
    double q_best[RA_MAX_M];// subgradient at the best dual point
    unsigned long long t_start; // device global timer (ns) at setup
    unsigned long long t_done;  // device global timer (ns) when the solve stopped
    double r_prev[RA_MAX_M];
    double cand_U[kCand];
    int32_t cand_scaled[kCand];
    double cand_r[kCand][RA_MAX_M];
    double cand_lam[kCand][RA_MAX_M];
    double lp_theta[kCand]; // weights found by the last master LP (over cand slots)
    double theta[kCand];    // certificate of the best lower bound
    double theta_lam[kCand][RA_MAX_M];
    int32_t theta_scaled[kCand];
    int32_t theta_n;
    double lam_cur[RA_MAX_M];
    double q_cur[RA_MAX_M];
    double d[RA_MAX_M];
    double lam_trial[RA_MAX_M];   // prices of the evaluation in flight
    double lam_prev_eval[RA_MAX_M];
    double lam_best[RA_MAX_M];
    double lam_lb[RA_MAX_M];      // prices whose scaled allocation gave U_best
    double s_lag[RA_MAX_M];       // column scaling of the previous evaluation (lower bound)
    double s_lin_lag[RA_MAX_M];   // the same for its linear-utility jobs
    double r_lin_prev[RA_MAX_M];  // r_lin of the previous evaluation
    double R[RA_MAX_M];
    // L-BFGS pairs in FP32: they only shape the search direction (prices,
    // dual values and the gap stay FP64)
    float S[kMaxLbfgsMem][RA_MAX_M];
    float Y[kMaxLbfgsMem][RA_MAX_M];
    float rho[kMaxLbfgsMem];
    // bound of each evaluation's own column-scaled allocation (single solves
    // without the per-job cap), formed from the evaluation's sums as soon as
    // it ends instead of from its records in a later pass
    int32_t own_lb;         // 1 = form it (no records), 2 = form it and keep the lagged bound
    int32_t own_ok;         // the evaluation just finished reduced what it needs
    double own_U;           // the bound (-inf where that scaling admits none)
    double own_s[RA_MAX_M]; // its column scaling (non-linear and linear jobs)
    double own_sl[RA_MAX_M];
    // stall exit for the tie-aware repair (single-problem solves): the loop
    // leaves the device when the gap has not halved within stall_window
    // evaluations, so that the host can re-mix the jobs at ties
    int32_t stall_window;   // 0 = never leave for a repair
    int32_t mark_evals;     // evaluation at which gap_mark was set
    double gap_mark;
    unsigned long long t_last;   // end of the last solver step (global timer, ns)
    // verbose history, one row per evaluation; kept last: a single solve's
    // step stages everything before it in shared memory and writes back only
    // the rows it appended
    double hist[kHist][kHistCols];
};

// Internal solver status: the loop stopped for a repair of the lower bound.
constexpr int kStatusStalled = 100;

}  // namespace ra

struct ra_problem {
    int64_t n;
    int32_t m;
    uint32_t flags;
    const float *A;
    const uint8_t *kind;
    const float *w;
    const float *param;
    const double *R;
    cudaStream_t stream;
    int device;
    int num_sms;
    int mt;              // compile-time width used for this m (4, 8, 16, 32)
    int stages;
    int grid_dual;       // CTAs of the streaming dual kernel
    int grid_aux;        // CTAs of the lighter passes
    int grid_init;       // CTAs of the initial-price and ray-scaling passes (their own
    int grid_ray;        // occupancy: a grid above it would run in a second wave)
    size_t smem_dual;
    // workspace (library-owned)
    double *partials;    // max(grid) * kPartW
    unsigned *ticket;    // one counter per kernel family
    int *status;
    float2 *lbt[2];      // per job (t_P, t_Q): throughput from each used resource
    uchar2 *lbj[2];      // per job (P, Q), 255 = none
    ra::EvalOut *ev;     // evaluation result slots (2)
    double *s_buf;       // m: column scaling for the lower-bound pass
    ra::SolverState *st;
    int32_t *graph_flag;
    double *tmp;         // small scratch (m + 8 doubles)
    unsigned char *warm; // warm-start scratch (kWarmBytes)
    cudaStream_t side;   // warm start: statistics and network beside the cold-start pass
    cudaEvent_t fork, join;
    void *rep;           // allocation-repair workspace (ra_repair.cu), made on first use
    // the solve loop's CUDA graph, built on the first graph solve and kept
    // (it depends only on the problem's buffers and the wait limit)
    cudaGraph_t loop_graph;
    cudaGraphExec_t loop_exec;
    uint64_t loop_wait_ns;
    void *host_state;    // pinned host copy of the solver's result fields
    // the solve's lower-bound pass runs beside the price update on this
    // stream (created on the first solve); its results alternate between two
    // slots, so that the update reads the previous evaluation's bound while
    // the pass writes this evaluation's
    double *lb_slot;
    // the prices of the last ra_warmstart_prices call, whose pass was also
    // the first evaluation of a solve from them (NULL once anything else ran)
    const double *pre_lam0;
    cudaStream_t lb_side;
    cudaEvent_t lb_fork, lb_join;
};

namespace ra {

struct DualParams {
    const float *A;
    const uint8_t *kind;
    const float *w;
    const float *param;
    const double *R;
    int64_t n;
    int m;
    const double *lam;        // m prices
    // lagged lower bound (all NULL = off)
    const float2 *lbt_prev;
    const uchar2 *lbj_prev;
    const double *s_prev;
    const double *s_lin_prev; // scaling of the linear-utility jobs (NULL: s_prev)
    // compact record of this evaluation (NULL = not written)
    float2 *lbt_out;
    uchar2 *lbj_out;
    double *partials;
    unsigned *ticket;
    int *status;
    EvalOut *out;
    const int32_t *skip;      // when non-NULL and *skip != 0 the launch does nothing
    const int32_t *skip2;     // the same, a second flag (a solve's first evaluation made earlier)
    // solver mode: record buffers selected by a device-side parity word and
    // the lagged bound switched on by a device flag (NULL = fields above)
    float2 *lbt_buf[2];
    uchar2 *lbj_buf[2];
    const int32_t *pingpong;
    const int32_t *lag_on;
    const int32_t *rec_on;    // device flag (NULL = 1): 0 nothing extra; bit 0 write the
                              // records; nonzero: also reduce r_lin and, without the
                              // cap, the remainder sum s2neg of the own bound
    uint64_t wait_ns;         // bound of the mbarrier waits (set by the launchers)
};

// One problem of a batch (device copy).
struct BatchProblem {
    const float *A;
    const uint8_t *kind;
    const float *w;
    const float *param;
    const double *R;
    long long n;
    int m;
    int cls;              // width class: MT = 4 << cls
    int chunk_begin;      // this problem's chunks in its class's chunk list
    int chunk_end;
    float2 *lbt[2];
    uchar2 *lbj[2];
};

constexpr int kChunkTiles = 16;  // tiles of one problem per chunk (batched evaluation)

struct BatchDualArgs {
    const BatchProblem *probs;
    SolverState *st;
    EvalOut *ev;
    const int32_t *pingpong;
    const int32_t *lag_on;
    const int32_t *chunk_prob;
    const int32_t *chunk_tile0;
    const int32_t *chunk_ntiles;
    int nchunks;
    double *partials;     // nchunks x kPartW
    unsigned *ticket;     // per problem
    int *status;
    int stages;
    int cap;
    uint64_t wait_ns;     // bound of the mbarrier waits (set by the launcher)
};

// Launchers (ra_dual.cu).
cudaError_t launch_dual(const ra_problem *p, const DualParams &dp, cudaStream_t s);
cudaError_t launch_lower_bound(const ra_problem *p, const float2 *lbt, const uchar2 *lbj,
                               const EvalOut *src, double *U_lb, cudaStream_t s);
// tstride > 1: from every tstride-th full tile only (a strided sample)
cudaError_t launch_init(const ra_problem *p, double *lam1, cudaStream_t s, long long n_all = 0,
                        long long tstride = 1);
cudaError_t launch_ray_scale(const ra_problem *p, double *lam, cudaStream_t s, long long tstride = 1);
cudaError_t launch_dual_exact(const ra_problem *p, const double *lam, EvalOut *out, cudaStream_t s);
void release_loop_graph(ra_problem *p);
// g at two price vectors in one pass; with first_eval also the solver's first
// evaluation at lam_a (p->ev, records into buffer 1)
cudaError_t launch_dual_g2(const ra_problem *p, const double *lam_a, const double *lam_b,
                           double *g_out, bool first_eval, cudaStream_t s);
cudaError_t launch_records(const ra_problem *p, int32_t *j12, float *t12, cudaStream_t s);
// the solver's lower-bound pass over the records the last evaluation wrote
// (into p->lb_slot[p->ev->rec_buf]); does nothing when *skip != 0
cudaError_t launch_lagged_bound(const ra_problem *p, const int32_t *skip, cudaStream_t s);
cudaError_t launch_recover(const ra_problem *p, const double *lam, int32_t *jstar, int32_t *j12,
                           float *x12, float *t, float *X, double *U, uint8_t *near_tie,
                           unsigned long long *n_ties, cudaStream_t s);
cudaError_t configure_dual(ra_problem *p);
cudaError_t launch_batch_dual(int mt, const BatchDualArgs &a, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_batch_init(int mt, const BatchDualArgs &a, double *lam1_concat,
                              const long long *lam_off, int grid, cudaStream_t s);
int batch_stages(int mt, int cap);
size_t batch_smem(int mt, int cap);
cudaError_t batch_configure(int mt, int cap, int *blocks_per_sm);

// One problem for the warm-start statistics (device copy or by value).
struct FeatProblem {
    const float *A;
    const uint8_t *kind;
    const float *w;
    const double *R;
    long long n;
    int m;
    long long row0;   // first output row (resource 0) of this problem
};

// Warm start (ra_warm.cu).
cudaError_t launch_features(const FeatProblem *probs, const FeatProblem &one, int P, int m_max,
                            float *stats, float *feats, cudaStream_t s);
cudaError_t mlp_reserve(ra_mlp *net, int rows);
cudaError_t mlp_forward(ra_mlp *net, const float *X, int rows, float *y_out, cudaStream_t s);
cudaError_t mlp_train_step(ra_mlp *net, const float *X, const float *target, int rows, float lr,
                           float *loss, cudaStream_t s);
cudaError_t launch_exp_prices(int m, const float *y, double *lam, cudaStream_t s);
// one problem's statistics, network input, network and start prices (two launches)
cudaError_t launch_warm_network(const FeatProblem &one, int m, float *stats, const ra_mlp *net,
                                float *feats, float *y, double *lam, cudaStream_t s);
cudaError_t launch_choose(int m, const double *lam_w, const double *lam_c, const double *g2,
                          double *lam0, int32_t *used, cudaStream_t s);

// Solver (ra_solve.cu).
ra_status solve(ra_problem *p, const ra_solve_opts *o, const double *lambda0, double *lambda_out,
                double *lambda_lb, ra_solve_info *info);
int32_t solve_history(ra_problem *p, double *hist, int32_t cap);
int32_t solve_certificate(ra_problem *p, double *theta, double *lam, int32_t *scaled);

ra_status batch_solve(ra_batch *b, const ra_solve_opts *o, const double *lambda0,
                      double *lambda_out, ra_solve_info *infos, double *seconds);
ra_status solve_sharded(ra_problem *p, int64_t n_total, int32_t rank, int32_t world, double *send,
                        double *recv, ra_allgather_fn fn, void *ctx, const ra_solve_opts *o,
                        const double *lambda0, double *lambda_out, ra_solve_info *info);
ra_status eval_partial(ra_problem *p, const double *lambda, double *part);
ra_status batch_rebalance(ra_batch *b, const double *lambda, const double *R_total, double step);
ra_status combine_partials(int32_t S, int32_t m, const double *parts, const double *lambda,
                           const double *R, double *g, double *q, void *stream);

// Error reporting (ra_api.cu).
ra_status fail(ra_status s, const char *fmt, ...);

// Bound of the kernels' device waits in ns (ra_set_wait_timeout; ra_api.cu).
uint64_t wait_limit_ns();

// Feasible allocation with tie-aware repair (ra_repair.cu).
ra_status repair_allocation(ra_problem *p, const double *lam, const ra_repair_opts &o, int32_t *jk,
                            float *xk, float *X, ra_repair_info *info);
void release_repair_work(ra_problem *p);

}  // namespace ra

struct ra_batch {
    int P;
    uint32_t flags;
    cudaStream_t stream;
    int device;
    int num_sms;
    long long *n_h;            // host copies
    int *m_h;
    long long *lam_off_h;      // offset of problem p's prices in the concatenated vector
    long long m_total;
    ra::BatchProblem *probs;   // device, P
    ra::SolverState *st;       // device, P
    ra::EvalOut *ev;           // device, P
    int32_t *pingpong;         // device, P
    int32_t *lag_on;           // device, P
    long long *lam_off;        // device, P
    int32_t *active;           // device, 1: problems still iterating
    unsigned *ticket;          // device, P
    int *status;               // device
    float2 *lbt_pool[2];
    uchar2 *lbj_pool[2];
    double *lam_tmp;           // device, m_total
    int nchunks[4];
    int32_t *chunk_prob[4];
    int32_t *chunk_tile0[4];
    int32_t *chunk_ntiles[4];
    double *partials[4];
    int grid[4];               // CTAs of the batched dual pass per class
    int grid_init[4];
    unsigned long long *t0;    // device: global timer at the start of the solve
    ra_solve_info *info;       // device, P
    double *secs;              // device, P
    ra::FeatProblem *feat_probs; // device, P (warm-start statistics)
    float *feat_stats;         // device, m_total x RA_MLP_STATS
    int m_max;
};

struct ra_mlp {
    cudaStream_t stream;
    float *theta;      // RA_MLP_PARAMS each: parameters, last gradient, Adam moments
    float *grad;
    float *m1;
    float *m2;
    float *act;        // activations of up to cap_rows rows
    int cap_rows;
    int t;             // Adam step count
};
