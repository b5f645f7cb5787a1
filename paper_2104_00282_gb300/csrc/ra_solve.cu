// Price discovery loop (Algorithm 2 of arXiv 2104.00282, Section 5) kept on
// the device: every iteration is {fused dual evaluation, price update}; the
// update runs in one warp in FP64 and decides on its own whether to continue,
// so the whole loop is one CUDA graph whose while-node condition the update
// kernel sets.  Nothing returns to the host until the gap test passes.
//
// Price update: projected L-BFGS (memory <= 16) with Armijo backtracking on
// the box lambda >= floor -- the quasi-Newton update the paper recommends
// ("More efficient price updates"; Section 6.1 uses memory 10) -- or the
// projected subgradient step lambda+ = max(lambda - a_k q, floor) with
// a_k = a_0 / sqrt(k).  Stopping: the relative duality gap between the best
// dual value and the best feasible utility (column-scaled allocation of an
// earlier evaluation, Section 5).

#include <cstdio>
#include <cstring>

#include "ra_internal.cuh"

namespace ra {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ float wsumf(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ double wmax(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

__device__ __forceinline__ int wmin_i(int v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

__device__ __forceinline__ unsigned long long device_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Set one solver's first trial point and constants (one warp).  lam0 may be
// NULL when the initial prices have already been written to st->lam_trial.
__device__ void setup_one(SolverState *st, const double *lam0, const double *R, int m, double tol,
                          int max_evals, int mem, int update, double lam_floor, int cap,
                          int use_master, double init_step, int32_t *pingpong, int32_t *lag_on,
                          int stall_window)
{
    const int j = threadIdx.x;
    double l = 0.0;
    if (j < m) {
        l = lam0 ? lam0[j] : st->lam_trial[j];
        st->R[j] = R[j];
    }
    const double lmax = wmax(j < m ? l : 0.0);
    double fl = lam_floor;
    if (fl < 0.0) fl = cap ? 0.0 : 1e-12 * lmax;
    if (j < m) st->lam_trial[j] = fmax(l, fl);
    if (j == 0) {
        st->phase = 0;
        st->done = 0;
        st->status = RA_OK;
        st->k = 0;
        st->evals = 0;
        st->ls_iter = 0;
        st->ls_fail = 0;
        st->mem_count = 0;
        st->mem_head = 0;
        st->have_lb_prev = 0;
        st->own_lb = 0;
        st->own_ok = 0;
        st->m = m;
        st->mem = mem;
        st->max_evals = max_evals;
        st->update = update;
        st->hist_len = 0;
        st->cap = cap;
        st->tol = tol;
        st->lam_floor = fl;
        st->g_best = __longlong_as_double(0x7ff0000000000000ll);
        st->U_best = -__longlong_as_double(0x7ff0000000000000ll);
        st->gap = __longlong_as_double(0x7ff0000000000000ll);
        st->step = 1.0;
        st->g_bt = __longlong_as_double(0x7ff0000000000000ll);
        st->last_step = init_step * lmax;
        st->init_step = init_step;
        st->sg_pending = 0;
        st->cand_count = 0;
        st->cand_head = 0;
        st->lb_stall = 0;
        st->use_master = use_master;
        st->master_ok = 0;
        st->theta_n = 0;
        st->U_master = -__longlong_as_double(0x7ff0000000000000ll);
        st->t_start = device_ns();
        st->t_done = 0ull;
        st->t_last = st->t_start;
        st->eval_ns = 0.0;
        st->step_ns = 0.0;
        st->stall_window = stall_window;
        st->mark_evals = 0;
        st->gap_mark = __longlong_as_double(0x7ff0000000000000ll);
        *pingpong = 0;
        *lag_on = 0;
    }
}

__global__ void solver_setup_kernel(SolverState *st, const double *lam0, const double *R, int m,
                                    double tol, int max_evals, int mem, int update,
                                    double lam_floor, int cap, int use_master, double init_step,
                                    int32_t *pingpong, int32_t *lag_on, int stall_window,
                                    int own_lb)
{
    setup_one(st, lam0, R, m, tol, max_evals, mem, update, lam_floor, cap, use_master, init_step,
              pingpong, lag_on, stall_window);
    if (threadIdx.x == 0) st->own_lb = own_lb;
}

// After a host-side repair of the lower bound (ra_repair.cu) at the best
// prices: adopt its utility U_rep if it is better, record it as the
// certificate (one repaired allocation at lam_best), update the gap and
// decide whether the solve is done; otherwise let the loop resume without a
// stall exit.  The repair used the lower-bound record buffers, so the next
// evaluation carries no lagged bound.
__global__ void repair_accept_kernel(SolverState *st, double U_rep, const EvalOut *exact,
                                     double tol_exact, int32_t *lag_on, int32_t *rec_on,
                                     int next_window)
{
    const int j = threadIdx.x;
    const int m = st->m;
    // the repaired utility is exact (FP64), and so is g at lam_best from the
    // FP64 pass: their gap needs no allowance for FP32 rounding.  When it
    // meets the request the pair certifies the solve even if a bound formed
    // with FP32 per-job arithmetic was nominally higher.
    const double g64 = exact->g;
    const double den64 = fmax(fmax(fabs(U_rep), fabs(g64)), 1.0);
    const bool exact_ok = isfinite(g64) && isfinite(U_rep) && (g64 - U_rep) / den64 <= tol_exact;
    const bool better = U_rep > st->U_best || exact_ok;
    if (better && j < m) {
        st->lam_lb[j] = st->lam_best[j];
        st->theta_lam[0][j] = st->lam_best[j];
    }
    __syncwarp();
    if (j == 0) {
        if (better) {
            st->U_best = U_rep;
            st->theta_n = 1;
            st->theta[0] = 1.0;
            st->theta_scaled[0] = 2;
            st->master_ok = 0;
        }
        const double den = fmax(fmax(fabs(st->U_best), fabs(st->g_best)), 1.0);
        double gap = (st->g_best - st->U_best) / den;
        if (exact_ok) {
            st->g_best = g64;
            gap = (g64 - U_rep) / den64;
        }
        st->gap = gap;
        const int h = st->hist_len;
        if (better && h > 0) {
            st->hist[h - 1][2] = st->U_best;
            st->hist[h - 1][3] = gap;
        }
        if (gap <= st->tol || exact_ok) {
            st->done = 1;
            st->status = RA_OK;
        } else if (st->evals >= st->max_evals) {
            st->done = 1;
            st->status = RA_ENOTCONV;
        } else {
            st->done = 0;
            st->status = RA_OK;
            st->stall_window = next_window;   // the next exit waits longer (0: none)
            st->gap_mark = gap;
            st->mark_evals = st->evals;
        }
        st->have_lb_prev = 0;
        *lag_on = 0;
        *rec_on = 1;
        st->t_last = device_ns();   // the repair's time counts as neither
    }
}

// Batched setup: block p sets up problem p; its starting prices are
// lam0[lam_off[p] .. + m_p).
__global__ void batch_setup_kernel(SolverState *st, const BatchProblem *probs, const double *lam0,
                                   const long long *lam_off, double tol, int max_evals, int mem,
                                   int update, double lam_floor, int cap, int use_master,
                                   double init_step, int32_t *pingpong, int32_t *lag_on)
{
    const int p = blockIdx.x;
    setup_one(st + p, lam0 + lam_off[p], probs[p].R, probs[p].m, tol, max_evals, mem, update,
              lam_floor, cap, use_master, init_step, pingpong + p, lag_on + p, 0);
}

// Graph condition of the batched loop: continue while any problem iterates.
__global__ void __launch_bounds__(1024)
    batch_any_active_kernel(const SolverState *st, int P, cudaGraphConditionalHandle cond,
                            int use_cond, int32_t *active)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) mine |= st[p].done == 0;
    if (__syncthreads_or(mine) && threadIdx.x == 0) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        *active = any;
        if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
}

// Projected L-BFGS direction at the current point (two-loop recursion on the
// free coordinates; lane j owns coordinate j).
// Search direction d = -H q_cur by the two-loop recursion over the stored
// pairs, lane j holding coordinate j; coordinates at the price floor with a
// positive subgradient are held fixed (the projection).  The recursion is a
// chain of dependent warp sums, so it runs in FP32 (FP64 arithmetic is slow
// on this GPU and a direction needs no more): all pairs are loaded at once,
// and the loops are unrolled over the largest memory so that the
// coefficients stay in registers.
__device__ void lbfgs_direction(SolverState *st, int j, int m, bool active)
{
    const double q = active ? st->q_cur[j] : 0.0;
    const double l = active ? st->lam_cur[j] : 0.0;
    const bool fixed = !active || (l <= st->lam_floor && q > 0.0);
    const int cnt = st->mem_count, mem = st->mem, head = st->mem_head;
    float sr[kMaxLbfgsMem], yr[kMaxLbfgsMem], rr[kMaxLbfgsMem], alph[kMaxLbfgsMem];
#pragma unroll
    for (int c = 0; c < kMaxLbfgsMem; ++c) {   // newest first
        const bool in = c < cnt;
        const int idx = in ? (head - 1 - c + mem) % mem : 0;   // >= 0 since c < cnt <= mem
        sr[c] = (in && !fixed) ? st->S[idx][j] : 0.0f;
        yr[c] = (in && !fixed) ? st->Y[idx][j] : 0.0f;
        rr[c] = in ? st->rho[idx] : 0.0f;
    }
    float v = fixed ? 0.0f : static_cast<float>(q);
#pragma unroll
    for (int c = 0; c < kMaxLbfgsMem; ++c) {
        if (c < cnt) {
            const float a = rr[c] * wsumf(sr[c] * v);
            alph[c] = a;
            v -= a * yr[c];
        }
    }
    float gamma;
    // update 0: diagonal without the per-job cap (g is smooth there except at
    // linear jobs), scalar with it (g is piecewise smooth with kinks that pin
    // the prices; the diagonal's long moves along flat directions land on
    // other points of the optimal face); 3: diagonal, 2: scalar
    const bool diag = st->update == 3 || (st->update == 0 && !st->cap);
    if (diag) {
        // Diagonal initial inverse Hessian D_j = lambda_j / r_j: the Newton
        // scale of a market where every buyer's spending on j is fixed (log
        // utilities: r_j = W_j / lambda_j, so dq_j / dlambda_j = r_j /
        // lambda_j); with the newest pair it is scaled so that s^T y =
        // y^T D y (the Barzilai-Borwein ratio in the D-metric), without one
        // it is halved (a damped Newton step).  Prices at zero use 1e-3 of
        // the largest price, usage below 1e-3 R_j counts as 1e-3 R_j.
        const double lmax = wmax(l);
        const double rj = active ? st->R[j] - q : 0.0;
        const double Rj = active ? st->R[j] : 0.0;
        const float dj = active ? static_cast<float>(fmax(l, 1e-3 * lmax) /
                                                     fmax(rj, fmax(1e-3 * Rj, 1e-300)))
                                : 0.0f;
        float scale = 0.5f;
        if (cnt > 0) {
            const int idx = (head - 1 + mem) % mem;
            const float sj = active ? st->S[idx][j] : 0.0f, yj = active ? st->Y[idx][j] : 0.0f;
            scale = wsumf(sj * yj) / fmaxf(wsumf(yj * dj * yj), 1e-37f);
        }
        gamma = isfinite(dj * scale) ? dj * scale : 0.0f;
    } else if (cnt > 0) {
        const int idx = (head - 1 + mem) % mem;
        const float sj = active ? st->S[idx][j] : 0.0f, yj = active ? st->Y[idx][j] : 0.0f;
        gamma = wsumf(sj * yj) / fmaxf(wsumf(yj * yj), 1e-37f);
    } else {
        const double ln = sqrt(wsum(l * l)), qn = sqrt(wsum(fixed ? 0.0 : q * q));
        gamma = qn > 0.0 ? static_cast<float>(st->init_step * fmax(ln, 1e-300) / qn) : 0.0f;
    }
    v *= gamma;
#pragma unroll
    for (int c = kMaxLbfgsMem - 1; c >= 0; --c) {   // oldest first
        if (c < cnt) {
            const float b = rr[c] * wsumf(yr[c] * v);
            v += sr[c] * (alph[c] - b);
        }
    }
    double d = fixed ? 0.0 : -static_cast<double>(v);
    // not a descent direction: drop the memory and take a scaled gradient step
    if (wsum(d * (active ? q : 0.0)) >= 0.0) {
        const double ln = sqrt(wsum(l * l)), qn = sqrt(wsum(fixed ? 0.0 : q * q));
        const double g0 = qn > 0.0 ? st->init_step * fmax(ln, 1e-300) / qn : 0.0;
        d = fixed ? 0.0 : -g0 * q;
        if (j == 0) {
            st->mem_count = 0;
            st->mem_head = 0;
        }
    }
    if (active) st->d[j] = d;
}

// ---------------------------------------------------------------------------- own lower bound

// Lower bound on the utility of an evaluation's own allocation after the
// column scaling of Section 5 (without the per-job cap: column_scales), from
// the evaluation's sums alone, so that the gap test sees it as soon as the
// evaluation ends.  Without the cap job i uses one resource j, and at its
// subproblem optimum t_i u_i'(t_i) = c_i t_i = lambda_j x_ij (Section 4.1).
// Scaling its throughput by s > 0 then gives
//     u_i(s t_i) >= u_i(t_i) + lambda_j x_ij ln s - rem_i,
// with equality for w log t, rem_i = 0 for w t^p, 0 < p < 1 (s^p >= 1 + p ln s),
// and for -w t^p, p < 0, the Taylor remainder of s^p:
//     rem_i <= p^2 (ln s)^2 / 2 e^(|p| |ln s|) |u_i(t_i)|,  |p| <= 64.
// Summed over the non-linear jobs of column j this is lambda_j (r_j - r_lin_j)
// ln s_j.  Linear utilities are kept whole or scaled up, which never lowers
// them; a column that scales them down admits no bound here (-inf).
// Warp 0; block b serves problem b.
__device__ void own_bound_body(SolverState *st, const EvalOut *ev)
{
    const int j = threadIdx.x;
    st += blockIdx.x;
    ev += blockIdx.x;
    if (st->done) return;
    const int m = st->m;
    const bool active = j < m;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const double s2 = ev->s2neg;
    const bool formed = st->own_lb && !isnan(s2);
    int ok = formed && isfinite(ev->Ux) ? 1 : 0;
    double term = 0.0, L = 0.0, sc = 1.0, scl = 1.0;
    if (formed && active) {
        const double r = ev->r[j], rl = ev->r_lin[j];
        if (!isfinite(r) || !isfinite(rl)) {
            ok = 0;
        } else {
            column_scales(st->R[j], r, rl, 0, sc, scl);
            if (scl < 1.0 && rl > 0.0) ok = 0;   // linear jobs scaled down
            const double ro = r - rl;
            if (ro > 0.0 && sc != 1.0) {
                const double ls = log(sc);
                term = st->lam_trial[j] * ro * ls;
                L = fabs(ls);
            }
        }
    }
    ok = wmin_i(active ? ok : 1) && formed && isfinite(ev->Ux);
    const double tsum = wsum(term);
    L = wmax(L);
    double U = ev->Ux + tsum;
    if (s2 > 0.0) U -= 0.5 * L * L * exp(64.0 * L) * s2;
    if (!ok || !isfinite(U)) U = -inf;
    if (active) {
        st->own_s[j] = sc;
        st->own_sl[j] = scl;
    }
    if (j == 0) {
        st->own_ok = formed ? 1 : 0;
        st->own_U = U;
    }
}

// ---------------------------------------------------------------------------- master LP

constexpr int kLpRows = RA_MAX_M + 2;              // m resource rows, convexity, objective
constexpr int kLpCols = kCand + RA_MAX_M + 1;      // candidates, slacks, right-hand side
constexpr int kLpThreads = 256;

// Lower bound from the evaluated allocations (the paper's column-scaled
// allocations and the raw subproblem solutions): weights theta >= 0,
// sum theta = 1, sum_k theta_k r_k <= R make sum_k theta_k X^k feasible, and by
// concavity of every u_i its utility is >= sum_k theta_k U_k.  The best such
// bound is the LP  max sum theta_k U_k  over that set, solved here by a dense
// tableau simplex in FP64 (Bland's rule) started from the best single
// feasible candidate.  The weights are re-checked against the constraints in
// FP64 before the bound is used.
struct LpShared {
    double T[kLpRows][kLpCols];
    double Cr[kCand][RA_MAX_M];                        // candidate usage, staged
    double CU[kCand];                                  // candidate utility, staged
};

__device__ void master_body(SolverState *st, const EvalOut *ev, double ulb_prev)
{
    extern __shared__ __align__(16) unsigned char lp_dyn[];
    LpShared &S = *reinterpret_cast<LpShared *>(lp_dyn);
    auto &T = S.T;
    auto &Cr = S.Cr;
    auto &CU = S.CU;
    __shared__ double th[kCand];
    __shared__ double fac[kLpRows];
    __shared__ double Rr[RA_MAX_M];                    // R
    __shared__ double Ri[RA_MAX_M];                    // 1 / row scale
    __shared__ int basis[RA_MAX_M + 1];
    __shared__ int feas[kCand];
    __shared__ int s_enter, s_leave, s_slotU, s_slotS, s_slotO, s_k0, s_run, s_degen, s_iters, s_ok;
    __shared__ double s_ius, s_U;
    const int tid = threadIdx.x;
    st += blockIdx.x;  // block b: problem b of a batch (one block for a single solve)
    ev += blockIdx.x;
    if (st->done) return;
    const int m = st->m;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    // append this evaluation's raw allocation and the previous one's scaled allocation
    if (tid == 0) {
        int count = st->cand_count, head = st->cand_head;
        bool fin = isfinite(ev->Ux);
        for (int j = 0; j < m; ++j) fin = fin && isfinite(ev->r[j]);
        int su = -1, ss = -1;
        if (fin) {
            su = head;
            head = (head + 1) % kCand;
            count = min(count + 1, kCand);
        }
        if (st->have_lb_prev && isfinite(ulb_prev)) {
            ss = head;
            head = (head + 1) % kCand;
            count = min(count + 1, kCand);
        }
        int so = -1;   // this evaluation's own scaled allocation
        if (fin && st->own_ok && isfinite(st->own_U)) {
            so = head;
            head = (head + 1) % kCand;
            count = min(count + 1, kCand);
        }
        st->cand_count = count;
        st->cand_head = head;
        if (su >= 0) {
            st->cand_U[su] = ev->Ux;
            st->cand_scaled[su] = 0;
        }
        if (ss >= 0) {
            st->cand_U[ss] = ulb_prev;
            st->cand_scaled[ss] = 1;
        }
        if (so >= 0) {
            st->cand_U[so] = st->own_U;
            st->cand_scaled[so] = 1;
        }
        s_slotU = su;
        s_slotS = ss;
        s_slotO = so;
        // the LP runs when the column-scaled bound has stopped closing the
        // gap near convergence, and on every sixteenth evaluation otherwise
        s_run = st->use_master && count >= 2 && !(st->gap <= st->tol) &&
                ((st->gap < 1e-2 && st->lb_stall >= 2) || (st->evals & 15) == 0);
        st->U_master = -inf;
        st->mu_ok = 0;
        st->lp_iters = 0;
    }
    __syncthreads();
    if (tid < m) {
        if (s_slotU >= 0) {
            st->cand_r[s_slotU][tid] = ev->r[tid];
            st->cand_lam[s_slotU][tid] = st->lam_trial[tid];
        }
        if (s_slotS >= 0) {
            // usage of the scaled allocation
            st->cand_r[s_slotS][tid] = st->s_lag[tid] * (st->r_prev[tid] - st->r_lin_prev[tid]) +
                                       st->s_lin_lag[tid] * st->r_lin_prev[tid];
            st->cand_lam[s_slotS][tid] = st->lam_prev_eval[tid];
        }
        if (s_slotO >= 0) {
            st->cand_r[s_slotO][tid] = st->own_s[tid] * (ev->r[tid] - ev->r_lin[tid]) +
                                       st->own_sl[tid] * ev->r_lin[tid];
            st->cand_lam[s_slotO][tid] = st->lam_trial[tid];
        }
        Rr[tid] = st->R[tid];
        Ri[tid] = st->R[tid] > 0.0 ? 1.0 / st->R[tid] : 1.0;
    }
    __syncthreads();
    if (!s_run) return;
    const int N = st->cand_count;
    const int cols = N + m + 1, rhs = N + m;
    // stage the candidates in shared memory (coalesced, all threads)
    for (int idx = tid; idx < N * m; idx += kLpThreads) Cr[idx / m][idx % m] = st->cand_r[idx / m][idx % m];
    if (tid < N) CU[tid] = st->cand_U[tid];
    __syncthreads();
    if (tid < N) {
        int f = isfinite(CU[tid]) ? 1 : 0;
        for (int j = 0; j < m; ++j) f &= Cr[tid][j] <= Rr[j] ? 1 : 0;
        feas[tid] = f;
    }
    __syncthreads();
    // best single feasible candidate (the starting basis) and the objective scale
    if (tid == 0) {
        int k0 = -1;
        double best = -inf, us = 1.0;
        for (int k = 0; k < N; ++k) {
            if (isfinite(CU[k])) us = fmax(us, fabs(CU[k]));
            if (feas[k] && CU[k] > best) {
                best = CU[k];
                k0 = k;
            }
        }
        s_k0 = k0;
        s_ius = 1.0 / us;
    }
    __syncthreads();
    const int k0 = s_k0;
    if (k0 < 0) return;
    const double ius = s_ius;
    for (int idx = tid; idx < (m + 2) * cols; idx += kLpThreads) {
        const int i = idx / cols, c = idx % cols;
        double v = 0.0;
        if (i < m) {                                   // resource rows, basis: slack i
            if (c < N) v = (c == k0 || !isfinite(CU[c])) ? 0.0 : (Cr[c][i] - Cr[k0][i]) * Ri[i];
            else if (c < rhs) v = (c - N == i) ? 1.0 : 0.0;
            else v = (Rr[i] - Cr[k0][i]) * Ri[i];
        } else if (i == m) {                           // convexity row, basis: theta_k0
            v = c < N ? 1.0 : (c == rhs ? 1.0 : 0.0);
        } else {                                       // reduced costs; rhs holds -value
            if (c < N) v = (c == k0 || !isfinite(CU[c])) ? 0.0 : (CU[c] - CU[k0]) * ius;
            else if (c == rhs) v = -CU[k0] * ius;
        }
        T[i][c] = v;
    }
    if (tid < m) basis[tid] = N + tid;
    if (tid == 0) {
        basis[m] = k0;
        s_degen = 0;
        s_iters = 0;
    }
    __syncthreads();
    for (int iter = 0; iter < 8 * kLpRows; ++iter) {
        // pricing: largest reduced cost (Dantzig); after a run of degenerate
        // pivots switch to the lowest index with a positive one (Bland),
        // which cannot cycle
        const bool bland = s_degen > kLpRows;
        if (tid < 32) {
            // reduced costs are in units of max|U_k|: 1e-11 is far below any
            // gap that matters and above the rounding the pivots accumulate
            double bv = 1e-11;
            int bc = 0x7fffffff;
            for (int c = tid; c < N + m; c += 32) {
                const double d = T[m + 1][c];
                if (bland ? (d > 1e-11 && c < bc) : (d > bv)) {
                    bv = d;
                    bc = c;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                if (bland ? (oc < bc) : (ov > bv || (ov == bv && oc < bc))) {
                    bv = ov;
                    bc = oc;
                }
            }
            // ratio test over the m + 1 constraint rows, division-free:
            // rhs_i / a_i < rhs_b / a_b  <=>  rhs_i a_b < rhs_b a_i  (a > 0);
            // ties to the lowest basis index
            int brow = -1, bb = 0x7fffffff;
            double bnum = 0.0, bden = 1.0;
            if (bc != 0x7fffffff) {
                for (int i = tid; i <= m; i += 32) {
                    const double a = T[i][bc];
                    if (a > 1e-12) {
                        const double num = fmax(T[i][rhs], 0.0);
                        const double l = num * bden, r = bnum * a;
                        if (brow < 0 || l < r || (l == r && basis[i] < bb)) {
                            bnum = num;
                            bden = a;
                            bb = basis[i];
                            brow = i;
                        }
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const double onum = __shfl_xor_sync(0xffffffffu, bnum, off);
                    const double oden = __shfl_xor_sync(0xffffffffu, bden, off);
                    const int ob = __shfl_xor_sync(0xffffffffu, bb, off);
                    const int orow = __shfl_xor_sync(0xffffffffu, brow, off);
                    if (orow < 0) continue;
                    const double l = onum * bden, r = bnum * oden;
                    if (brow < 0 || l < r || (l == r && ob < bb)) {
                        bnum = onum;
                        bden = oden;
                        bb = ob;
                        brow = orow;
                    }
                }
            }
            if (tid == 0) {
                s_enter = bc;
                s_leave = brow;
                s_degen = (brow >= 0 && bnum <= 0.0) ? s_degen + 1 : 0;
            }
        }
        __syncthreads();
        const int e = s_enter, pr = s_leave;
        if (e == 0x7fffffff || pr < 0) break;          // optimal (or no bounded step)
        if (tid < m + 2) fac[tid] = T[tid][e];
        __syncthreads();
        const double ipiv = 1.0 / fac[pr];
        for (int c = tid; c < cols; c += kLpThreads) T[pr][c] *= ipiv;
        __syncthreads();
        for (int idx = tid; idx < (m + 2) * cols; idx += kLpThreads) {
            const int i = idx / cols, c = idx % cols;
            if (i != pr) T[i][c] -= fac[i] * T[pr][c];
        }
        if (tid == 0) {
            basis[pr] = e;
            s_iters = iter + 1;
        }
        __syncthreads();
    }
    // weights, exact re-check against the limits, and the bound in original units
    if (tid < kCand) th[tid] = 0.0;
    __syncthreads();
    if (tid == 0) {
        double tsum = 0.0;
        for (int i = 0; i <= m; ++i)
            if (basis[i] < N) {
                const double t = fmax(T[i][rhs], 0.0);
                th[basis[i]] = t;
                tsum += t;
            }
        s_ok = tsum > 0.5;
        const double inv = s_ok ? 1.0 / tsum : 0.0;
        double U = 0.0;
        for (int k = 0; k < N; ++k) {
            th[k] *= inv;
            if (th[k] > 0.0) U += th[k] * CU[k];
        }
        s_U = U;
    }
    __syncthreads();
    if (tid < m && s_ok) {
        double r = 0.0;
        for (int k = 0; k < N; ++k)
            if (th[k] > 0.0) r += th[k] * Cr[k][tid];
        if (!(r <= Rr[tid] * (1.0 + 1e-12))) atomicAnd(&s_ok, 0);
    }
    __syncthreads();
    if (tid < kCand) st->lp_theta[tid] = tid < N ? th[tid] : 0.0;
    // resource duals of the scaled LP: mu_j = -(reduced cost of slack j) max|U| / R_j;
    // (mu, nu) minimise the cutting-plane model max_k [U_k + mu^T (R - r_k)] of g
    if (tid < m) st->mu_lp[tid] = fmax(-T[m + 1][N + tid], 0.0) * Ri[tid] / ius;
    if (tid == 0) {
        st->U_master = s_ok ? s_U : -inf;
        st->mu_ok = s_ok ? 1 : 0;
        st->lp_iters = s_iters;
    }
}

// lambda_trial = max(v, floor); with a zero floor, prices below 1e-12 of the
// largest one, or below 1e-30, are set to exactly zero (the FP32 kernels
// treat prices under 1e-30 as zero: their inverse would overflow and tie).
__device__ void set_trial(SolverState *st, int j, bool active, double v)
{
    v = active ? fmax(v, st->lam_floor) : 0.0;
    const double vmax = wmax(v);
    if (st->lam_floor == 0.0 && (v < 1e-12 * vmax || v < 1e-30)) v = 0.0;
    if (active) st->lam_trial[j] = v;
}

// Store the pair (s, y) = (lambda_t - lambda_cur, q_t - q_cur) when it has
// positive curvature, then make lambda_t the current point.
__device__ void accept_point(SolverState *st, int j, bool active, double g_t, double q_t,
                             double lam_t, bool store_pair)
{
    if (store_pair && st->phase == 1) {
        // the differences in FP64, the pair and its products in FP32
        const float sv = active ? static_cast<float>(lam_t - st->lam_cur[j]) : 0.0f;
        const float yv = active ? static_cast<float>(q_t - st->q_cur[j]) : 0.0f;
        const float sy = wsumf(sv * yv);
        const float ss = wsumf(sv * sv), yy = wsumf(yv * yv);
        if (sy > 1e-12f * sqrtf(ss) * sqrtf(yy) && sy > 0.0f && isfinite(1.0f / sy)) {
            const int idx = st->mem_head;
            if (active) {
                st->S[idx][j] = sv;
                st->Y[idx][j] = yv;
            }
            __syncwarp();
            if (j == 0) {
                st->rho[idx] = 1.0f / sy;
                st->mem_head = (idx + 1) % st->mem;
                st->mem_count = min(st->mem_count + 1, st->mem);
            }
        }
        if (j == 0) st->last_step = sqrt(static_cast<double>(ss));
    }
    __syncwarp();
    if (active) {
        st->lam_cur[j] = lam_t;
        st->q_cur[j] = q_t;
    }
    if (j == 0) {
        if (st->phase == 1) st->k = st->k + 1;
        st->g_cur = g_t;
        st->phase = 1;
        st->ls_iter = 0;
        st->step = 1.0;
        st->g_bt = __longlong_as_double(0x7ff0000000000000ll);
        st->sg_pending = 0;
    }
    __syncwarp();
}

// Projected L-BFGS step control.  A trial is accepted on the Armijo condition
// g_t <= g_cur + 1e-4 q_cur^T (lambda_t - lambda_cur); otherwise the step is
// cut by safeguarded quadratic interpolation (to [0.1, 0.5] of itself).  After
// 12 cuts the best decreasing trial is taken; when no trial decreased g (a
// kink of g: q_cur is only one subgradient) the memory is cleared and a
// projected subgradient step of half the last step length is taken without a
// decrease test -- the method's fallback (Section 5).  The best g and lower
// bound are tracked separately, so non-monotone steps lose nothing.
// Trial halfway towards the minimiser of the cutting-plane model (the master
// LP's duals), taken without a decrease test: it adds cuts on the far side
// of the kink the iterates are stuck at, which is what the master bound
// needs to close the gap when g is not differentiable at its minimum.
__device__ void bundle_step(SolverState *st, int j, bool active)
{
    if (active) st->d[j] = 0.5 * (st->mu_lp[j] - st->lam_cur[j]);
    if (j == 0) {
        st->mem_count = 0;
        st->mem_head = 0;
        st->ls_iter = 0;
        st->step = 1.0;
        st->sg_pending = 1;
        st->g_bt = __longlong_as_double(0x7ff0000000000000ll);
    }
    __syncwarp();
}

// The dual has stopped improving by more than a tenth of the tolerance while
// the gap is still open: the lower bound, not g, is what is left to close.
__device__ bool dual_stalled(const SolverState *st, double g_prev, double g_new)
{
    return st->mu_ok && st->use_master && st->phase == 1 &&
           g_prev - g_new < 0.1 * st->tol * fmax(fabs(g_new), 1.0);
}

__device__ void lbfgs_update(SolverState *st, int j, int m, bool active, double g_t, double q_t,
                             double lam_t)
{
    const bool fin = isfinite(g_t);
    const double g_prev = st->g_cur;
    if (st->sg_pending && !fin) {
        if (j == 0) st->step = 0.25 * st->step;   // shorten the fallback step
    } else if (st->phase == 0 || st->sg_pending) {
        accept_point(st, j, active, g_t, q_t, lam_t, st->phase == 1);
        lbfgs_direction(st, j, m, active);
    } else {
        const double dl = active ? lam_t - st->lam_cur[j] : 0.0;
        const double slope = wsum(active ? st->q_cur[j] * dl : 0.0);
        const bool armijo = fin && g_t <= st->g_cur + 1e-4 * slope;
        if (armijo) {
            const bool stalled = dual_stalled(st, g_prev, g_t);
            accept_point(st, j, active, g_t, q_t, lam_t, true);
            if (stalled) bundle_step(st, j, active);
            else lbfgs_direction(st, j, m, active);
        } else {
            if (fin && g_t < st->g_bt) {
                if (active) {
                    st->lam_bt[j] = lam_t;
                    st->q_bt[j] = q_t;
                }
                __syncwarp();
                if (j == 0) st->g_bt = g_t;
            }
            __syncwarp();
            const int iter = st->ls_iter + 1;
            if (iter < 12) {
                if (j == 0) {
                    double cut = 0.1;
                    const double den = g_t - st->g_cur - slope;
                    if (fin && den > 0.0 && slope < 0.0) cut = fmin(0.5, fmax(0.1, -slope / (2.0 * den)));
                    st->step = st->step * cut;
                    st->ls_iter = iter;
                }
            } else if (st->g_bt < st->g_cur) {
                const double lb = active ? st->lam_bt[j] : 0.0, qb = active ? st->q_bt[j] : 0.0;
                const bool stalled = dual_stalled(st, g_prev, st->g_bt);
                accept_point(st, j, active, st->g_bt, qb, lb, true);
                if (stalled) bundle_step(st, j, active);
                else lbfgs_direction(st, j, m, active);
            } else if (st->mu_ok && st->use_master) {
                if (j == 0) st->ls_fail = st->ls_fail + 1;
                bundle_step(st, j, active);
            } else {
                // kink: subgradient fallback from the current point
                const double qn = sqrt(wsum(active ? st->q_cur[j] * st->q_cur[j] : 0.0));
                const double len = 0.5 * st->last_step;
                if (active) st->d[j] = qn > 0.0 ? -st->q_cur[j] * (len / qn) : 0.0;
                if (j == 0) {
                    st->ls_fail = st->ls_fail + 1;
                    st->mem_count = 0;
                    st->mem_head = 0;
                    st->ls_iter = 0;
                    st->step = 1.0;
                    st->last_step = len;
                    st->sg_pending = 1;
                    st->g_bt = __longlong_as_double(0x7ff0000000000000ll);
                }
            }
        }
    }
    __syncwarp();
    // Without the per-job cap a price at the floor makes the dual unbounded
    // (demand of log / power jobs has no limit), and a trial there is a
    // wasted evaluation: the first trial of a line search lowers no price by
    // more than half.
    if (st->lam_floor > 0.0 && st->ls_iter == 0 && !st->sg_pending) {
        const double dj = active ? st->d[j] : 0.0;
        const double lim = (active && dj < 0.0) ? 0.5 * st->lam_cur[j] / -dj : __longlong_as_double(0x7ff0000000000000ll);
        double smax = lim;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) smax = fmin(smax, __shfl_xor_sync(kFull, smax, off));
        if (j == 0 && smax < st->step) st->step = smax;
        __syncwarp();
    }
    set_trial(st, j, active, st->lam_cur[j] + st->step * st->d[j]);
}

// One update after the evaluation of st->lam_trial (results in *ev).
__device__ void update_body(SolverState *st, const EvalOut *ev, double ulb_prev, int32_t *pingpong,
                            int32_t *lag_on, int32_t *rec_on, const int *kstatus,
                            cudaGraphConditionalHandle cond, int use_cond, int32_t *done_host_flag)
{
    const int j = threadIdx.x;
    st += blockIdx.x;  // block b: problem b of a batch (one block for a single solve)
    ev += blockIdx.x;
    pingpong += blockIdx.x;
    lag_on += blockIdx.x;
    const int m = st->m;
    const bool active = j < m;
    if (st->done) {
        if (use_cond && j == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const double g_t = ev->g;
    const double q_t = active ? ev->q[j] : 0.0;
    const double r_t = active ? ev->r[j] : 0.0;
    const double lam_t = active ? st->lam_trial[j] : 0.0;
    const int evals = st->evals + 1;

    // lower bounds: the lagged column-scaled bound of the previous evaluation,
    // and U(X) itself whenever X(lambda_t) already meets r <= R
    double U_best = st->U_best;
    const double U_prev = U_best;
    const double lam_pe = active ? st->lam_prev_eval[j] : 0.0;
    // certificate of the best bound: one allocation with weight 1, or the
    // master LP's mixture (copied, since the candidate ring moves on)
    int cert = 0;     // 1 scaled previous, 2 raw current, 3 master mixture, 4 scaled current
    if (st->have_lb_prev && ulb_prev > U_best) {
        U_best = ulb_prev;
        cert = 1;
    }
    if (st->own_ok && st->own_U > U_best) {
        U_best = st->own_U;
        cert = 4;
    }
    const int feasible = wmin_i(active ? (q_t >= 0.0 ? 1 : 0) : 1);
    if (feasible && ev->Ux > U_best) {
        U_best = ev->Ux;
        cert = 2;
    }
    // progress of the bounds this evaluation made without the master LP
    const double own = cert ? U_best : U_prev;
    const bool own_gain = isfinite(U_prev) ? (own - U_prev > 0.1 * (st->g_best - U_prev)) : cert != 0;
    if (st->use_master && st->U_master > U_best) {
        U_best = st->U_master;
        cert = 3;
    }
    if (cert == 1 || cert == 2 || cert == 4) {
        if (active) {
            st->lam_lb[j] = cert == 1 ? lam_pe : lam_t;
            st->theta_lam[0][j] = cert == 1 ? lam_pe : lam_t;
        }
        if (j == 0) {
            st->theta_n = 1;
            st->theta[0] = 1.0;
            st->theta_scaled[0] = cert != 2;
            st->master_ok = 0;
        }
    } else if (cert == 3) {
        const int N = st->cand_count;
        for (int k = 0; k < N; ++k)
            if (active) st->theta_lam[k][j] = st->cand_lam[k][j];
        for (int k = j; k < N; k += 32) {
            st->theta[k] = st->lp_theta[k];
            st->theta_scaled[k] = st->cand_scaled[k];
        }
        if (j == 0) {
            st->theta_n = N;
            st->master_ok = 1;
        }
    }
    if (active) {
        st->lam_prev_eval[j] = lam_t;
        st->r_prev[j] = r_t;
        st->r_lin_prev[j] = ev->r_lin[j];
    }
    double g_best = st->g_best;
    const double g_best_old = g_best;
    const bool improved = g_t < g_best;
    if (improved) {
        g_best = g_t;
        if (active) {
            st->lam_best[j] = lam_t;
            st->q_best[j] = q_t;
        }
    }
    // column scaling of this evaluation, consumed by the next pass
    if (active) {
        double sc, scl;
        column_scales(st->R[j], r_t, ev->r_lin[j], st->cap, sc, scl);
        st->s_lag[j] = sc;
        st->s_lin_lag[j] = scl;
    }
    const double den = fmax(fmax(fabs(U_best), fabs(g_best)), 1.0);
    const bool finite = isfinite(U_best) && isfinite(g_best);
    const double gap = finite ? (g_best - U_best) / den : __longlong_as_double(0x7ff0000000000000ll);
    __syncwarp();
    if (j == 0) {
        st->evals = evals;
        st->lb_stall = own_gain ? 0 : st->lb_stall + 1;
        st->g_best = g_best;
        st->U_best = U_best;
        st->gap = gap;
        const int h = st->hist_len;
        if (h < kHist) {
            st->hist[h][0] = evals;
            st->hist[h][1] = g_t;
            st->hist[h][2] = U_best;
            st->hist[h][3] = gap;
            st->hist[h][4] = st->U_master;
            st->hist[h][5] = st->lp_iters;
            st->hist_len = h + 1;
        }
    }
    bool done = false;
    int status = RA_OK;
    if (*kstatus != 0) {
        done = true;
        status = RA_ETIMEOUT;
    } else if (gap <= st->tol) {
        done = true;
    } else if (evals >= st->max_evals) {
        done = true;
        status = RA_ENOTCONV;
    } else if (!isfinite(g_t) && st->phase == 0) {
        done = true;             // the starting prices already give an unbounded dual
        status = RA_EUNBOUNDED;
    }
    // the gap has not halved within stall_window evaluations: leave after this
    // update so that the host can repair the lower bound at the best prices
    bool stall = false;
    if (!done && st->stall_window > 0 && isfinite(gap)) {
        if (!(gap >= 0.5 * st->gap_mark)) {
            if (j == 0) {
                st->gap_mark = gap;
                st->mark_evals = evals;
            }
        } else if (evals - st->mark_evals >= st->stall_window) {
            stall = true;
        }
    }

    if (!done) {
        if (st->update == 1) {
            // projected subgradient, a_k = a_0 / sqrt(k)
            if (st->phase == 0) {
                const double ln = sqrt(wsum(lam_t * lam_t)), qn = sqrt(wsum(q_t * q_t));
                if (j == 0) st->sg_a0 = qn > 0.0 ? 0.1 * ln / qn : 0.0;
                __syncwarp();
                if (j == 0) st->phase = 1;
            }
            const double a = st->sg_a0 / sqrt(static_cast<double>(evals));
            if (active) st->lam_cur[j] = lam_t;
            set_trial(st, j, active, lam_t - a * q_t);
            if (j == 0) st->k = st->k + 1;
        } else {
            lbfgs_update(st, j, m, active, g_t, q_t, lam_t);
        }
    }
    __syncwarp();
    if (stall) {
        done = true;
        status = kStatusStalled;
    }
    if (j == 0) {
        if (done) {
            st->done = 1;
            st->status = status;
            st->t_done = device_ns();
        }
        *pingpong = *pingpong ^ 1;  // this evaluation's records become "previous"
        if (rec_on) {
            // The lagged bound of the next evaluation needs this one's records.
            // Far from the optimum that bound is useless, so the records are
            // written only once the dual is in its local regime: the best g
            // improved by less than 1 % in this evaluation, or the gap is
            // below 1 % (and from then on).  Where the own bound is formed,
            // the next evaluation writes no records (flag 2: only r_lin and
            // the remainder sum) unless this one's scaling admitted none.
            const int cur = *rec_on;   // set bytewise by a memset: 0, 0x01010101 or 0x02020202
            const int wrote = cur & 1;
            *lag_on = wrote;
            st->have_lb_prev = wrote;
            const double dec = isfinite(g_best_old) ? (g_best_old - g_best) / fmax(fabs(g_best), 1.0) : 1.0;
            int next = (cur != 0 || dec < 1e-2 || gap < 1e-2) ? 1 : 0;
            if (next && st->own_lb == 1 && !(st->own_ok && !isfinite(st->own_U))) next = 2;
            *rec_on = next;
        } else {
            *lag_on = 1;
            st->have_lb_prev = 1;
        }
        const int fin = st->done;
        if (done_host_flag) *done_host_flag = fin;
        if (use_cond) cudaGraphSetConditional(cond, fin ? 0u : 1u);
    }
}

__global__ void stamp_kernel(unsigned long long *t) { *t = device_ns(); }

// Per-problem results of a batched solve: best prices into the concatenated
// output, the info record and the seconds from the batch start (t0) until
// the problem's solve stopped.
__global__ void batch_finish_kernel(const SolverState *st, const BatchProblem *probs,
                                    const long long *lam_off, const unsigned long long *t0,
                                    double *lam_out, ra_solve_info *info, double *secs)
{
    const int p = blockIdx.x, j = threadIdx.x;
    const SolverState *S = st + p;
    if (j < S->m) lam_out[lam_off[p] + j] = S->lam_best[j];
    if (j == 0) {
        ra_solve_info r;
        r.status = S->status;
        r.iters = S->k;
        r.evals = S->evals;
        r.ls_fail = S->ls_fail;
        r.g = S->g_best;
        r.U_lb = S->U_best;
        r.rel_gap = S->gap;
        r.gap_per_job = (S->g_best - S->U_best) / static_cast<double>(probs[p].n);
        r.repairs = 0;
        r.n_flex = 0;
        r.eval_ms = S->eval_ns * 1e-6;   // the batched passes it waited for
        r.step_ms = S->step_ns * 1e-6;
        info[p] = r;
        secs[p] = S->t_done > *t0 ? static_cast<double>(S->t_done - *t0) * 1e-9 : 0.0;
    }
}

// One solver step after an evaluation: the master LP (all threads of the
// CTA, when it runs), then the bookkeeping and price update (warp 0).  Block
// b serves problem b of a batch.
// Bytes of the solver state before the history table, and where a staged
// copy of the state sits in the step kernel's dynamic shared memory.
constexpr size_t kStateHot = offsetof(SolverState, hist);
// the fields a solve reports (phase .. step_ns) lie at the start of the state
constexpr size_t kResultBytes = offsetof(SolverState, step_ns) + sizeof(double);
static_assert(kResultBytes <= 256, "result fields fit the pinned host buffer");
constexpr size_t kStageOff = (sizeof(LpShared) + 15) / 16 * 16;
constexpr size_t kStepSmemStaged = kStageOff + sizeof(SolverState);
static_assert(kStateHot % 8 == 0, "state copy works in 8-byte words");

// dst[0, bytes) <- src[0, bytes) by all threads of the CTA (16-byte words
// where both sides allow, 8-byte words for the rest)
__device__ void copy_state(void *__restrict__ dst, const void *__restrict__ src, size_t bytes)
{
    const bool v16 = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
    size_t done = 0;
    if (v16) {
        // four loads in flight per thread before their stores
        const size_t n16 = bytes / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        const size_t step = blockDim.x;
        size_t i = threadIdx.x;
        for (; i + 3 * step < n16; i += 4 * step) {
            const uint4 a = s4[i], b = s4[i + step], c = s4[i + 2 * step], d = s4[i + 3 * step];
            d4[i] = a;
            d4[i + step] = b;
            d4[i + 2 * step] = c;
            d4[i + 3 * step] = d;
        }
        for (; i < n16; i += step) d4[i] = s4[i];
        done = n16 * 16;
    }
    const size_t n8 = (bytes - done) / 8;
    for (size_t i = threadIdx.x; i < n8; i += blockDim.x)
        reinterpret_cast<uint2 *>(static_cast<char *>(dst) + done)[i] =
            reinterpret_cast<const uint2 *>(static_cast<const char *>(src) + done)[i];
}

// STAGE (a single solve, one CTA): the step works on a copy of the solver
// state in shared memory -- its chains of dependent reads would otherwise
// each wait for L2 or DRAM (the evaluation in between streams the problem
// through L2) -- and writes the copy back, with the history rows it added.
template <bool STAGE>
__global__ void __launch_bounds__(kLpThreads)
    step_kernel(SolverState *st, const EvalOut *ev, int32_t *pingpong, int32_t *lag_on,
                int32_t *rec_on, const int *kstatus, cudaGraphConditionalHandle cond, int use_cond,
                int32_t *done_host_flag, const double *lb_slot, int32_t *first_flag)
{
    // the previous evaluation's column-scaled bound: from the evaluation
    // itself (lagged pass) or, when the bound has its own pass, from the slot
    // that pass wrote (the other slot is being written for this evaluation)
    const double ulb_prev = lb_slot != nullptr ? lb_slot[pingpong[blockIdx.x] & 1]
                                               : ev[blockIdx.x].Ulb_prev;
    extern __shared__ __align__(16) unsigned char lp_dyn[];
    SolverState *const glob = st;
    if (STAGE) {
        SolverState *sh = reinterpret_cast<SolverState *>(lp_dyn + kStageOff);
        copy_state(sh, glob, kStateHot);
        __syncthreads();
        st = sh;
    }
    SolverState *S = st + blockIdx.x;
    const int hist0 = S->hist_len;
    const unsigned long long t0 = device_ns();
    const bool live = !S->done;
    if (threadIdx.x < 32) own_bound_body(st, ev);
    __syncthreads();
    master_body(st, ev, ulb_prev);
    __syncthreads();
    if (threadIdx.x < 32)
        update_body(st, ev, ulb_prev, pingpong, lag_on, rec_on, kstatus, cond, use_cond,
                    done_host_flag);
    if (threadIdx.x == 0 && live) {
        const unsigned long long t1 = device_ns();
        if (t0 > S->t_last) S->eval_ns += static_cast<double>(t0 - S->t_last);
        if (t1 > t0) S->step_ns += static_cast<double>(t1 - t0);
        S->t_last = t1;
    }
    if (STAGE) {
        __syncthreads();
        copy_state(glob, S, kStateHot);
        const int h1 = S->hist_len;
        for (int i = hist0 * kHistCols + threadIdx.x; i < h1 * kHistCols; i += blockDim.x)
            glob->hist[i / kHistCols][i % kHistCols] = S->hist[i / kHistCols][i % kHistCols];
    }
    // a first evaluation made before the solve has been consumed
    if (first_flag != nullptr && threadIdx.x == 0) *first_flag = 0;
}

// The relative gap the loop stops at.  With FP32 per-job arithmetic the
// solver's own g and U_lb carry FP32 rounding (fast log/exp, FP32 records):
// measured up to 3.3e-7 of the relative gap against the FP64 oracle on the
// parity workloads.  The loop therefore stops at half the requested gap, so
// that the gap the FP64 oracle certifies for its result meets the request.
// FP64 per-job arithmetic stops at the request itself.
// ---------------------------------------------------------------------------- sharded solve

// One shard's evaluation sums as exchanged between the shards of a problem
// split by job range: [sum h, U(X), lagged U_lb, status word, r[m], r_lin[m]].
__host__ __device__ inline int shard_width(int m) { return 4 + 2 * m; }

__global__ void shard_pack_kernel(const EvalOut *ev, const int *status, int m, double *send)
{
    const int j = threadIdx.x;
    if (j == 0) {
        send[0] = ev->sumh;
        send[1] = ev->Ux;
        send[2] = ev->Ulb_prev;
        send[3] = static_cast<double>(*status);
    }
    if (j < m) {
        send[4 + j] = ev->r[j];
        send[4 + m + j] = ev->r_lin[j];
    }
}

// The whole problem's evaluation from every shard's sums, added in shard
// order (the same bits on every shard): g = lambda^T R + sum h, q = R - r;
// the status words are or-ed, so that every shard stops alike.
__global__ void shard_combine_kernel(const double *recv, int world, int m, const double *lam,
                                     const double *R, EvalOut *ev, int *status)
{
    const int j = threadIdx.x;
    const int W = shard_width(m);
    if (j < m) {
        double r = 0.0, rl = 0.0;
        for (int s = 0; s < world; ++s) {
            r += recv[static_cast<size_t>(s) * W + 4 + j];
            rl += recv[static_cast<size_t>(s) * W + 4 + m + j];
        }
        ev->r[j] = r;
        ev->q[j] = R[j] - r;
        ev->r_lin[j] = rl;
    }
    if (j == 0) {
        double h = 0.0, ux = 0.0, ul = 0.0;
        int st = 0;
        for (int s = 0; s < world; ++s) {
            const double *v = recv + static_cast<size_t>(s) * W;
            h += v[0];
            ux += v[1];
            ul += v[2];
            st |= static_cast<int>(v[3]);
        }
        double lr = 0.0;
        for (int k = 0; k < m; ++k) lr += lam[k] * R[k];
        ev->sumh = h;
        ev->g = lr + h;
        ev->Ux = ux;
        ev->Ulb_prev = ul;
        *status = st;
    }
}

// g and q alone from the shards' sums (shard order), for ra_combine_partials.
__global__ void shard_gq_kernel(const double *parts, int world, int m, const double *lam,
                                const double *R, double *g, double *q)
{
    const int j = threadIdx.x;
    const int W = shard_width(m);
    if (j < m && q) {
        double r = 0.0;
        for (int s = 0; s < world; ++s) r += parts[static_cast<size_t>(s) * W + 4 + j];
        q[j] = R[j] - r;
    }
    if (j == 0 && g) {
        double h = 0.0;
        for (int s = 0; s < world; ++s) h += parts[static_cast<size_t>(s) * W];
        double lr = 0.0;
        for (int k = 0; k < m; ++k) lr += lam[k] * R[k];
        *g = lr + h;
    }
}

// out[j] = sum over shards (in order) of entry j of each shard's count values.
__global__ void shard_sum_kernel(const double *recv, int world, int count, double *out)
{
    const int j = threadIdx.x;
    if (j < count) {
        double v = 0.0;
        for (int s = 0; s < world; ++s) v += recv[static_cast<size_t>(s) * count + j];
        out[j] = v;
    }
}

// ---------------------------------------------------------------------------- price coordination

// Budgets of M shards of one problem (Section 7: each shard solved on its
// own with budget R_k, the resources then moved from shards with lower
// prices to those with higher prices).  Block j, one warp: the mean price
// pbar_j of resource j over the shards, the step
//     R_kj + step (lambda_kj - pbar_j) / pbar_j * R_j / M,
// then the Euclidean projection onto {R_kj >= 0, sum_k R_kj = R_j}
// (threshold tau with sum_k max(y_k - tau, 0) = R_j, found by bisection).
// Smallest share of a resource a shard keeps, as a fraction of R_j / M.
constexpr double kRebalanceFloor = 1e-3;

__global__ void rebalance_kernel(const BatchProblem *probs, int P, int m, const double *lam,
                                 const double *R_tot, double step, double *y)
{
    const int j = blockIdx.x, lane = threadIdx.x;
    double sum = 0.0;
    for (int k = lane; k < P; k += 32) sum += lam[static_cast<size_t>(k) * m + j];
    const double pbar = wsum(sum) / P;
    const double Rj = R_tot[j];
    double ymin = INFINITY, ymax = -INFINITY;
    for (int k = lane; k < P; k += 32) {
        const double Rk = probs[k].R[j];
        const double dk = pbar > 0.0 ? (lam[static_cast<size_t>(k) * m + j] - pbar) / pbar : 0.0;
        const double v = Rk + step * dk * (Rj / P);
        y[static_cast<size_t>(k) * m + j] = v;
        ymin = fmin(ymin, v);
        ymax = fmax(ymax, v);
    }
    for (int off = 16; off > 0; off >>= 1) {
        ymin = fmin(ymin, __shfl_xor_sync(kFull, ymin, off));
        ymax = fmax(ymax, __shfl_xor_sync(kFull, ymax, off));
    }
    __syncwarp();
    // projection onto {R_k >= fl, sum_k R_k = R_j}: R_k = max(y_k - tau, fl)
    const double fl = kRebalanceFloor * Rj / P;
    double lo = ymin - Rj / P, hi = ymax;   // f(lo) >= Rj >= f(hi) = P fl
    for (int it = 0; it < 100; ++it) {
        const double tau = 0.5 * (lo + hi);
        double f = 0.0;
        for (int k = lane; k < P; k += 32) f += fmax(y[static_cast<size_t>(k) * m + j] - tau, fl);
        f = wsum(f);
        if (f > Rj) lo = tau;
        else hi = tau;
    }
    const double tau = 0.5 * (lo + hi);
    // write max(y - tau, fl), then restore sum = R_j exactly on the largest entry
    double tot = 0.0;
    for (int k = lane; k < P; k += 32) {
        const double v = fmax(y[static_cast<size_t>(k) * m + j] - tau, fl);
        const_cast<double *>(probs[k].R)[j] = v;
        tot += v;
    }
    tot = wsum(tot);
    __syncwarp();
    if (lane == 0) {
        int kbig = 0;
        double vbig = -1.0;
        for (int k = 0; k < P; ++k)
            if (probs[k].R[j] > vbig) {
                vbig = probs[k].R[j];
                kbig = k;
            }
        const_cast<double *>(probs[kbig].R)[j] = fmax(vbig + (Rj - tot), fl);
    }
}

}  // namespace

void release_loop_graph(ra_problem *p)
{
    if (p->loop_exec) cudaGraphExecDestroy(p->loop_exec);
    if (p->loop_graph) cudaGraphDestroy(p->loop_graph);
    p->loop_exec = nullptr;
    p->loop_graph = nullptr;
}

namespace {

constexpr int kMaxRepairs = 12;  // lower-bound repairs per solve (the last at max_evals)
// jobs from which a single solve without the cap forms only its own bound
constexpr long long kOwnOnlyJobs = 4000000;
constexpr int kMaxRepairWindow = 64;

double stop_tolerance(double tol, uint32_t flags)
{
    return (flags & RA_FP64_JOBMATH) ? tol : 0.5 * tol;
}

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

}  // namespace

int32_t solve_history(ra_problem *p, double *hist, int32_t cap)
{
    int32_t len = 0;
    cudaError_t e = cudaMemcpyAsync(&len, &p->st->hist_len, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return -1;
    if (len > cap) len = cap;
    if (len <= 0) return 0;
    e = cudaMemcpyAsync(hist, p->st->hist, sizeof(double) * kHistCols * len, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e == cudaSuccess ? len : -1;
}

int32_t solve_certificate(ra_problem *p, double *theta, double *lam, int32_t *scaled)
{
    int32_t nk = 0;
    SolverState *st = p->st;
    cudaError_t e = cudaMemcpyAsync(&nk, &st->theta_n, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess || nk < 0 || nk > kCand) return -1;
    if (nk == 0) return 0;
    e = cudaMemcpyAsync(theta, st->theta, sizeof(double) * nk, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(scaled, st->theta_scaled, sizeof(int32_t) * nk, cudaMemcpyDeviceToHost, p->stream);
    for (int k = 0; k < nk && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(lam + static_cast<size_t>(k) * p->m, st->theta_lam[k], sizeof(double) * p->m,
                            cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e == cudaSuccess ? nk : -1;
}

ra_status solve(ra_problem *p, const ra_solve_opts *o, const double *lambda0, double *lambda_out,
                double *lambda_lb, ra_solve_info *info)
{
    ra_solve_opts opts;
    ra_solve_opts_default(&opts);
    if (o) opts = *o;
    if (opts.lbfgs_mem < 1 || opts.lbfgs_mem > kMaxLbfgsMem)
        return fail(RA_EINVAL, "lbfgs_mem must be in [1, %d]", kMaxLbfgsMem);
    if (opts.update < 0 || opts.update > 3) return fail(RA_EINVAL, "update must be 0, 1, 2 or 3");
    if (opts.max_evals < 1) return fail(RA_EINVAL, "max_evals must be >= 1");
    if (!(opts.tol_rel >= 0.0)) return fail(RA_EINVAL, "tol_rel must be >= 0");
    if (!(opts.init_step > 0.0)) return fail(RA_EINVAL, "init_step must be > 0");
    if (!lambda_out) return fail(RA_EINVAL, "lambda_out is NULL");
    if (opts.repair_window < -1) return fail(RA_EINVAL, "repair_window must be >= -1");
    // automatic window: few jobs per resource leave the column-scaled bound
    // stalled at ties early, so repair after 4 evaluations without the gap
    // halving; otherwise after 16
    const int repair_window = opts.repair_window >= 0
                                  ? opts.repair_window
                                  : (p->n < 4096LL * p->m ? 4 : 16);
    cudaStream_t s = p->stream;
    cudaError_t e;
    SolverState *st = p->st;
    int32_t *pingpong = p->graph_flag;
    int32_t *lag_on = p->graph_flag + 1;
    int32_t *done_flag = p->graph_flag + 2;
    int32_t *rec_on = p->graph_flag + 3;   // the evaluation in flight writes lower-bound records
    // set by ra_warmstart_prices when its pass was this solve's first
    // evaluation (at the network's prices, when they were chosen): the first
    // evaluation launch then does nothing and the step reads that pass
    int32_t *first_flag = p->graph_flag + 4;
    const bool pre = lambda0 != nullptr && lambda0 == p->pre_lam0;
    p->pre_lam0 = nullptr;
    const int cap = !(p->flags & RA_NO_JOB_CAP);
    // Without the cap each evaluation bounds its own allocation from its sums
    // (1).  Below kOwnOnlyJobs jobs, and with FP64 job math, the records and
    // the lagged exact bound are kept as well (2): there the bound pass hides
    // behind the step and the record writes cost little, and the exact bound
    // is the tighter of the two where ties hold the column scaling back.
    const int own = cap ? 0 : (p->n >= kOwnOnlyJobs && !(p->flags & RA_FP64_JOBMATH)) ? 1 : 2;
    // A cold start writes no records until the dual is in its local regime;
    // prices the caller supplies may already be near the optimum, so the
    // first evaluation at them writes its records (or, forming its own bound,
    // reduces what that needs).
    if ((e = cudaMemsetAsync(p->status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(rec_on, lambda0 ? (own == 1 ? 2 : 1) : 0, sizeof(int32_t), s)) != cudaSuccess ||
        (!pre && (e = cudaMemsetAsync(first_flag, 0, sizeof(int32_t), s)) != cudaSuccess))
        return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (!lambda0) {
        // With the ray scaling, Eq. e-initialization only gives the start's
        // direction and the scale is the minimiser of g along it: on large
        // problems both passes read every ts-th tile only (at least eight
        // tiles per CTA, ts <= 16), about 0.5 ms less at n = 1e7
        const bool ray = !cap && opts.init_scale;
        long long ts = 1;
        if (ray) {
            const int g = p->grid_init > p->grid_ray ? p->grid_init : p->grid_ray;
            ts = (p->n / kTile) / (8LL * (g > 0 ? g : 1));
            if (ts > 16) ts = 16;
            if (ts < 1) ts = 1;
        }
        if ((e = launch_init(p, st->lam_trial, s, 0, ts)) != cudaSuccess)
            return fail(RA_ECUDA, "init launch: %s", cudaGetErrorString(e));
        if (ray && (e = launch_ray_scale(p, st->lam_trial, s, ts)) != cudaSuccess)
            return fail(RA_ECUDA, "ray-scale launch: %s", cudaGetErrorString(e));
    }
    solver_setup_kernel<<<1, 32, 0, s>>>(st, lambda0, p->R, p->m,
                                         stop_tolerance(opts.tol_rel, p->flags), opts.max_evals,
                                         opts.lbfgs_mem, opts.update, opts.lam_floor, cap,
                                         opts.master_lb, opts.init_step, pingpong, lag_on,
                                         repair_window, own);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(RA_ECUDA, "setup launch: %s", cudaGetErrorString(e));

    if ((e = cudaFuncSetAttribute(step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kStepSmemStaged))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(step_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sizeof(LpShared)))) != cudaSuccess)
        return fail(RA_ECUDA, "master kernel attribute: %s", cudaGetErrorString(e));
    DualParams dp{};
    dp.A = p->A;
    dp.kind = p->kind;
    dp.w = p->w;
    dp.param = p->param;
    dp.R = p->R;
    dp.n = p->n;
    dp.m = p->m;
    dp.lam = st->lam_trial;
    dp.s_prev = st->s_lag;
    dp.s_lin_prev = st->s_lin_lag;
    // The evaluation writes its records; the column-scaled bound over them is
    // a separate pass that runs beside the price update on a second stream
    // (the update consumes the previous evaluation's bound, as a lagged
    // bound would).  The pass reads 19 B per job instead of adding its work
    // to the evaluation's instruction-bound loop.
    dp.lbt_prev = nullptr;    // NULL selects the instantiation without the lagged bound
    dp.lbj_prev = nullptr;
    dp.lbt_out = p->lbt[1];
    dp.lbj_out = p->lbj[1];
    dp.lbt_buf[0] = p->lbt[0];
    dp.lbt_buf[1] = p->lbt[1];
    dp.lbj_buf[0] = p->lbj[0];
    dp.lbj_buf[1] = p->lbj[1];
    dp.pingpong = pingpong;
    dp.lag_on = lag_on;
    dp.rec_on = rec_on;
    dp.partials = p->partials;
    dp.ticket = p->ticket;
    dp.status = p->status;
    dp.out = p->ev;
    dp.skip = nullptr;
    dp.skip2 = first_flag;

    // the loop as one CUDA graph: a conditional while node whose body is
    // {dual evaluation, solver step}.  It depends only on the problem's
    // buffers and the wait limit, so it is built once and kept with the
    // problem (a repair of the lower bound resumes it too).
    if (!p->lb_side) {
        e = cudaStreamCreateWithFlags(&p->lb_side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lb_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->lb_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(RA_ECUDA, "lower-bound stream: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    if (opts.use_graph) {
        const uint64_t wns = wait_limit_ns();
        if (p->loop_exec && p->loop_wait_ns != wns) release_loop_graph(p);
        if (!p->loop_exec) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t ex = nullptr;
            cudaGraphConditionalHandle cond;
            bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
            ok = ok && cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) ==
                           cudaSuccess;
            cudaGraphNode_t node;
            cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
            cp.conditional.handle = cond;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
            if (ok) {
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    // {evaluation; then the bound pass (side stream) beside the step}
                    cudaError_t e1 = launch_dual(p, dp, s);
                    if (e1 == cudaSuccess) e1 = cudaEventRecord(p->lb_fork, s);
                    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(p->lb_side, p->lb_fork, 0);
                    if (e1 == cudaSuccess) e1 = launch_lagged_bound(p, nullptr, p->lb_side);
                    if (e1 == cudaSuccess) e1 = cudaEventRecord(p->lb_join, p->lb_side);
                    step_kernel<true><<<1, kLpThreads, kStepSmemStaged, s>>>(
                        st, p->ev, pingpong, lag_on, rec_on, p->status, cond, 1, nullptr, p->lb_slot,
                        first_flag);
                    cudaError_t e2 = cudaGetLastError();
                    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, p->lb_join, 0);
                    cudaError_t e3 = cudaStreamEndCapture(s, &body);
                    ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess;
                }
            }
            ok = ok && cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess;
            if (ok) {
                p->loop_graph = graph;
                p->loop_exec = ex;
                p->loop_wait_ns = wns;
            } else {   // the host-driven loop below does the same work
                (void)cudaGetLastError();
                if (ex) cudaGraphExecDestroy(ex);
                if (graph) cudaGraphDestroy(graph);
            }
        }
        exec = p->loop_exec;
    }
    // run the loop until its while node (or the host-driven fallback) stops
    auto run_loop = [&]() -> ra_status {
        if (exec) {
            if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess)
                return fail(RA_ECUDA, "graph launch: %s", cudaGetErrorString(e));
            return RA_OK;
        }
        // host-driven fallback: launch 8 iterations at a time, then check the flag
        int32_t done_h = 0;
        DualParams dh = dp;
        dh.skip = done_flag;
        if ((e = cudaMemsetAsync(done_flag, 0, sizeof(int32_t), s)) != cudaSuccess)
            return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        for (int it = 0; it < opts.max_evals && !done_h; it += 8) {
            for (int k = 0; k < 8; ++k) {
                if ((e = launch_dual(p, dh, s)) != cudaSuccess ||
                    (e = launch_lagged_bound(p, done_flag, s)) != cudaSuccess)
                    return fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
                step_kernel<true><<<1, kLpThreads, kStepSmemStaged, s>>>(st, p->ev, pingpong, lag_on, rec_on, p->status, 0, 0,
                                                      done_flag, p->lb_slot, first_flag);
            }
            if ((e = cudaMemcpyAsync(&done_h, done_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return fail(RA_ECUDA, "solver loop: %s", cudaGetErrorString(e));
        }
        return RA_OK;
    };
    struct {
        int32_t done, status, k, evals, ls_fail;
        double g, U, gap, eval_ns, step_ns;
    } h;
    // the result fields lie in the state's first kResultBytes: one copy into
    // the problem's pinned buffer, then one synchronisation
    auto read_state = [&]() -> ra_status {
        e = cudaMemcpyAsync(p->host_state, st, kResultBytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(RA_ECUDA, "solver result: %s", cudaGetErrorString(e));
        const SolverState *hs = static_cast<const SolverState *>(p->host_state);
        h.done = hs->done;
        h.status = hs->status;
        h.k = hs->k;
        h.evals = hs->evals;
        h.ls_fail = hs->ls_fail;
        h.g = hs->g_best;
        h.U = hs->U_best;
        h.gap = hs->gap;
        h.eval_ns = hs->eval_ns;
        h.step_ns = hs->step_ns;
        return RA_OK;
    };
    // the best prices go out before the results are read (the usual case has
    // no repair after that read, so nothing is left to enqueue after it)
    auto copy_prices = [&]() -> ra_status {
        if ((e = cudaMemcpyAsync(lambda_out, st->lam_best, sizeof(double) * p->m,
                                 cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(RA_ECUDA, "copy prices: %s", cudaGetErrorString(e));
        if (lambda_lb && (e = cudaMemcpyAsync(lambda_lb, st->lam_lb, sizeof(double) * p->m,
                                              cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(RA_ECUDA, "copy prices: %s", cudaGetErrorString(e));
        return RA_OK;
    };
    int repairs = 0;
    int64_t n_flex = 0;
    bool copied = false;
    for (;;) {
        ra_status rs = run_loop();
        if (rs == RA_OK) rs = copy_prices();
        if (rs == RA_OK) rs = read_state();
        if (rs != RA_OK) return rs;
        copied = true;
        // the lower bound stalled (or the evaluations ran out): re-mix the jobs
        // at ties at the best prices (ra_repair.cu), then stop or resume
        // (the last repair is kept for max_evals, where the prices are best)
        const bool want = repair_window > 0 &&
                          ((h.status == kStatusStalled && repairs + 1 < kMaxRepairs) ||
                           (h.status == RA_ENOTCONV && repairs < kMaxRepairs));
        if (!want) break;
        ra_repair_opts ro;
        ra_repair_opts_default(&ro);
        ra_repair_info ri;
        rs = repair_allocation(p, st->lam_best, ro, nullptr, nullptr, nullptr, &ri);
        if (rs != RA_OK) return rs;
        ++repairs;
        n_flex = ri.n_flex;
        // while the prices are still moving a repair may fall short: exit again
        // after twice as many evaluations without the gap halving
        int next = 0;
        if (repairs + 1 < kMaxRepairs) {
            next = repair_window << (repairs < 5 ? repairs : 5);
            if (next > kMaxRepairWindow) next = kMaxRepairWindow;
        }
        if ((e = launch_dual_exact(p, st->lam_best, p->ev + 1, s)) != cudaSuccess)
            return fail(RA_ECUDA, "exact evaluation: %s", cudaGetErrorString(e));
        repair_accept_kernel<<<1, 32, 0, s>>>(st, ri.U, p->ev + 1, opts.tol_rel, lag_on, rec_on, next);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return fail(RA_ECUDA, "repair accept: %s", cudaGetErrorString(e));
        copied = false;
        if ((rs = read_state()) != RA_OK) return rs;
        if (h.done) break;   // closed the gap, or out of evaluations: otherwise resume
    }
    if (h.status == kStatusStalled) h.status = RA_ENOTCONV;  // defensive: never leaves the library
    if (!copied) {
        const ra_status rs = copy_prices();
        if (rs != RA_OK) return rs;
    }
    if (info) {
        info->status = h.status;
        info->iters = h.k;
        info->evals = h.evals;
        info->ls_fail = h.ls_fail;
        info->g = h.g;
        info->U_lb = h.U;
        info->rel_gap = h.gap;
        info->gap_per_job = (h.g - h.U) / static_cast<double>(p->n);
        info->repairs = repairs;
        info->n_flex = static_cast<int32_t>(n_flex);
        info->eval_ms = h.eval_ns * 1e-6;
        info->step_ms = h.step_ns * 1e-6;
    }
    if (h.status == RA_ETIMEOUT) return fail(RA_ETIMEOUT, "a device wait gave up during the solve");
    if (h.status == RA_EUNBOUNDED) return fail(RA_EUNBOUNDED, "dual value not finite: a price reached zero without the per-job cap");
    if (h.status == RA_ENOTCONV) return fail(RA_ENOTCONV, "stopped after %d evaluations at relative gap %.3e", h.evals, h.gap);
    return RA_OK;
}


// Batched price discovery: P independent problems advance together, one
// evaluation each per loop trip (the batched dual pass of every width class,
// then the master LP and the price update with one block per problem); a
// problem that has met its gap test is skipped by all three.  The loop is a
// graph while-node that stops when no problem is left iterating.
ra_status batch_solve(ra_batch *b, const ra_solve_opts *o, const double *lambda0,
                      double *lambda_out, ra_solve_info *infos, double *seconds)
{
    ra_solve_opts opts;
    ra_solve_opts_default(&opts);
    if (o) opts = *o;
    if (opts.lbfgs_mem < 1 || opts.lbfgs_mem > kMaxLbfgsMem)
        return fail(RA_EINVAL, "lbfgs_mem must be in [1, %d]", kMaxLbfgsMem);
    if (opts.update < 0 || opts.update > 3) return fail(RA_EINVAL, "update must be 0, 1, 2 or 3");
    if (opts.max_evals < 1) return fail(RA_EINVAL, "max_evals must be >= 1");
    if (!(opts.tol_rel >= 0.0)) return fail(RA_EINVAL, "tol_rel must be >= 0");
    if (!(opts.init_step > 0.0)) return fail(RA_EINVAL, "init_step must be > 0");
    if (!lambda_out || !infos) return fail(RA_EINVAL, "lambda_out and infos must not be NULL");
    cudaStream_t s = b->stream;
    cudaError_t e;
    const int P = b->P;
    const int cap = !(b->flags & RA_NO_JOB_CAP);
    if ((e = cudaMemsetAsync(b->status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->ticket, 0, sizeof(unsigned) * P, s)) != cudaSuccess)
        return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    stamp_kernel<<<1, 1, 0, s>>>(b->t0);

    BatchDualArgs args[4];
    for (int c = 0; c < 4; ++c) {
        BatchDualArgs &a = args[c];
        a.probs = b->probs;
        a.st = b->st;
        a.ev = b->ev;
        a.pingpong = b->pingpong;
        a.lag_on = b->lag_on;
        a.chunk_prob = b->chunk_prob[c];
        a.chunk_tile0 = b->chunk_tile0[c];
        a.chunk_ntiles = b->chunk_ntiles[c];
        a.nchunks = b->nchunks[c];
        a.partials = b->partials[c];
        a.ticket = b->ticket;
        a.status = b->status;
        a.stages = batch_stages(4 << c, cap);
        a.cap = cap;
    }
    const double *lam0 = lambda0;
    if (!lam0) {
        // Eq. e-initialization for every problem; the done flags read by the
        // chunk walk are not consulted by this pass
        for (int c = 0; c < 4; ++c) {
            if (!b->nchunks[c]) continue;
            if ((e = launch_batch_init(4 << c, args[c], b->lam_tmp, b->lam_off, b->grid_init[c], s)) !=
                cudaSuccess)
                return fail(RA_ECUDA, "batched init launch: %s", cudaGetErrorString(e));
        }
        lam0 = b->lam_tmp;
    }
    batch_setup_kernel<<<P, 32, 0, s>>>(b->st, b->probs, lam0, b->lam_off,
                                        stop_tolerance(opts.tol_rel, b->flags),
                                        opts.max_evals, opts.lbfgs_mem, opts.update, opts.lam_floor,
                                        cap, opts.master_lb, opts.init_step, b->pingpong,
                                        b->lag_on);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(RA_ECUDA, "batched setup launch: %s", cudaGetErrorString(e));
    if ((e = cudaFuncSetAttribute(step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kStepSmemStaged))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(step_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sizeof(LpShared)))) != cudaSuccess)
        return fail(RA_ECUDA, "master kernel attribute: %s", cudaGetErrorString(e));

    auto body = [&](cudaGraphConditionalHandle cond, int use_cond) -> cudaError_t {
        for (int c = 0; c < 4; ++c) {
            if (!b->nchunks[c]) continue;
            cudaError_t e1 = launch_batch_dual(4 << c, args[c], b->grid[c], batch_smem(4 << c, cap), s);
            if (e1 != cudaSuccess) return e1;
        }
        step_kernel<false><<<P, kLpThreads, sizeof(LpShared), s>>>(b->st, b->ev, b->pingpong, b->lag_on, nullptr, b->status, cond,
                                              0, nullptr, nullptr, nullptr);
        batch_any_active_kernel<<<1, 1024, 0, s>>>(b->st, P, cond, use_cond, b->active);
        return cudaGetLastError();
    };

    bool graph_ok = false;
    if (opts.use_graph) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphConditionalHandle cond;
        bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
        ok = ok && cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) ==
                       cudaSuccess;
        cudaGraphNode_t node;
        cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
        if (ok) {
            cudaGraph_t g_body = cp.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(s, g_body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaError_t e1 = body(cond, 1);
                cudaError_t e3 = cudaStreamEndCapture(s, &g_body);
                ok = e1 == cudaSuccess && e3 == cudaSuccess;
            }
        }
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        ok = ok && cudaGraphLaunch(exec, s) == cudaSuccess;
        if (ok) graph_ok = true;
        if (!ok) (void)cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
    if (!graph_ok) {
        // host-driven loop: 8 trips per check of the device's "any active" word
        int32_t active_h = 1;
        cudaGraphConditionalHandle none{};
        for (int it = 0; it < opts.max_evals && active_h; it += 8) {
            for (int k = 0; k < 8; ++k)
                if ((e = body(none, 0)) != cudaSuccess)
                    return fail(RA_ECUDA, "batched loop launch: %s", cudaGetErrorString(e));
            if ((e = cudaMemcpyAsync(&active_h, b->active, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return fail(RA_ECUDA, "batched loop: %s", cudaGetErrorString(e));
        }
    }
    batch_finish_kernel<<<P, 32, 0, s>>>(b->st, b->probs, b->lam_off, b->t0, lambda_out, b->info,
                                         b->secs);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(RA_ECUDA, "batched finish launch: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(infos, b->info, sizeof(ra_solve_info) * P, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && seconds)
        e = cudaMemcpyAsync(seconds, b->secs, sizeof(double) * P, cudaMemcpyDeviceToHost, s);
    int kstatus = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&kstatus, b->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(RA_ECUDA, "batched results: %s", cudaGetErrorString(e));
    if (kstatus != 0) return fail(RA_ETIMEOUT, "a device wait gave up during the batched solve");
    int n_unb = 0, n_nc = 0;
    for (int p = 0; p < P; ++p) {
        n_unb += infos[p].status == RA_EUNBOUNDED;
        n_nc += infos[p].status == RA_ENOTCONV;
    }
    if (n_unb) return fail(RA_EUNBOUNDED, "%d of %d problems have an unbounded dual", n_unb, P);
    if (n_nc) return fail(RA_ENOTCONV, "%d of %d problems stopped before the gap test passed", n_nc, P);
    return RA_OK;
}

// Price discovery for one problem split by job range across shards (devices
// or processes): jobs are independent given the prices (Section 3), so each
// shard evaluates its own jobs, the shards exchange m-sized sums once per
// evaluation, and every shard runs the same FP64 price update on the same
// combined values -- the prices stay identical everywhere.  Host-driven loop:
// {dual pass over this shard, pack, exchange (caller's all-gather), combine
// in shard order, solver step}.
ra_status solve_sharded(ra_problem *p, int64_t n_total, int32_t rank, int32_t world, double *send,
                        double *recv, ra_allgather_fn fn, void *ctx, const ra_solve_opts *o,
                        const double *lambda0, double *lambda_out, ra_solve_info *info)
{
    ra_solve_opts opts;
    ra_solve_opts_default(&opts);
    if (o) opts = *o;
    if (world < 1 || rank < 0 || rank >= world) return fail(RA_EINVAL, "rank %d of %d", rank, world);
    if (!fn || !send || !recv || !lambda_out) return fail(RA_EINVAL, "NULL exchange, buffers or output");
    if (n_total < p->n) return fail(RA_EINVAL, "n_total = %lld < shard size %lld", (long long)n_total, (long long)p->n);
    if (opts.lbfgs_mem < 1 || opts.lbfgs_mem > kMaxLbfgsMem)
        return fail(RA_EINVAL, "lbfgs_mem must be in [1, %d]", kMaxLbfgsMem);
    if (opts.update < 0 || opts.update > 3) return fail(RA_EINVAL, "update must be 0, 1, 2 or 3");
    if (opts.max_evals < 1) return fail(RA_EINVAL, "max_evals must be >= 1");
    if (!(opts.tol_rel >= 0.0) || !(opts.init_step > 0.0)) return fail(RA_EINVAL, "bad tolerance or step");
    cudaStream_t s = p->stream;
    cudaError_t e;
    SolverState *st = p->st;
    int32_t *pingpong = p->graph_flag;
    int32_t *lag_on = p->graph_flag + 1;
    int32_t *done_flag = p->graph_flag + 2;
    const int m = p->m;
    const int cap = !(p->flags & RA_NO_JOB_CAP);
    auto exchange = [&](int count) -> ra_status {
        const int32_t rc = fn(ctx, count, static_cast<void *>(s));
        if (rc != 0) return fail(RA_ECUDA, "the caller's all-gather returned %d", rc);
        return RA_OK;
    };
    if ((e = cudaMemsetAsync(p->status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(done_flag, 0, sizeof(int32_t), s)) != cudaSuccess)
        return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (!lambda0) {
        // Eq. e-initialization over the whole problem: per-shard sums (already
        // divided by n_total), added in shard order
        if ((e = launch_init(p, p->tmp, s, n_total)) != cudaSuccess ||
            (e = cudaMemcpyAsync(send, p->tmp, sizeof(double) * m, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return fail(RA_ECUDA, "init: %s", cudaGetErrorString(e));
        ra_status rs = exchange(m);
        if (rs != RA_OK) return rs;
        shard_sum_kernel<<<1, 32, 0, s>>>(recv, world, m, st->lam_trial);
    }
    solver_setup_kernel<<<1, 32, 0, s>>>(st, lambda0, p->R, m, stop_tolerance(opts.tol_rel, p->flags),
                                         opts.max_evals, opts.lbfgs_mem, opts.update, opts.lam_floor,
                                         cap, opts.master_lb, opts.init_step, pingpong, lag_on, 0, 0);
    if ((e = cudaFuncSetAttribute(step_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(kStepSmemStaged))) != cudaSuccess ||
        (e = cudaFuncSetAttribute(step_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(sizeof(LpShared)))) != cudaSuccess)
        return fail(RA_ECUDA, "step attribute: %s", cudaGetErrorString(e));
    DualParams dp{};
    dp.A = p->A;
    dp.kind = p->kind;
    dp.w = p->w;
    dp.param = p->param;
    dp.R = p->R;
    dp.n = p->n;
    dp.m = m;
    dp.lam = st->lam_trial;
    dp.s_prev = st->s_lag;
    dp.s_lin_prev = st->s_lin_lag;
    dp.lbt_prev = p->lbt[0];
    dp.lbj_prev = p->lbj[0];
    dp.lbt_out = p->lbt[1];
    dp.lbj_out = p->lbj[1];
    dp.lbt_buf[0] = p->lbt[0];
    dp.lbt_buf[1] = p->lbt[1];
    dp.lbj_buf[0] = p->lbj[0];
    dp.lbj_buf[1] = p->lbj[1];
    dp.pingpong = pingpong;
    dp.lag_on = lag_on;
    dp.partials = p->partials;
    dp.ticket = p->ticket;
    dp.status = p->status;
    dp.out = p->ev;
    const int W = shard_width(m);
    int32_t done_h = 0;
    for (int it = 0; it < opts.max_evals && !done_h; ++it) {
        if ((e = launch_dual(p, dp, s)) != cudaSuccess)
            return fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
        shard_pack_kernel<<<1, 32, 0, s>>>(p->ev, p->status, m, send);
        ra_status rs = exchange(W);
        if (rs != RA_OK) return rs;
        shard_combine_kernel<<<1, 32, 0, s>>>(recv, world, m, st->lam_trial, p->R, p->ev, p->status);
        step_kernel<true><<<1, kLpThreads, kStepSmemStaged, s>>>(st, p->ev, pingpong, lag_on, nullptr, p->status, 0, 0,
                                                          done_flag, nullptr, nullptr);
        if ((e = cudaMemcpyAsync(&done_h, done_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(RA_ECUDA, "sharded loop: %s", cudaGetErrorString(e));
    }
    int32_t ints[8];
    double dbl[8];
    e = cudaMemcpyAsync(ints, &st->phase, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbl, &st->tol, sizeof(double) * 8, cudaMemcpyDeviceToHost, s);
    double tm[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tm, &st->eval_ns, sizeof(double) * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lambda_out, st->lam_best, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(RA_ECUDA, "sharded result: %s", cudaGetErrorString(e));
    if (info) {
        info->status = ints[2];
        info->iters = ints[3];
        info->evals = ints[4];
        info->ls_fail = ints[6];
        info->g = dbl[4];
        info->U_lb = dbl[5];
        info->rel_gap = dbl[6];
        info->gap_per_job = (dbl[4] - dbl[5]) / static_cast<double>(n_total);
        info->repairs = 0;
        info->n_flex = 0;
        info->eval_ms = tm[0] * 1e-6;   // evaluation and exchange of the sums
        info->step_ms = tm[1] * 1e-6;
    }
    if (ints[2] == RA_ETIMEOUT) return fail(RA_ETIMEOUT, "a device wait gave up on some shard");
    if (ints[2] == RA_EUNBOUNDED) return fail(RA_EUNBOUNDED, "dual value not finite");
    if (ints[2] != RA_OK) return fail(RA_ENOTCONV, "stopped after %d evaluations at relative gap %.3e", ints[4], dbl[6]);
    return RA_OK;
}

ra_status eval_partial(ra_problem *p, const double *lambda, double *part)
{
    DualParams dp{};
    dp.A = p->A;
    dp.kind = p->kind;
    dp.w = p->w;
    dp.param = p->param;
    dp.R = p->R;
    dp.n = p->n;
    dp.m = p->m;
    dp.lam = lambda;
    dp.partials = p->partials;
    dp.ticket = p->ticket;
    dp.status = p->status;
    dp.out = p->ev;
    cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = launch_dual(p, dp, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
    shard_pack_kernel<<<1, 32, 0, p->stream>>>(p->ev, p->status, p->m, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(RA_ECUDA, "pack: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status combine_partials(int32_t S, int32_t m, const double *parts, const double *lambda,
                           const double *R, double *g, double *q, void *stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    shard_gq_kernel<<<1, 32, 0, s>>>(parts, S, m, lambda, R, g, q);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RA_ECUDA, "combine: %s", cudaGetErrorString(e));
    return RA_OK;
}
ra_status batch_rebalance(ra_batch *b, const double *lambda, const double *R_total, double step)
{
    const int m = b->m_h[0];
    for (int k = 1; k < b->P; ++k)
        if (b->m_h[k] != m) return fail(RA_EINVAL, "rebalancing needs every problem to have the same m");
    if (!(step >= 0.0)) return fail(RA_EINVAL, "step = %g must be >= 0", step);
    // the batch's price scratch (sum_p m_p = P m doubles) holds the proposed budgets
    rebalance_kernel<<<m, 32, 0, b->stream>>>(b->probs, b->P, m, lambda, R_total, step, b->lam_tmp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RA_ECUDA, "rebalance: %s", cudaGetErrorString(e));
    return RA_OK;
}

}  // namespace ra
