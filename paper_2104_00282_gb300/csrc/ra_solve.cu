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

// Set the solver's first trial point and constants.  lam0 may be NULL when the
// initial prices have already been written to st->lam_trial.
__global__ void solver_setup_kernel(SolverState *st, const double *lam0, const double *R, int m,
                                    double tol, int max_evals, int mem, int update,
                                    double lam_floor, int cap, int32_t *pingpong, int32_t *lag_on)
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
        st->m = m;
        st->mem = mem;
        st->max_evals = max_evals;
        st->update = update;
        st->hist_len = 0;
        st->tol = tol;
        st->lam_floor = fl;
        st->g_best = __longlong_as_double(0x7ff0000000000000ll);
        st->U_best = -__longlong_as_double(0x7ff0000000000000ll);
        st->gap = __longlong_as_double(0x7ff0000000000000ll);
        st->step = 1.0;
        st->g_bt = __longlong_as_double(0x7ff0000000000000ll);
        st->last_step = 0.05 * lmax;
        st->sg_pending = 0;
        *pingpong = 0;
        *lag_on = 0;
    }
}

// Projected L-BFGS direction at the current point (two-loop recursion on the
// free coordinates; lane j owns coordinate j).
__device__ void lbfgs_direction(SolverState *st, int j, int m, bool active)
{
    const double q = active ? st->q_cur[j] : 0.0;
    const double l = active ? st->lam_cur[j] : 0.0;
    const bool fixed = !active || (l <= st->lam_floor && q > 0.0);
    double v = fixed ? 0.0 : q;
    double alph[kMaxLbfgsMem];
    const int cnt = st->mem_count, mem = st->mem, head = st->mem_head;
    for (int c = 0; c < cnt; ++c) {  // newest first
        const int idx = (head - 1 - c + mem) % mem;
        const double sj = fixed ? 0.0 : st->S[idx][j];
        const double yj = fixed ? 0.0 : st->Y[idx][j];
        const double a = st->rho[idx] * wsum(sj * v);
        alph[c] = a;
        v -= a * yj;
    }
    double gamma;
    if (cnt > 0) {
        const int idx = (head - 1 + mem) % mem;
        const double sj = active ? st->S[idx][j] : 0.0, yj = active ? st->Y[idx][j] : 0.0;
        gamma = wsum(sj * yj) / fmax(wsum(yj * yj), 1e-300);
    } else {
        const double ln = sqrt(wsum(l * l)), qn = sqrt(wsum(fixed ? 0.0 : q * q));
        gamma = qn > 0.0 ? 0.05 * fmax(ln, 1e-300) / qn : 0.0;
    }
    v *= gamma;
    for (int c = cnt - 1; c >= 0; --c) {  // oldest first
        const int idx = (head - 1 - c + mem) % mem;
        const double sj = fixed ? 0.0 : st->S[idx][j];
        const double yj = fixed ? 0.0 : st->Y[idx][j];
        const double b = st->rho[idx] * wsum(yj * v);
        v += sj * (alph[c] - b);
    }
    double d = fixed ? 0.0 : -v;
    // not a descent direction: drop the memory and take a scaled gradient step
    if (wsum(d * (active ? q : 0.0)) >= 0.0) {
        const double ln = sqrt(wsum(l * l)), qn = sqrt(wsum(fixed ? 0.0 : q * q));
        const double g0 = qn > 0.0 ? 0.05 * fmax(ln, 1e-300) / qn : 0.0;
        d = fixed ? 0.0 : -g0 * q;
        if (j == 0) {
            st->mem_count = 0;
            st->mem_head = 0;
        }
    }
    if (active) st->d[j] = d;
}

// Store the pair (s, y) = (lambda_t - lambda_cur, q_t - q_cur) when it has
// positive curvature, then make lambda_t the current point.
__device__ void accept_point(SolverState *st, int j, bool active, double g_t, double q_t,
                             double lam_t, bool store_pair)
{
    if (store_pair && st->phase == 1) {
        const double sv = active ? lam_t - st->lam_cur[j] : 0.0;
        const double yv = active ? q_t - st->q_cur[j] : 0.0;
        const double sy = wsum(sv * yv);
        const double ss = wsum(sv * sv), yy = wsum(yv * yv);
        if (sy > 1e-12 * sqrt(ss * yy) && sy > 0.0) {
            const int idx = st->mem_head;
            if (active) {
                st->S[idx][j] = sv;
                st->Y[idx][j] = yv;
            }
            __syncwarp();
            if (j == 0) {
                st->rho[idx] = 1.0 / sy;
                st->mem_head = (idx + 1) % st->mem;
                st->mem_count = min(st->mem_count + 1, st->mem);
            }
        }
        if (j == 0) st->last_step = sqrt(ss);
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
__device__ void lbfgs_update(SolverState *st, int j, int m, bool active, double g_t, double q_t,
                             double lam_t)
{
    const bool fin = isfinite(g_t);
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
            accept_point(st, j, active, g_t, q_t, lam_t, true);
            lbfgs_direction(st, j, m, active);
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
                accept_point(st, j, active, st->g_bt, qb, lb, true);
                lbfgs_direction(st, j, m, active);
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
    if (active) st->lam_trial[j] = fmax(st->lam_cur[j] + st->step * st->d[j], st->lam_floor);
}

// One update after the evaluation of st->lam_trial (results in *ev).
__global__ void __launch_bounds__(32)
    solver_update_kernel(SolverState *st, const EvalOut *ev, int32_t *pingpong, int32_t *lag_on,
                         const int *kstatus, cudaGraphConditionalHandle cond, int use_cond,
                         int32_t *done_host_flag)
{
    const int j = threadIdx.x;
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
    const double lam_pe = active ? st->lam_prev_eval[j] : 0.0;
    if (st->have_lb_prev && ev->Ulb_prev > U_best) {
        U_best = ev->Ulb_prev;
        if (active) st->lam_lb[j] = lam_pe;
    }
    const int feasible = wmin_i(active ? (q_t >= 0.0 ? 1 : 0) : 1);
    if (feasible && ev->Ux > U_best) {
        U_best = ev->Ux;
        if (active) st->lam_lb[j] = lam_t;
    }
    if (active) st->lam_prev_eval[j] = lam_t;
    double g_best = st->g_best;
    const bool improved = g_t < g_best;
    if (improved) {
        g_best = g_t;
        if (active) st->lam_best[j] = lam_t;
    }
    // column scaling of this evaluation, consumed by the next pass
    if (active) st->s_lag[j] = r_t > st->R[j] ? st->R[j] / r_t : 1.0;
    const double den = fmax(fmax(fabs(U_best), fabs(g_best)), 1.0);
    const bool finite = isfinite(U_best) && isfinite(g_best);
    const double gap = finite ? (g_best - U_best) / den : __longlong_as_double(0x7ff0000000000000ll);
    __syncwarp();
    if (j == 0) {
        st->evals = evals;
        st->g_best = g_best;
        st->U_best = U_best;
        st->gap = gap;
        const int h = st->hist_len;
        if (h < kHist) {
            st->hist[h][0] = evals;
            st->hist[h][1] = g_t;
            st->hist[h][2] = U_best;
            st->hist[h][3] = gap;
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
            if (active) {
                st->lam_cur[j] = lam_t;
                st->lam_trial[j] = fmax(lam_t - a * q_t, st->lam_floor);
            }
            if (j == 0) st->k = st->k + 1;
        } else {
            lbfgs_update(st, j, m, active, g_t, q_t, lam_t);
        }
    }
    __syncwarp();
    if (j == 0) {
        if (done) {
            st->done = 1;
            st->status = status;
        }
        *pingpong = *pingpong ^ 1;  // this evaluation's records become "previous"
        *lag_on = 1;
        st->have_lb_prev = 1;
        const int fin = st->done;
        if (done_host_flag) *done_host_flag = fin;
        if (use_cond) cudaGraphSetConditional(cond, fin ? 0u : 1u);
    }
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
    e = cudaMemcpyAsync(hist, p->st->hist, sizeof(double) * 4 * len, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e == cudaSuccess ? len : -1;
}

ra_status solve(ra_problem *p, const ra_solve_opts *o, const double *lambda0, double *lambda_out,
                double *lambda_lb, ra_solve_info *info)
{
    ra_solve_opts opts;
    ra_solve_opts_default(&opts);
    if (o) opts = *o;
    if (opts.lbfgs_mem < 1 || opts.lbfgs_mem > kMaxLbfgsMem)
        return fail(RA_EINVAL, "lbfgs_mem must be in [1, %d]", kMaxLbfgsMem);
    if (opts.max_evals < 1) return fail(RA_EINVAL, "max_evals must be >= 1");
    if (!(opts.tol_rel >= 0.0)) return fail(RA_EINVAL, "tol_rel must be >= 0");
    if (!lambda_out) return fail(RA_EINVAL, "lambda_out is NULL");
    cudaStream_t s = p->stream;
    cudaError_t e;
    SolverState *st = p->st;
    int32_t *pingpong = p->graph_flag;
    int32_t *lag_on = p->graph_flag + 1;
    int32_t *done_flag = p->graph_flag + 2;
    const int cap = !(p->flags & RA_NO_JOB_CAP);
    if ((e = cudaMemsetAsync(p->status, 0, sizeof(int), s)) != cudaSuccess)
        return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    if (!lambda0) {
        if ((e = launch_init(p, st->lam_trial, s)) != cudaSuccess)
            return fail(RA_ECUDA, "init launch: %s", cudaGetErrorString(e));
    }
    solver_setup_kernel<<<1, 32, 0, s>>>(st, lambda0, p->R, p->m, opts.tol_rel, opts.max_evals,
                                         opts.lbfgs_mem, opts.update, opts.lam_floor, cap,
                                         pingpong, lag_on);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return fail(RA_ECUDA, "setup launch: %s", cudaGetErrorString(e));

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
    dp.lbt_prev = p->lbt[0];  // non-NULL selects the lagged instantiation
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
    dp.skip = nullptr;

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
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                cudaError_t e1 = launch_dual(p, dp, s);
                solver_update_kernel<<<1, 32, 0, s>>>(st, p->ev, pingpong, lag_on, p->status, cond,
                                                      1, nullptr);
                cudaError_t e2 = cudaGetLastError();
                cudaError_t e3 = cudaStreamEndCapture(s, &body);
                ok = e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess;
            }
        }
        ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        ok = ok && cudaGraphLaunch(exec, s) == cudaSuccess;
        if (ok) graph_ok = true;
        if (!ok) (void)cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);   // destruction waits for nothing; launch is queued
        if (graph) cudaGraphDestroy(graph);
    }
    if (!graph_ok) {
        // host-driven fallback: launch 8 iterations at a time, then check the flag
        int32_t done_h = 0;
        dp.skip = done_flag;
        if ((e = cudaMemsetAsync(done_flag, 0, sizeof(int32_t), s)) != cudaSuccess)
            return fail(RA_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        for (int it = 0; it < opts.max_evals && !done_h; it += 8) {
            for (int k = 0; k < 8; ++k) {
                if ((e = launch_dual(p, dp, s)) != cudaSuccess)
                    return fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
                solver_update_kernel<<<1, 32, 0, s>>>(st, p->ev, pingpong, lag_on, p->status, 0, 0,
                                                      done_flag);
            }
            if ((e = cudaMemcpyAsync(&done_h, done_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)
                return fail(RA_ECUDA, "solver loop: %s", cudaGetErrorString(e));
        }
    }
    if ((e = cudaMemcpyAsync(lambda_out, st->lam_best, sizeof(double) * p->m,
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return fail(RA_ECUDA, "copy prices: %s", cudaGetErrorString(e));
    if (lambda_lb && (e = cudaMemcpyAsync(lambda_lb, st->lam_lb, sizeof(double) * p->m,
                                          cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return fail(RA_ECUDA, "copy prices: %s", cudaGetErrorString(e));
    struct {
        int32_t status, k, evals, ls_fail;
        double g, U, gap;
    } h;
    int32_t ints[8];
    double dbl[8];
    e = cudaMemcpyAsync(ints, &st->phase, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbl, &st->tol, sizeof(double) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(RA_ECUDA, "solver result: %s", cudaGetErrorString(e));
    h.status = ints[2];
    h.k = ints[3];
    h.evals = ints[4];
    h.ls_fail = ints[6];
    h.g = dbl[4];
    h.U = dbl[5];
    h.gap = dbl[6];
    if (info) {
        info->status = h.status;
        info->iters = h.k;
        info->evals = h.evals;
        info->ls_fail = h.ls_fail;
        info->g = h.g;
        info->U_lb = h.U;
        info->rel_gap = h.gap;
        info->gap_per_job = (h.g - h.U) / static_cast<double>(p->n);
    }
    if (h.status == RA_ETIMEOUT) return fail(RA_ETIMEOUT, "a device wait gave up during the solve");
    if (h.status == RA_EUNBOUNDED) return fail(RA_EUNBOUNDED, "dual value not finite: a price reached zero without the per-job cap");
    if (h.status == RA_ENOTCONV) return fail(RA_ENOTCONV, "stopped after %d evaluations at relative gap %.3e", h.evals, h.gap);
    return RA_OK;
}

}  // namespace ra
