// C ABI of libra: problem lifetime, argument checks, error strings and the
// thin host wrappers around the kernels of ra_dual.cu / ra_solve.cu.

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>
#include <vector>

#include "ra_internal.cuh"

namespace ra {

static thread_local char g_err[512] = "";

ra_status fail(ra_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static std::atomic<uint64_t> g_wait_ns{2000000000ull};

uint64_t wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

// Host-side data checks (RA_VALIDATE): problem (e-res-alloc) needs A >= 0,
// w > 0, p in (0,1), T > 0, R >= 0, all finite, and a positive efficiency for
// every log-utility job (Section 2.4: a_i = 0 with log utility is infeasible).
static ra_status validate(const ra_problem *p)
{
    const int64_t n = p->n;
    const int m = p->m;
    std::vector<float> A(static_cast<size_t>(n) * m), w(n), par(n);
    std::vector<uint8_t> kind(n);
    std::vector<double> R(m);
    cudaError_t e = cudaMemcpyAsync(A.data(), p->A, A.size() * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.data(), p->w, n * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(par.data(), p->param, n * 4, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(kind.data(), p->kind, n, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.data(), p->R, m * 8, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "validate copy: %s", cudaGetErrorString(e));
    for (int j = 0; j < m; ++j)
        if (!(std::isfinite(R[j]) && R[j] >= 0.0)) return fail(RA_EINVAL, "R[%d] = %g is not finite and >= 0", j, R[j]);
    for (int64_t i = 0; i < n; ++i) {
        if (kind[i] > RA_U_TARGET) return fail(RA_EINVAL, "kind[%lld] = %d is not a utility kind", (long long)i, kind[i]);
        if (!(std::isfinite(w[i]) && w[i] > 0.f)) return fail(RA_EINVAL, "w[%lld] = %g must be finite and > 0", (long long)i, w[i]);
        if (kind[i] == RA_U_POWER && !((par[i] > 0.f && par[i] < 1.f) || (par[i] < 0.f && par[i] >= -64.f)))
            return fail(RA_EINVAL, "param[%lld] = %g: power exponent must lie in (0, 1) or [-64, 0)",
                        (long long)i, par[i]);
        if (kind[i] >= RA_U_LINCAP && !(std::isfinite(par[i]) && par[i] > 0.f))
            return fail(RA_EINVAL, "param[%lld] = %g: target throughput must be finite and > 0", (long long)i, par[i]);
        bool any = false;
        for (int j = 0; j < m; ++j) {
            const float a = A[static_cast<size_t>(i) * m + j];
            if (!(std::isfinite(a) && a >= 0.f))
                return fail(RA_EINVAL, "A[%lld,%d] = %g must be finite and >= 0", (long long)i, j, a);
            any = any || a > 0.f;
        }
        if (!any && kind[i] == RA_U_LOG)
            return fail(RA_EINVAL, "job %lld has log utility and a zero efficiency row", (long long)i);
    }
    return RA_OK;
}

}  // namespace ra

using ra::fail;

namespace {
// A_out = A / d row by row (one demand per job) or entry by entry.
__global__ void scale_by_demand_kernel(long long n, int m, const float *A, const float *d,
                                       int per_resource, float *A_out)
{
    const long long total = n * m;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
         e += static_cast<long long>(gridDim.x) * blockDim.x)
        A_out[e] = A[e] / (per_resource ? d[e] : d[e / m]);
}
}  // namespace

extern "C" {

const char *ra_status_string(ra_status s)
{
    switch (s) {
    case RA_OK: return "ok";
    case RA_EINVAL: return "invalid argument";
    case RA_ENOMEM: return "out of device memory";
    case RA_ECUDA: return "CUDA error";
    case RA_ENOTCONV: return "not converged";
    case RA_ETIMEOUT: return "device wait timed out";
    case RA_EUNBOUNDED: return "unbounded";
    }
    return "unknown status";
}

const char *ra_last_error(void) { return ra::g_err; }

const char *ra_version(void) { return "libra 0.2 sm_103a"; }


ra_status ra_scale_by_demand(int64_t n, int32_t m, const float *A, const float *d,
                             int32_t per_resource, float *A_out, void *stream)
{
    if (n < 1 || m < 1 || m > RA_MAX_M) return fail(RA_EINVAL, "n = %lld, m = %d", (long long)n, m);
    if (!A || !d || !A_out) return fail(RA_EINVAL, "NULL argument");
    long long blocks = (n * m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    scale_by_demand_kernel<<<static_cast<int>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, m, A, d, per_resource ? 1 : 0, A_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RA_ECUDA, "demand scaling launch: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_set_wait_timeout(double seconds)
{
    if (!(seconds >= 0.0 && seconds <= 60.0))
        return fail(RA_EINVAL, "wait timeout %g s must lie in [0, 60]", seconds);
    ra::g_wait_ns.store(static_cast<uint64_t>(seconds * 1e9 + 0.5), std::memory_order_relaxed);
    return RA_OK;
}

void ra_solve_opts_default(ra_solve_opts *o)
{
    if (!o) return;
    o->tol_rel = 1e-6;
    o->max_evals = 500;
    o->lbfgs_mem = 10;
    o->update = 0;
    o->use_graph = 1;
    o->lam_floor = -1.0;
    o->master_lb = 1;
    o->repair_window = -1;
    o->init_scale = 1;
    o->pad_ = 0;
    o->init_step = 0.05;
}

ra_status ra_problem_create(int64_t n, int32_t m, const float *A, const uint8_t *kind,
                            const float *w, const float *param, const double *R, uint32_t flags,
                            void *stream, ra_problem **out)
{
    ra::g_err[0] = 0;
    if (!out) return fail(RA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1) return fail(RA_EINVAL, "n = %lld must be >= 1", (long long)n);
    if (m < 1 || m > RA_MAX_M) return fail(RA_EINVAL, "m = %d must lie in [1, %d]", m, RA_MAX_M);
    if (n > (int64_t(1) << 40)) return fail(RA_EINVAL, "n = %lld too large", (long long)n);
    if (!A || !kind || !w || !param || !R) return fail(RA_EINVAL, "a data pointer is NULL");
    if (!ra::aligned16(A) || !ra::aligned16(kind) || !ra::aligned16(w) || !ra::aligned16(param))
        return fail(RA_EINVAL, "A, kind, w and param must be 16-byte aligned");
    if (flags & ~(RA_NO_JOB_CAP | RA_FP64_JOBMATH | RA_VALIDATE)) return fail(RA_EINVAL, "unknown flags 0x%x", flags);
    ra_problem *p = new (std::nothrow) ra_problem();
    if (!p) return fail(RA_ENOMEM, "host allocation failed");
    memset(p, 0, sizeof(*p));
    p->n = n;
    p->m = m;
    p->flags = flags;
    p->A = A;
    p->kind = kind;
    p->w = w;
    p->param = param;
    p->R = R;
    p->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e == cudaSuccess) e = ra::configure_dual(p);
    if (e != cudaSuccess) {
        delete p;
        return fail(RA_ECUDA, "device query: %s", cudaGetErrorString(e));
    }
    if (flags & RA_VALIDATE) {
        ra_status vs = ra::validate(p);
        if (vs != RA_OK) {
            delete p;
            return vs;
        }
    }
    const int gmax = p->grid_dual > p->grid_aux ? p->grid_dual : p->grid_aux;
    bool ok = true;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
    };
    alloc(reinterpret_cast<void **>(&p->partials), sizeof(double) * ra::kPartW * gmax);
    alloc(reinterpret_cast<void **>(&p->ticket), sizeof(unsigned) * 8);
    alloc(reinterpret_cast<void **>(&p->status), sizeof(int) * 4);
    // throughput records: FP32 pairs, FP64 pairs with FP64 per-job arithmetic
    const size_t rec_bytes = (flags & RA_FP64_JOBMATH) ? sizeof(double2) : sizeof(float2);
    for (int b = 0; b < 2; ++b) {
        alloc(reinterpret_cast<void **>(&p->lbt[b]), rec_bytes * n);
        alloc(reinterpret_cast<void **>(&p->lbj[b]), sizeof(uchar2) * n);
    }
    alloc(reinterpret_cast<void **>(&p->ev), sizeof(ra::EvalOut) * 2);
    alloc(reinterpret_cast<void **>(&p->s_buf), sizeof(double) * RA_MAX_M);
    alloc(reinterpret_cast<void **>(&p->st), sizeof(ra::SolverState));
    alloc(reinterpret_cast<void **>(&p->graph_flag), sizeof(int32_t) * 8);
    alloc(reinterpret_cast<void **>(&p->tmp), sizeof(double) * (RA_MAX_M + 8));
    alloc(reinterpret_cast<void **>(&p->lb_slot), sizeof(double) * 2);
    alloc(reinterpret_cast<void **>(&p->warm), ra::kWarmBytes);
    if (ok && cudaHostAlloc(&p->host_state, 256, cudaHostAllocDefault) != cudaSuccess) ok = false;
    if (!ok) {
        (void)cudaGetLastError();
        ra_problem_destroy(p);
        return fail(RA_ENOMEM, "workspace allocation of about %lld bytes failed", (long long)(20 * n));
    }
    e = cudaMemsetAsync(p->ticket, 0, sizeof(unsigned) * 8, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int) * 4, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->graph_flag, 0, sizeof(int32_t) * 8, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ev, 0, sizeof(ra::EvalOut) * 2, p->stream);
    if (e != cudaSuccess) {
        ra_problem_destroy(p);
        return fail(RA_ECUDA, "workspace init: %s", cudaGetErrorString(e));
    }
    *out = p;
    return RA_OK;
}

void ra_problem_destroy(ra_problem *p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    cudaFree(p->partials);
    cudaFree(p->ticket);
    cudaFree(p->status);
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->lbt[b]);
        cudaFree(p->lbj[b]);
    }
    cudaFree(p->ev);
    cudaFree(p->s_buf);
    cudaFree(p->st);
    cudaFree(p->graph_flag);
    cudaFree(p->tmp);
    cudaFree(p->lb_slot);
    cudaFree(p->warm);
    if (p->host_state) cudaFreeHost(p->host_state);
    ra::release_loop_graph(p);
    ra::release_repair_work(p);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    if (p->lb_side) cudaStreamDestroy(p->lb_side);
    if (p->lb_fork) cudaEventDestroy(p->lb_fork);
    if (p->lb_join) cudaEventDestroy(p->lb_join);
    delete p;
}

static ra_status check_status_word(ra_problem *p)
{
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "status read: %s", cudaGetErrorString(e));
    if (st & ra::kStatusTimeout) return fail(RA_ETIMEOUT, "a device wait gave up (status 0x%x)", st);
    return RA_OK;
}

ra_status ra_eval_dual(ra_problem *p, const double *lambda, double *g, double *q, double *U_lb)
{
    if (!p || !lambda) return fail(RA_EINVAL, "NULL problem or lambda");
    p->pre_lam0 = nullptr;   // overwrites the evaluation a warm start left for ra_solve
    ra::DualParams dp{};
    dp.A = p->A;
    dp.kind = p->kind;
    dp.w = p->w;
    dp.param = p->param;
    dp.R = p->R;
    dp.n = p->n;
    dp.m = p->m;
    dp.lam = lambda;
    dp.lbt_out = U_lb ? p->lbt[0] : nullptr;
    dp.lbj_out = U_lb ? p->lbj[0] : nullptr;
    dp.partials = p->partials;
    dp.ticket = p->ticket;
    dp.status = p->status;
    dp.out = p->ev;
    // the status word reports this call's waits only
    cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "status reset: %s", cudaGetErrorString(e));
    e = ra::launch_dual(p, dp, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
    if (U_lb) {
        e = ra::launch_lower_bound(p, p->lbt[0], p->lbj[0], p->ev, U_lb, p->stream);
        if (e != cudaSuccess) return fail(RA_ECUDA, "lower-bound launch: %s", cudaGetErrorString(e));
    }
    if (g) {
        e = cudaMemcpyAsync(g, &p->ev->g, sizeof(double), cudaMemcpyDeviceToDevice, p->stream);
        if (e != cudaSuccess) return fail(RA_ECUDA, "copy g: %s", cudaGetErrorString(e));
    }
    if (q) {
        e = cudaMemcpyAsync(q, p->ev->q, sizeof(double) * p->m, cudaMemcpyDeviceToDevice, p->stream);
        if (e != cudaSuccess) return fail(RA_ECUDA, "copy q: %s", cudaGetErrorString(e));
    }
    return RA_OK;
}

ra_status ra_eval_records(ra_problem *p, int32_t *j12, float *t12)
{
    if (!p || !j12 || !t12) return fail(RA_EINVAL, "NULL argument");
    cudaError_t e = ra::launch_records(p, j12, t12, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "records launch: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_init_prices(ra_problem *p, double *lambda1)
{
    if (!p || !lambda1) return fail(RA_EINVAL, "NULL problem or output");
    p->pre_lam0 = nullptr;
    cudaError_t e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = ra::launch_init(p, lambda1, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "init launch: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_solve(ra_problem *p, const ra_solve_opts *opts, const double *lambda0,
                   double *lambda_out, double *lambda_lb, ra_solve_info *info)
{
    if (!p) return fail(RA_EINVAL, "NULL problem");
    ra_status s = ra::solve(p, opts, lambda0, lambda_out, lambda_lb, info);
    if (s == RA_OK || s == RA_ENOTCONV) {
        ra_status w = check_status_word(p);
        if (w != RA_OK) return w;
    }
    return s;
}

int32_t ra_solve_history(ra_problem *p, double *hist, int32_t cap)
{
    if (!p || !hist || cap < 0) {
        fail(RA_EINVAL, "bad arguments");
        return -1;
    }
    return ra::solve_history(p, hist, cap);
}

int32_t ra_solve_certificate(ra_problem *p, double *theta, double *lam, int32_t *scaled)
{
    if (!p || !theta || !lam || !scaled) {
        fail(RA_EINVAL, "NULL argument");
        return -1;
    }
    return ra::solve_certificate(p, theta, lam, scaled);
}

ra_status ra_recover_primal(ra_problem *p, const double *lambda, int32_t *jstar, int32_t *j12,
                            float *x12, float *t, float *X_dense, double *U, uint8_t *near_tie,
                            int64_t *n_near_ties)
{
    if (!p || !lambda) return fail(RA_EINVAL, "NULL problem or lambda");
    p->pre_lam0 = nullptr;
    unsigned long long *cnt = nullptr;
    cudaError_t e;
    if (n_near_ties) {
        cnt = reinterpret_cast<unsigned long long *>(p->tmp);
        e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), p->stream);
        if (e != cudaSuccess) return fail(RA_ECUDA, "memset: %s", cudaGetErrorString(e));
    }
    e = ra::launch_recover(p, lambda, jstar, j12, x12, t, X_dense, U, near_tie, cnt, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "recover launch: %s", cudaGetErrorString(e));
    if (n_near_ties) {
        unsigned long long h = 0;
        e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return fail(RA_ECUDA, "tie count: %s", cudaGetErrorString(e));
        *n_near_ties = static_cast<int64_t>(h);
    }
    return RA_OK;
}


ra_status ra_eval_partial(ra_problem *p, const double *lambda, double *part)
{
    if (!p || !lambda || !part) return fail(RA_EINVAL, "NULL argument");
    p->pre_lam0 = nullptr;
    return ra::eval_partial(p, lambda, part);
}

ra_status ra_combine_partials(int32_t S, int32_t m, const double *parts, const double *lambda,
                              const double *R, double *g, double *q, void *stream)
{
    if (S < 1 || m < 1 || m > RA_MAX_M) return fail(RA_EINVAL, "S = %d, m = %d", S, m);
    if (!parts || !lambda || !R) return fail(RA_EINVAL, "NULL argument");
    return ra::combine_partials(S, m, parts, lambda, R, g, q, stream);
}

ra_status ra_solve_sharded(ra_problem *p, int64_t n_total, int32_t rank, int32_t world,
                           double *send, double *recv, ra_allgather_fn fn, void *ctx,
                           const ra_solve_opts *opts, const double *lambda0, double *lambda_out,
                           ra_solve_info *info)
{
    if (!p) return fail(RA_EINVAL, "NULL problem");
    p->pre_lam0 = nullptr;
    ra_status s = ra::solve_sharded(p, n_total, rank, world, send, recv, fn, ctx, opts, lambda0,
                                    lambda_out, info);
    if (s == RA_OK || s == RA_ENOTCONV) {
        ra_status w = check_status_word(p);
        if (w != RA_OK) return w;
    }
    return s;
}

ra_status ra_batch_rebalance(ra_batch *b, const double *lambda, const double *R_total, double step)
{
    if (!b || !lambda || !R_total) return fail(RA_EINVAL, "NULL argument");
    return ra::batch_rebalance(b, lambda, R_total, step);
}

void ra_repair_opts_default(ra_repair_opts *o)
{
    if (!o) return;
    o->tie_rel = 1e-3;
    o->max_flex = 512;
    o->pad_ = 0;
}

ra_status ra_recover_feasible(ra_problem *p, const double *lambda, const ra_repair_opts *opts,
                              int32_t *jk, float *xk, float *X_dense, ra_repair_info *info)
{
    if (!p || !lambda || !info) return fail(RA_EINVAL, "NULL problem, lambda or info");
    if ((jk == nullptr) != (xk == nullptr)) return fail(RA_EINVAL, "jk and xk go together");
    p->pre_lam0 = nullptr;
    ra_repair_opts o;
    ra_repair_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.tie_rel > 0.0 && o.tie_rel <= 1.0)) return fail(RA_EINVAL, "tie_rel = %g must lie in (0, 1]", o.tie_rel);
    if (o.max_flex < 1 || o.max_flex > 4096) return fail(RA_EINVAL, "max_flex = %d must lie in [1, 4096]", o.max_flex);
    return ra::repair_allocation(p, lambda, o, jk, xk, X_dense, info);
}

// ---------------------------------------------------------------------------- batches

void ra_batch_destroy(ra_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    cudaFree(b->probs);
    cudaFree(b->st);
    cudaFree(b->ev);
    cudaFree(b->pingpong);
    cudaFree(b->lag_on);
    cudaFree(b->lam_off);
    cudaFree(b->active);
    cudaFree(b->ticket);
    cudaFree(b->status);
    cudaFree(b->t0);
    cudaFree(b->info);
    cudaFree(b->secs);
    cudaFree(b->lam_tmp);
    cudaFree(b->feat_probs);
    cudaFree(b->feat_stats);
    for (int k = 0; k < 2; ++k) {
        cudaFree(b->lbt_pool[k]);
        cudaFree(b->lbj_pool[k]);
    }
    for (int c = 0; c < 4; ++c) {
        cudaFree(b->chunk_prob[c]);
        cudaFree(b->chunk_tile0[c]);
        cudaFree(b->chunk_ntiles[c]);
        cudaFree(b->partials[c]);
    }
    delete[] b->n_h;
    delete[] b->m_h;
    delete[] b->lam_off_h;
    delete b;
}

ra_status ra_batch_create(int32_t P, const int64_t *n, const int32_t *m, const float *const *A,
                          const uint8_t *const *kind, const float *const *w,
                          const float *const *param, const double *const *R, uint32_t flags,
                          void *stream, ra_batch **out)
{
    return ra_batch_create_shaped(P, n, m, A, kind, w, param, R, flags, nullptr, stream, out);
}

ra_status ra_batch_create_shaped(int32_t P, const int64_t *n, const int32_t *m, const float *const *A,
                                 const uint8_t *const *kind, const float *const *w,
                                 const float *const *param, const double *const *R, uint32_t flags,
                                 const ra_batch_shape *shape, void *stream, ra_batch **out)
{
    ra_batch_shape sh{ra::kChunkTiles, 0, 0, 0};
    if (shape) sh = *shape;
    if (sh.chunk_tiles < 1 || sh.chunk_tiles > 4096)
        return fail(RA_EINVAL, "chunk_tiles = %d must lie in [1, 4096]", sh.chunk_tiles);
    if (sh.whole_tiles < 0 || sh.ctas_per_sm < 0 || sh.ctas_per_sm > 8)
        return fail(RA_EINVAL, "whole_tiles must be >= 0 and ctas_per_sm in [0, 8]");
    ra::g_err[0] = 0;
    if (!out) return fail(RA_EINVAL, "out is NULL");
    *out = nullptr;
    if (P < 1) return fail(RA_EINVAL, "P = %d must be >= 1", P);
    if (!n || !m || !A || !kind || !w || !param || !R) return fail(RA_EINVAL, "an argument array is NULL");
    if (flags & ~RA_NO_JOB_CAP) return fail(RA_EINVAL, "only RA_NO_JOB_CAP may be set (flags 0x%x)", flags);
    long long total = 0, m_total = 0;
    for (int p = 0; p < P; ++p) {
        if (n[p] < 1 || n[p] > (int64_t(1) << 31))
            return fail(RA_EINVAL, "problem %d: n = %lld must lie in [1, 2^31]", p, (long long)n[p]);
        if (m[p] < 1 || m[p] > RA_MAX_M)
            return fail(RA_EINVAL, "problem %d: m = %d must lie in [1, %d]", p, m[p], RA_MAX_M);
        if (!A[p] || !kind[p] || !w[p] || !param[p] || !R[p])
            return fail(RA_EINVAL, "problem %d: a data pointer is NULL", p);
        if (!ra::aligned16(A[p]) || !ra::aligned16(kind[p]) || !ra::aligned16(w[p]) ||
            !ra::aligned16(param[p]))
            return fail(RA_EINVAL, "problem %d: A, kind, w and param must be 16-byte aligned", p);
        // each problem's slice of the record pools starts at a multiple of 8
        // jobs, so its records can be bulk-copied (16-byte aligned) with its tiles
        total += (n[p] + 7) & ~7LL;
        m_total += m[p];
    }
    ra_batch *b = new (std::nothrow) ra_batch();
    if (!b) return fail(RA_ENOMEM, "host allocation failed");
    memset(b, 0, sizeof(*b));
    b->P = P;
    b->flags = flags;
    b->stream = static_cast<cudaStream_t>(stream);
    b->n_h = new (std::nothrow) long long[P];
    b->m_h = new (std::nothrow) int[P];
    b->lam_off_h = new (std::nothrow) long long[P];
    if (!b->n_h || !b->m_h || !b->lam_off_h) {
        ra_batch_destroy(b);
        return fail(RA_ENOMEM, "host allocation failed");
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        ra_batch_destroy(b);
        return fail(RA_ECUDA, "device query: %s", cudaGetErrorString(e));
    }
    // problems -> width classes -> chunks of up to kChunkTiles tiles
    std::vector<ra::BatchProblem> probs(P);
    std::vector<int32_t> cp[4], ct0[4], cnt[4];
    long long job_off = 0;
    for (int p = 0; p < P; ++p) {
        b->n_h[p] = n[p];
        b->m_h[p] = m[p];
        b->lam_off_h[p] = b->m_total;
        b->m_total += m[p];
        ra::BatchProblem &q = probs[p];
        q.A = A[p];
        q.kind = kind[p];
        q.w = w[p];
        q.param = param[p];
        q.R = R[p];
        q.n = n[p];
        q.m = m[p];
        q.cls = m[p] <= 4 ? 0 : m[p] <= 8 ? 1 : m[p] <= 16 ? 2 : 3;
        const int c = q.cls;
        const long long tiles = (n[p] + ra::kTile - 1) / ra::kTile;
        // a problem of at most whole_tiles tiles is one chunk: one CTA visits all of it
        const long long ck = tiles <= sh.whole_tiles ? tiles : sh.chunk_tiles;
        q.chunk_begin = static_cast<int>(cp[c].size());
        for (long long t0 = 0; t0 < tiles; t0 += ck) {
            cp[c].push_back(p);
            ct0[c].push_back(static_cast<int32_t>(t0));
            cnt[c].push_back(static_cast<int32_t>(tiles - t0 < ck ? tiles - t0 : ck));
        }
        q.chunk_end = static_cast<int>(cp[c].size());
        q.lbt[0] = q.lbt[1] = nullptr;
        q.lbj[0] = q.lbj[1] = nullptr;
        job_off += n[p];
    }
    bool ok = true;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (!ok) return;
        if (cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
    };
    alloc(reinterpret_cast<void **>(&b->probs), sizeof(ra::BatchProblem) * P);
    alloc(reinterpret_cast<void **>(&b->st), sizeof(ra::SolverState) * P);
    alloc(reinterpret_cast<void **>(&b->ev), sizeof(ra::EvalOut) * P);
    alloc(reinterpret_cast<void **>(&b->pingpong), sizeof(int32_t) * P);
    alloc(reinterpret_cast<void **>(&b->lag_on), sizeof(int32_t) * P);
    alloc(reinterpret_cast<void **>(&b->lam_off), sizeof(long long) * P);
    alloc(reinterpret_cast<void **>(&b->active), sizeof(int32_t) * 4);
    alloc(reinterpret_cast<void **>(&b->ticket), sizeof(unsigned) * P);
    alloc(reinterpret_cast<void **>(&b->status), sizeof(int) * 4);
    alloc(reinterpret_cast<void **>(&b->t0), sizeof(unsigned long long));
    alloc(reinterpret_cast<void **>(&b->info), sizeof(ra_solve_info) * P);
    alloc(reinterpret_cast<void **>(&b->secs), sizeof(double) * P);
    alloc(reinterpret_cast<void **>(&b->lam_tmp), sizeof(double) * b->m_total);
    alloc(reinterpret_cast<void **>(&b->feat_probs), sizeof(ra::FeatProblem) * P);
    alloc(reinterpret_cast<void **>(&b->feat_stats), sizeof(float) * RA_MLP_STATS * b->m_total);
    for (int k = 0; k < 2; ++k) {
        alloc(reinterpret_cast<void **>(&b->lbt_pool[k]), sizeof(float2) * total);
        alloc(reinterpret_cast<void **>(&b->lbj_pool[k]), sizeof(uchar2) * total);
    }
    for (int c = 0; c < 4; ++c) {
        b->nchunks[c] = static_cast<int>(cp[c].size());
        if (!b->nchunks[c]) continue;
        alloc(reinterpret_cast<void **>(&b->chunk_prob[c]), sizeof(int32_t) * b->nchunks[c]);
        alloc(reinterpret_cast<void **>(&b->chunk_tile0[c]), sizeof(int32_t) * b->nchunks[c]);
        alloc(reinterpret_cast<void **>(&b->chunk_ntiles[c]), sizeof(int32_t) * b->nchunks[c]);
        alloc(reinterpret_cast<void **>(&b->partials[c]), sizeof(double) * ra::kPartW * b->nchunks[c]);
    }
    if (!ok) {
        (void)cudaGetLastError();
        ra_batch_destroy(b);
        return fail(RA_ENOMEM, "batch workspace allocation (about %lld bytes of records) failed",
                    (long long)(20 * total));
    }
    job_off = 0;
    for (int p = 0; p < P; ++p) {
        for (int k = 0; k < 2; ++k) {
            probs[p].lbt[k] = b->lbt_pool[k] + job_off;
            probs[p].lbj[k] = b->lbj_pool[k] + job_off;
        }
        job_off += (n[p] + 7) & ~7LL;   // as in `total`
    }
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
        if (!b->nchunks[c]) continue;
        int per_sm = 0;
        e = ra::batch_configure(4 << c, !(flags & RA_NO_JOB_CAP), &per_sm);
        if (e != cudaSuccess) break;
        if (per_sm < 1) per_sm = 1;
        if (sh.ctas_per_sm > 0 && sh.ctas_per_sm < per_sm) per_sm = sh.ctas_per_sm;
        const long long g = static_cast<long long>(b->num_sms) * per_sm;
        b->grid[c] = static_cast<int>(g < b->nchunks[c] ? g : b->nchunks[c]);
        const long long gi = static_cast<long long>(b->num_sms) * 4;
        b->grid_init[c] = static_cast<int>(gi < b->nchunks[c] ? gi : b->nchunks[c]);
        e = cudaMemcpy(b->chunk_prob[c], cp[c].data(), sizeof(int32_t) * b->nchunks[c], cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->chunk_tile0[c], ct0[c].data(), sizeof(int32_t) * b->nchunks[c], cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->chunk_ntiles[c], cnt[c].data(), sizeof(int32_t) * b->nchunks[c], cudaMemcpyHostToDevice);
    }
    std::vector<ra::FeatProblem> fp(P);
    for (int p = 0; p < P; ++p) {
        fp[p] = ra::FeatProblem{A[p], kind[p], w[p], R[p], n[p], m[p], b->lam_off_h[p]};
        if (m[p] > b->m_max) b->m_max = m[p];
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->feat_probs, fp.data(), sizeof(ra::FeatProblem) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->probs, probs.data(), sizeof(ra::BatchProblem) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->lam_off, b->lam_off_h, sizeof(long long) * P, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->ticket, 0, sizeof(unsigned) * P);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(b->st, 0, sizeof(ra::SolverState) * P);
    if (e == cudaSuccess) e = cudaMemset(b->ev, 0, sizeof(ra::EvalOut) * P);
    if (e == cudaSuccess) e = cudaMemset(b->pingpong, 0, sizeof(int32_t) * P);
    if (e == cudaSuccess) e = cudaMemset(b->lag_on, 0, sizeof(int32_t) * P);
    if (e != cudaSuccess) {
        ra_batch_destroy(b);
        return fail(RA_ECUDA, "batch workspace init: %s", cudaGetErrorString(e));
    }
    *out = b;
    return RA_OK;
}

ra_status ra_batch_solve(ra_batch *b, const ra_solve_opts *opts, const double *lambda0,
                         double *lambda_out, ra_solve_info *infos, double *seconds)
{
    if (!b) return fail(RA_EINVAL, "NULL batch");
    return ra::batch_solve(b, opts, lambda0, lambda_out, infos, seconds);
}

int64_t ra_batch_prices(const ra_batch *b) { return b ? static_cast<int64_t>(b->m_total) : -1; }


// ---------------------------------------------------------------------------- warm start

namespace {

// Offsets in the problem's warm-start scratch.
constexpr size_t kWsStats = 0;                                   // 32 x 13 floats
constexpr size_t kWsFeats = 1792;                                // 32 x 26 floats
constexpr size_t kWsY = kWsFeats + sizeof(float) * RA_MAX_M * RA_MLP_IN;
constexpr size_t kWsLamW = kWsY + sizeof(float) * RA_MAX_M;
constexpr size_t kWsLamC = kWsLamW + sizeof(double) * RA_MAX_M;
constexpr size_t kWsUsed = kWsLamC + sizeof(double) * RA_MAX_M;
constexpr size_t kWsG2 = kWsUsed + 16;                           // 2 doubles
static_assert(kWsStats + sizeof(float) * RA_MAX_M * RA_MLP_STATS <= kWsFeats, "scratch layout");
static_assert(kWsG2 + 16 <= ra::kWarmBytes, "scratch layout");

ra::FeatProblem feat_of(const ra_problem *p)
{
    return ra::FeatProblem{p->A, p->kind, p->w, p->R, p->n, p->m, 0};
}

}  // namespace

ra_status ra_mlp_create(const float *theta, void *stream, ra_mlp **out)
{
    ra::g_err[0] = 0;
    if (!out) return fail(RA_EINVAL, "out is NULL");
    *out = nullptr;
    ra_mlp *net = new (std::nothrow) ra_mlp();
    if (!net) return fail(RA_ENOMEM, "host allocation failed");
    memset(net, 0, sizeof(*net));
    net->stream = static_cast<cudaStream_t>(stream);
    float *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, sizeof(float) * 4 * RA_MLP_PARAMS);
    if (e != cudaSuccess) {
        delete net;
        return fail(RA_ENOMEM, "parameter allocation: %s", cudaGetErrorString(e));
    }
    net->theta = buf;
    net->grad = buf + RA_MLP_PARAMS;
    net->m1 = buf + 2 * RA_MLP_PARAMS;
    net->m2 = buf + 3 * RA_MLP_PARAMS;
    e = cudaMemsetAsync(buf, 0, sizeof(float) * 4 * RA_MLP_PARAMS, net->stream);
    if (e == cudaSuccess && theta)
        e = cudaMemcpyAsync(net->theta, theta, sizeof(float) * RA_MLP_PARAMS, cudaMemcpyHostToDevice,
                            net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) {
        ra_mlp_destroy(net);
        return fail(RA_ECUDA, "parameter upload: %s", cudaGetErrorString(e));
    }
    *out = net;
    return RA_OK;
}

void ra_mlp_destroy(ra_mlp *net)
{
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    cudaFree(net->theta);
    cudaFree(net->act);
    delete net;
}

static ra_status mlp_copy(ra_mlp *net, float *host, const float *dev)
{
    cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(float) * RA_MLP_PARAMS, cudaMemcpyDeviceToHost,
                                    net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "parameter copy: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_mlp_get_params(ra_mlp *net, float *theta)
{
    if (!net || !theta) return fail(RA_EINVAL, "NULL argument");
    return mlp_copy(net, theta, net->theta);
}

ra_status ra_mlp_get_grads(ra_mlp *net, float *grad)
{
    if (!net || !grad) return fail(RA_EINVAL, "NULL argument");
    return mlp_copy(net, grad, net->grad);
}

ra_status ra_mlp_set_params(ra_mlp *net, const float *theta)
{
    if (!net || !theta) return fail(RA_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(net->theta, theta, sizeof(float) * RA_MLP_PARAMS,
                                    cudaMemcpyHostToDevice, net->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(net->grad, 0, sizeof(float) * 3 * RA_MLP_PARAMS, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "parameter upload: %s", cudaGetErrorString(e));
    net->t = 0;
    return RA_OK;
}

ra_status ra_mlp_forward(ra_mlp *net, const float *feats, int32_t rows, float *log_lambda)
{
    if (!net || !feats || !log_lambda) return fail(RA_EINVAL, "NULL argument");
    if (rows < 1) return fail(RA_EINVAL, "rows = %d must be >= 1", rows);
    cudaError_t e = ra::mlp_forward(net, feats, rows, log_lambda, net->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "MLP forward: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_mlp_train_step(ra_mlp *net, const float *feats, const float *target, int32_t rows,
                            float lr, float *loss)
{
    if (!net || !feats || !target) return fail(RA_EINVAL, "NULL argument");
    if (rows < 1) return fail(RA_EINVAL, "rows = %d must be >= 1", rows);
    if (!(lr > 0.0f)) return fail(RA_EINVAL, "lr must be > 0");
    cudaError_t e = ra::mlp_train_step(net, feats, target, rows, lr, loss, net->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "MLP training step: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_warmstart_features(ra_problem *p, float *feats)
{
    if (!p || !feats) return fail(RA_EINVAL, "NULL argument");
    cudaError_t e = ra::launch_features(nullptr, feat_of(p), 1, p->m,
                                        reinterpret_cast<float *>(p->warm + kWsStats), feats, p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "features launch: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_batch_features(ra_batch *b, float *feats)
{
    if (!b || !feats) return fail(RA_EINVAL, "NULL argument");
    ra::FeatProblem none{};
    cudaError_t e = ra::launch_features(b->feat_probs, none, b->P, b->m_max, b->feat_stats, feats,
                                        b->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "features launch: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_warmstart_used(ra_problem *p, int32_t *used_warm)
{
    if (!p || !used_warm) return fail(RA_EINVAL, "NULL argument");
    if (!p->side) return fail(RA_EINVAL, "no ra_warmstart_prices call on this problem");
    const int32_t *used = reinterpret_cast<const int32_t *>(p->warm + kWsUsed);
    cudaError_t e = cudaMemcpyAsync(used_warm, used, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return fail(RA_ECUDA, "warm-start flag: %s", cudaGetErrorString(e));
    return RA_OK;
}

ra_status ra_warmstart_prices(ra_problem *p, ra_mlp *net, double *lambda0, int32_t *used_warm)
{
    if (!p || !net || !lambda0) return fail(RA_EINVAL, "NULL argument");
    if (p->flags & RA_FP64_JOBMATH) return fail(RA_EINVAL, "the warm start uses the FP32 job math");
    p->pre_lam0 = nullptr;
    cudaStream_t s = p->stream;
    float *stats = reinterpret_cast<float *>(p->warm + kWsStats);
    float *feats = reinterpret_cast<float *>(p->warm + kWsFeats);
    float *y = reinterpret_cast<float *>(p->warm + kWsY);
    double *lam_w = reinterpret_cast<double *>(p->warm + kWsLamW);
    double *lam_c = reinterpret_cast<double *>(p->warm + kWsLamC);
    int32_t *used = reinterpret_cast<int32_t *>(p->warm + kWsUsed);
    // the statistics and the network run on a side stream while the cold
    // start's pass over A runs on the problem's stream (the two are
    // independent; the side stream is created on the first call)
    cudaError_t e = cudaSuccess;
    if (!p->side) {
        e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(RA_ECUDA, "warm-start stream: %s", cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(p->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaEventRecord(p->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->fork, 0);
    if (e == cudaSuccess) e = ra::launch_warm_network(feat_of(p), p->m, stats, net, feats, y, lam_w, p->side);
    if (e == cudaSuccess) e = cudaEventRecord(p->join, p->side);
    if (e == cudaSuccess) e = ra::launch_init(p, lam_c, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join, 0);
    if (e != cudaSuccess) return fail(RA_ECUDA, "warm-start launch: %s", cudaGetErrorString(e));
    // g at both candidates in one pass over the data, which is also the first
    // evaluation of a solve from the network's prices: when they are chosen,
    // ra_solve from lambda0 (called next on this problem) starts from it
    double *g2 = reinterpret_cast<double *>(p->warm + kWsG2);
    if (e == cudaSuccess) e = ra::launch_dual_g2(p, lam_w, lam_c, g2, true, s);
    if (e == cudaSuccess) e = ra::launch_choose(p->m, lam_w, lam_c, g2, lambda0, used, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->graph_flag + 4, used, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(RA_ECUDA, "warm-start evaluation: %s", cudaGetErrorString(e));
    p->pre_lam0 = lambda0;
    if (used_warm) {
        e = cudaMemcpyAsync(used_warm, used, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(RA_ECUDA, "warm-start flag: %s", cudaGetErrorString(e));
        return check_status_word(p);
    }
    return RA_OK;
}

}  // extern "C"
