/*
 * FP64 CPU oracle for the dual price-discovery method of
 * "Allocation of Fungible Resources via a Fast, Scalable Price Discovery
 * Method" (Agrawal, Boyd, Narayanan, Kazhamiaka, Zaharia, arXiv 2104.00282).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, call or
 * link this file: only the tests, the smoke check and the CPU baseline leg of
 * the benchmark use it.  It shares no code, header or constant with the CUDA
 * library; the two meet only in the seeded input arrays.
 *
 * Everything is plain double precision; FP32 inputs are promoted exactly.
 * Prices are called lam (the paper's p); the power exponent and the target /
 * cap throughput share the per-job field `par`.
 *
 * Utility kinds (Section 2.2):
 *   0 log     u(t) = w log t                  (Eq. e-log-util, with a weight)
 *   1 power   u(t) = w t^par, 0 < par < 1, or -w t^par, par < 0
 *             ("Power utilities"; alpha-fair with alpha = 1 - par)
 *   2 lincap  u(t) = w min(t, par)            (Eq. e-target-priority-util + w par)
 *   3 target  u(t) = w min(t - par, 0)        (Eq. e-target-priority-util)
 *
 * Per-job subproblem (Eq. e-subprob / e-subproblem):
 *   maximize u(t) - lam^T x  s.t. x >= 0, 1^T x <= 1 (cap mode), t = a^T x.
 * Without the per-job cap (cap = 0) the constraint 1^T x <= 1 is dropped.
 *
 * Two solvers of that subproblem are given:
 *   ora_job_pairs -- Algorithm 1 read literally (Section 4): every pair of
 *                    points (0,0), (a_j, lam_j) defines an affine cost on
 *                    [a_P, a_Q] (Eqs. e-xixj, e-optcostij); maximise u minus
 *                    each affine piece on its interval and keep the best.
 *                    This is the definition, O(m^2) per job.  Without the
 *                    cap the pieces are the rays from the origin through
 *                    each point, O(m) per job (job_rays).
 *   ora_job_hull  -- Section 4.1 kink-point form: build the lower convex hull
 *                    c(t) of the same points, then walk its segments left to
 *                    right applying Eq. e-opt-t-log / e-opt-t-target on each
 *                    until the constrained optimum is not the right end.
 *
 * Per-job output record (ORA_NOUT doubles):
 *   [0] t        optimal throughput t*
 *   [1] h        optimal net utility u(t*) - c(t*)
 *   [2] jstar    argmin_j lam_j / a_j (ties: larger a_j, then lower j); -1 if none
 *   [3] j1 [4] j2 resources used (-1 = none); x_{j1} = [5], x_{j2} = [6]
 *   [7] tie_ratio  relative gap between the best and second-best lam_j/a_j
 *   [8] tie_seg    relative distance of the closest other point to the
 *                  supporting line of the segment holding t* (0 = x ambiguous)
 *   [9] tie_t      for kinds 2/3: min over visited segments of |w-alpha|/alpha
 *                  (small = t* itself near a switch); +inf otherwise
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_NOUT 10
#define ORA_MAXM 256
#define ORA_BLOCK 4096 /* jobs per partial sum: fixed-order, thread-count independent */

enum { K_LOG = 0, K_POWER = 1, K_LINCAP = 2, K_TARGET = 3 };

int ora_version(void) { return 4; }

/* u(t), Section 2.2. */
static double util(int kind, double w, double par, double t)
{
    switch (kind) {
    case K_LOG:    return w * log(t);
    case K_POWER:  return par > 0.0 ? w * pow(t, par) : -w * pow(t, par);
    case K_LINCAP: return w * fmin(t, par);
    default:       return w * fmin(t - par, 0.0);
    }
}

/* A supergradient u'(t) (Eq. e-initialization allows a supergradient where u
 * is not differentiable; kinds 2/3 take w below the target and 0 from it on). */
static double util_deriv(int kind, double w, double par, double t)
{
    switch (kind) {
    case K_LOG:   return w / t;
    case K_POWER: return w * fabs(par) * pow(t, par - 1.0);
    default:      return t < par ? w : 0.0;
    }
}

/* Smallest maximiser of u(t) - alpha t over [lo, hi] (hi may be +inf).
 * Strictly concave kinds: t = Pi_[lo,hi] (u')^{-1}(alpha)   (Eq. e-opt-t-log),
 *   (u')^{-1}(alpha) = w/alpha for log, (w |par|/alpha)^{1/(1-par)} for power;
 *   alpha <= 0 makes the objective increasing, so t = hi.  For power utilities
 *   u'(t) = w |par| t^(par - 1), so (u')^{-1}(alpha) = (w |par| / alpha)^{1/(1-par)}.
 * Kinds 2/3: slope w - alpha below par and -alpha above it (Eq. e-opt-t-target):
 *   w <= alpha -> lo; otherwise par clamped to [lo, hi] (hi when alpha < 0). */
static double argmax_interval(int kind, double w, double par, double alpha, double lo, double hi)
{
    double t;
    if (kind == K_LOG || kind == K_POWER) {
        if (!(alpha > 0.0)) return hi;
        t = (kind == K_LOG) ? w / alpha : pow(w * fabs(par) / alpha, 1.0 / (1.0 - par));
    } else {
        if (w <= alpha) return lo;
        if (alpha < 0.0) return hi;
        t = par;
    }
    if (t < lo) t = lo;
    if (t > hi) t = hi;
    return t;
}

static void set_empty(double *o)
{
    for (int k = 0; k < ORA_NOUT; ++k) o[k] = 0.0;
    o[2] = o[3] = o[4] = -1.0;
    o[7] = o[8] = o[9] = INFINITY;
}

/* argmin_j lam_j/a_j over a_j > 0 (ties: larger a_j, then lower j) and the
 * relative gap to the runner-up (Section 4.1: the first cost segment leaves
 * the origin towards the point of highest a_j/lam_j). */
static int ratio_argmin(int m, const double *a, const double *lam, double *tie)
{
    int best = -1;
    double br = INFINITY, second = INFINITY;
    for (int j = 0; j < m; ++j) {
        if (!(a[j] > 0.0)) continue;
        double rj = lam[j] / a[j];
        int better = best < 0 || rj < br || (rj == br && (a[j] > a[best]));
        if (better) {
            if (best >= 0) second = br;
            best = j;
            br = rj;
        } else if (rj < second) {
            second = rj;
        }
    }
    if (best < 0) { *tie = INFINITY; return -1; }
    if (second == INFINITY) *tie = INFINITY;
    else if (br > 0.0) *tie = (second - br) / br;
    else *tie = (second > 0.0) ? INFINITY : 0.0;
    return best;
}

/* x on the pair (P, Q), a_P < a_Q, at throughput t (Eq. e-xixj); P = -1 is the
 * origin (a_0 = lam_0 = 0, slack). */
static void pair_alloc(int P, int Q, const double *a, double t, double *o)
{
    double aP = (P < 0) ? 0.0 : a[P];
    double xQ = (t - aP) / (a[Q] - aP);
    double xP = (a[Q] - t) / (a[Q] - aP);
    /* canonical form: only entries with x > 0, lower-a resource first */
    o[3] = o[4] = -1;
    o[5] = o[6] = 0.0;
    int k = 3;
    if (P >= 0 && xP > 0.0) { o[k] = P; o[k + 2] = xP; ++k; }
    if (xQ > 0.0) { o[k] = Q; o[k + 2] = xQ; }
}

/* Relative distance of the closest point other than P, Q (origin included
 * when P is not the origin) to the line of slope alpha through P. */
static double line_margin(int m, const double *a, const double *lam, int P, int Q, double alpha)
{
    double aP = (P < 0) ? 0.0 : a[P], lP = (P < 0) ? 0.0 : lam[P];
    double best = INFINITY;
    for (int z = -1; z < m; ++z) {
        if (z == P || z == Q) continue;
        if (z >= 0 && !(a[z] > 0.0)) continue;
        double az = (z < 0) ? 0.0 : a[z], lz = (z < 0) ? 0.0 : lam[z];
        double line = lP + alpha * (az - aP);
        double scale = fmax(fabs(line), fmax(fabs(lz), 1e-300));
        double d = (lz - line) / scale;
        if (d < best) best = d;
    }
    return best < 0.0 ? 0.0 : best;
}

/* Uncapped subproblem: c(t) = t min_j lam_j/a_j on [0, inf). */
static void job_nocap(int m, const double *a, const double *lam, int kind, double w,
                      double par, double *o)
{
    set_empty(o);
    double tie;
    int js = ratio_argmin(m, a, lam, &tie);
    o[7] = tie;
    if (js < 0) { o[0] = 0.0; o[1] = util(kind, w, par, 0.0); return; }
    double alpha = lam[js] / a[js];
    double t = argmax_interval(kind, w, par, alpha, 0.0, INFINITY);
    o[0] = t;
    /* a free resource (alpha = 0) leaves a strictly increasing utility's
     * demand unbounded: the supremum, and so g, is +inf (Section 3) */
    o[1] = isinf(t) ? INFINITY : util(kind, w, par, t) - alpha * t;
    o[2] = js;
    if (t > 0.0) { o[3] = js; o[5] = t / a[js]; }
    o[8] = tie;
    if (kind >= K_LINCAP) o[9] = fabs(w - alpha) / fmax(alpha, 1e-300);
}

/* Algorithm 1 without the per-job cap, read literally: with 1^T x <= 1
 * dropped, each point (a_j, lam_j) spans a ray t -> (t / a_j) lam_j from the
 * origin, and c(t) is their pointwise minimum; maximise u minus each ray over
 * t >= 0 and keep the best (larger value, then smaller t, then larger a_j,
 * then lower j).  An independent reading of the same subproblem as
 * job_nocap, which goes straight to the cheapest ray. */
static void job_rays(int m, const double *a, const double *lam, int kind, double w, double par,
                     double *o)
{
    set_empty(o);
    double tie;
    o[2] = ratio_argmin(m, a, lam, &tie);
    o[7] = tie;
    double best = -INFINITY, bt = 0.0, balpha = 0.0;
    int bj = -1;
    for (int j = 0; j < m; ++j) {
        if (!(a[j] > 0.0)) continue;
        double alpha = lam[j] / a[j];
        double t = argmax_interval(kind, w, par, alpha, 0.0, INFINITY);
        double v = isinf(t) ? INFINITY : util(kind, w, par, t) - alpha * t;
        int take = bj < 0 || v > best ||
                   (v == best && (t < bt || (t == bt && a[j] > a[bj])));
        if (take) { best = v; bt = t; bj = j; balpha = alpha; }
    }
    if (bj < 0) { o[0] = 0.0; o[1] = util(kind, w, par, 0.0); return; }
    o[0] = bt;
    o[1] = best;
    if (bt > 0.0) { o[3] = bj; o[5] = bt / a[bj]; }
    o[8] = tie;
    if (kind >= K_LINCAP) o[9] = fabs(w - balpha) / fmax(balpha, 1e-300);
}

/* Algorithm 1 read literally: maximise u minus every pairwise affine piece
 * over its interval (Section 4, "Parametric solution of the LP" and
 * "Solving the subproblem"); the best value over all pairs is
 * max_t u(t) - c(t) since c is their pointwise minimum. */
void ora_job_pairs(int m, const double *a, const double *lam, int kind, double w, double par,
                   int cap, double *o)
{
    if (!cap) { job_rays(m, a, lam, kind, w, par, o); return; }
    set_empty(o);
    double tie;
    o[2] = ratio_argmin(m, a, lam, &tie);
    o[7] = tie;
    double best = -INFINITY, bt = 0.0, balpha = 0.0;
    int bP = -2, bQ = -2;
    for (int Q = 0; Q < m; ++Q) {
        if (!(a[Q] > 0.0)) continue;
        for (int P = -1; P < m; ++P) {
            double aP = (P < 0) ? 0.0 : a[P], lP = (P < 0) ? 0.0 : lam[P];
            if (!(aP < a[Q])) continue;
            double alpha = (lam[Q] - lP) / (a[Q] - aP);
            double beta = lP - alpha * aP;
            double t = argmax_interval(kind, w, par, alpha, aP, a[Q]);
            double v = util(kind, w, par, t) - (alpha * t + beta);
            if (v > best || (v == best && t < bt)) {
                best = v; bt = t; bP = P; bQ = Q; balpha = alpha;
            }
        }
    }
    if (bQ < -1) { /* no resource with a_j > 0: x = 0 */
        o[0] = 0.0; o[1] = util(kind, w, par, 0.0); return;
    }
    o[0] = bt;
    o[1] = best;
    pair_alloc(bP, bQ, a, bt, o);
    if (bt <= 0.0) { o[3] = o[4] = -1; o[5] = o[6] = 0.0; }
    o[8] = line_margin(m, a, lam, bP, bQ, balpha);
}

/* Section 4.1 form: kink points of c(t) = lower convex hull of (0,0) and
 * (a_j, lam_j), then a left-to-right walk of its segments. */
void ora_job_hull(int m, const double *a, const double *lam, int kind, double w, double par,
                  int cap, double *o)
{
    if (!cap) { job_nocap(m, a, lam, kind, w, par, o); return; }
    set_empty(o);
    double tie;
    o[2] = ratio_argmin(m, a, lam, &tie);
    o[7] = tie;
    int idx[ORA_MAXM];
    int k = 0;
    for (int j = 0; j < m; ++j)
        if (a[j] > 0.0) idx[k++] = j;
    if (k == 0) { o[0] = 0.0; o[1] = util(kind, w, par, 0.0); return; }
    /* insertion sort by (a ascending, lam ascending, j ascending) */
    for (int i = 1; i < k; ++i) {
        int v = idx[i], q = i - 1;
        while (q >= 0 && (a[idx[q]] > a[v] || (a[idx[q]] == a[v] && lam[idx[q]] > lam[v]))) {
            idx[q + 1] = idx[q];
            --q;
        }
        idx[q + 1] = v;
    }
    /* lower hull from the origin; collinear middle points are dropped */
    int hull[ORA_MAXM + 1];
    int hn = 0;
    hull[hn++] = -1;
    for (int i = 0; i < k; ++i) {
        int z = idx[i];
        if (hn >= 1 && hull[hn - 1] >= 0 && a[hull[hn - 1]] == a[z]) continue; /* same a, higher lam */
        while (hn >= 2) {
            int A0 = hull[hn - 2], B0 = hull[hn - 1];
            double ax = (A0 < 0) ? 0.0 : a[A0], ay = (A0 < 0) ? 0.0 : lam[A0];
            double bx = a[B0], by = lam[B0];
            double cross = (bx - ax) * (lam[z] - ay) - (by - ay) * (a[z] - ax);
            if (cross <= 0.0) --hn; else break;
        }
        hull[hn++] = z;
    }
    double min_wa = INFINITY;
    for (int s = 0; s + 1 < hn; ++s) {
        int P = hull[s], Q = hull[s + 1];
        double aP = (P < 0) ? 0.0 : a[P], lP = (P < 0) ? 0.0 : lam[P];
        double alpha = (lam[Q] - lP) / (a[Q] - aP);
        double t = argmax_interval(kind, w, par, alpha, aP, a[Q]);
        if (kind >= K_LINCAP) {
            double mwa = fabs(w - alpha) / fmax(fabs(alpha), 1e-300);
            if (mwa < min_wa) min_wa = mwa;
        }
        if (t < a[Q] || s + 2 == hn) {
            o[0] = t;
            o[1] = util(kind, w, par, t) - (lP + alpha * (t - aP));
            pair_alloc(P, Q, a, t, o);
            if (t <= 0.0) { o[3] = o[4] = -1; o[5] = o[6] = 0.0; }
            o[8] = line_margin(m, a, lam, P, Q, alpha);
            o[9] = (kind >= K_LINCAP) ? min_wa : INFINITY;
            return;
        }
    }
}

/* c(t) of Section 4.1 and a minimising x (the LP
 *   minimize lam^T x  s.t. x >= 0, 1^T x <= 1, a^T x = t),
 * read off the lower convex hull; returns +inf outside [0, max_j a_j].
 * x_out receives m values. */
double ora_cost(int m, const double *a, const double *lam, double t, double *x_out)
{
    for (int j = 0; j < m; ++j) x_out[j] = 0.0;
    int idx[ORA_MAXM], k = 0;
    for (int j = 0; j < m; ++j)
        if (a[j] > 0.0) idx[k++] = j;
    if (t == 0.0) return 0.0;
    if (k == 0 || t < 0.0) return INFINITY;
    for (int i = 1; i < k; ++i) {
        int v = idx[i], q = i - 1;
        while (q >= 0 && (a[idx[q]] > a[v] || (a[idx[q]] == a[v] && lam[idx[q]] > lam[v]))) {
            idx[q + 1] = idx[q];
            --q;
        }
        idx[q + 1] = v;
    }
    int hull[ORA_MAXM + 1], hn = 0;
    hull[hn++] = -1;
    for (int i = 0; i < k; ++i) {
        int z = idx[i];
        if (hull[hn - 1] >= 0 && a[hull[hn - 1]] == a[z]) continue;
        while (hn >= 2) {
            int A0 = hull[hn - 2], B0 = hull[hn - 1];
            double ax = (A0 < 0) ? 0.0 : a[A0], ay = (A0 < 0) ? 0.0 : lam[A0];
            double cross = (a[B0] - ax) * (lam[z] - ay) - (lam[B0] - ay) * (a[z] - ax);
            if (cross <= 0.0) --hn; else break;
        }
        hull[hn++] = z;
    }
    for (int s = 0; s + 1 < hn; ++s) {
        int P = hull[s], Q = hull[s + 1];
        double aP = (P < 0) ? 0.0 : a[P], lP = (P < 0) ? 0.0 : lam[P];
        if (t <= a[Q]) {
            double xQ = (t - aP) / (a[Q] - aP), xP = (a[Q] - t) / (a[Q] - aP);
            x_out[Q] = xQ;
            if (P >= 0) x_out[P] = xP;
            return lP * xP + lam[Q] * xQ;
        }
    }
    return INFINITY;
}

static void load_row(int m, const float *A, int64_t i, double *a)
{
    for (int j = 0; j < m; ++j) a[j] = (double)A[i * (int64_t)m + j];
}

static void solve_job(int m, const double *a, const double *lam, int kind, double w, double par,
                      int cap, int method, double *o)
{
    if (method == 0) ora_job_hull(m, a, lam, kind, w, par, cap, o);
    else ora_job_pairs(m, a, lam, kind, w, par, cap, o);
}

static int nthreads_of(int want)
{
#ifdef _OPENMP
    return want > 0 ? want : omp_get_max_threads();
#else
    (void)want;
    return 1;
#endif
}

int ora_max_threads(void) { return nthreads_of(0); }

/* Dual function and subgradient (Section 3, "Evaluating the dual function",
 * Eq. e-g-subgrad read as q = R - sum_i x_i):
 *   g = lam^T R + sum_i h_i,  r = sum_i x_i,  U = sum_i u_i(t_i) (unscaled X).
 * Sums are formed per block of ORA_BLOCK jobs and then added in block order,
 * so the result does not depend on the thread count. */
/* Per-block sums of the dual evaluation: block b holds jobs [b ORA_BLOCK,
 * (b+1) ORA_BLOCK); part is nb x (2m + 2): sum h, sum u(t), r[m], r_lin[m]
 * (the usage of the linear-utility jobs). */
static void dual_blocks(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
                        const float *par, const double *lam, int cap, int method, double *part,
                        int nthreads);

int ora_dual_blocks(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
                    const float *par, const double *lam, int cap, int method, double *part,
                    int nthreads)
{
    if (m <= 0 || m > ORA_MAXM || n < 0) return 1;
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    memset(part, 0, sizeof(double) * (size_t)nb * (2 * m + 2));
    dual_blocks(n, m, A, kind, w, par, lam, cap, method, part, nthreads);
    return 0;
}

int ora_dual(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
             const float *par, const double *R, const double *lam, int cap, int method,
             double *g, double *r, double *U, double *r_lin, int nthreads)
{
    if (m <= 0 || m > ORA_MAXM || n < 0) return 1;
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    int W = 2 * m + 2;   /* h, U, r[m], r_lin[m] (usage of linear-utility jobs) */
    double *part = (double *)calloc((size_t)(nb > 0 ? nb : 1) * W, sizeof(double));
    if (!part) return 2;
    dual_blocks(n, m, A, kind, w, par, lam, cap, method, part, nthreads);
    double sh = 0.0, su = 0.0;
    for (int j = 0; j < m; ++j) r[j] = 0.0;
    if (r_lin)
        for (int j = 0; j < m; ++j) r_lin[j] = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        sh += part[b * W];
        su += part[b * W + 1];
        for (int j = 0; j < m; ++j) r[j] += part[b * W + 2 + j];
        if (r_lin)
            for (int j = 0; j < m; ++j) r_lin[j] += part[b * W + 2 + m + j];
    }
    double lr = 0.0;
    for (int j = 0; j < m; ++j) lr += lam[j] * R[j];
    *g = lr + sh;
    if (U) *U = su;
    free(part);
    return 0;
}

static void dual_blocks(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
                        const float *par, const double *lam, int cap, int method, double *part,
                        int nthreads)
{
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    int W = 2 * m + 2;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads))
    for (int64_t b = 0; b < nb; ++b) {
        double a[ORA_MAXM], o[ORA_NOUT];
        double *pb = part + b * W;
        int64_t i1 = (b + 1) * ORA_BLOCK < n ? (b + 1) * ORA_BLOCK : n;
        for (int64_t i = b * ORA_BLOCK; i < i1; ++i) {
            load_row(m, A, i, a);
            solve_job(m, a, lam, kind[i], w[i], par[i], cap, method, o);
            pb[0] += o[1];
            pb[1] += util(kind[i], w[i], par[i], o[0]);
            if (o[3] >= 0) pb[2 + (int)o[3]] += o[5];
            if (o[4] >= 0) pb[2 + (int)o[4]] += o[6];
            if (kind[i] >= 2) {
                if (o[3] >= 0) pb[2 + m + (int)o[3]] += o[5];
                if (o[4] >= 0) pb[2 + m + (int)o[4]] += o[6];
            }
        }
    }
}

/* Utility of the column-scaled allocation X~ at prices lam (Section 5: scale
 * each column of X^k so that the limit holds):
 *   U(X~) = sum_i u_i(sum_j a_ij x_ij s_ij),
 * s_ij = s_lin[j] for jobs with a linear utility (kinds 2, 3) and s[j]
 * otherwise (s_lin = NULL: s for every job). */
int ora_scaled_utility(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
                       const float *par, const double *lam, const double *s,
                       const double *s_lin, int cap, int method, double *U_lb, int nthreads)
{
    if (m <= 0 || m > ORA_MAXM || n < 0) return 1;
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    double *part = (double *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    if (!part) return 2;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads))
    for (int64_t b = 0; b < nb; ++b) {
        double a[ORA_MAXM], o[ORA_NOUT];
        int64_t i1 = (b + 1) * ORA_BLOCK < n ? (b + 1) * ORA_BLOCK : n;
        for (int64_t i = b * ORA_BLOCK; i < i1; ++i) {
            load_row(m, A, i, a);
            solve_job(m, a, lam, kind[i], w[i], par[i], cap, method, o);
            const double *sc = (s_lin && kind[i] >= 2) ? s_lin : s;
            double t = 0.0;
            if (o[3] >= 0) t += a[(int)o[3]] * o[5] * sc[(int)o[3]];
            if (o[4] >= 0) t += a[(int)o[4]] * o[6] * sc[(int)o[4]];
            part[b] += util(kind[i], w[i], par[i], t);
        }
    }
    double su = 0.0;
    for (int64_t b = 0; b < nb; ++b) su += part[b];
    *U_lb = su;
    free(part);
    return 0;
}

/* Initial prices (Section 5, "Initialization", Eq. e-initialization):
 *   x_i = R/n, divided by kappa = 1^T R / n when kappa > 1 (cap mode only),
 *   lam^1 = (1/n) sum_i u_i'(a_i^T x_i) a_i. */
int ora_init(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
             const float *par, const double *R, int cap, double *lam1, int nthreads)
{
    if (m <= 0 || m > ORA_MAXM || n <= 0) return 1;
    double x0[ORA_MAXM], kappa = 0.0;
    for (int j = 0; j < m; ++j) kappa += R[j] / (double)n;
    double div = (cap && kappa > 1.0) ? kappa : 1.0;
    for (int j = 0; j < m; ++j) x0[j] = R[j] / ((double)n * div);
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    double *part = (double *)calloc((size_t)nb * m, sizeof(double));
    if (!part) return 2;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads))
    for (int64_t b = 0; b < nb; ++b) {
        int64_t i1 = (b + 1) * ORA_BLOCK < n ? (b + 1) * ORA_BLOCK : n;
        for (int64_t i = b * ORA_BLOCK; i < i1; ++i) {
            double t = 0.0;
            for (int j = 0; j < m; ++j) t += (double)A[i * (int64_t)m + j] * x0[j];
            double d = util_deriv(kind[i], w[i], par[i], t);
            for (int j = 0; j < m; ++j) part[b * m + j] += d * (double)A[i * (int64_t)m + j];
        }
    }
    for (int j = 0; j < m; ++j) lam1[j] = 0.0;
    for (int64_t b = 0; b < nb; ++b)
        for (int j = 0; j < m; ++j) lam1[j] += part[b * m + j];
    for (int j = 0; j < m; ++j) lam1[j] /= (double)n;
    free(part);
    return 0;
}

/* Per-job records for the jobs listed in idx (all jobs when idx is NULL). */
int ora_jobs(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
             const float *par, const double *lam, int cap, int method, int64_t nidx,
             const int64_t *idx, double *out, int nthreads)
{
    if (m <= 0 || m > ORA_MAXM) return 1;
    int64_t cnt = idx ? nidx : n;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t k = 0; k < cnt; ++k) {
        double a[ORA_MAXM];
        int64_t i = idx ? idx[k] : k;
        load_row(m, A, i, a);
        solve_job(m, a, lam, kind[i], w[i], par[i], cap, method, out + k * ORA_NOUT);
    }
    return 0;
}

/* One subproblem from FP64 data (used by the worked-example pins). */
void ora_job(int m, const double *a, const double *lam, int kind, double w, double par, int cap,
             int method, double *out)
{
    solve_job(m, a, lam, kind, w, par, cap, method, out);
}

/* Utility of a convex combination of subproblem allocations (Section 5: any
 * mixture sum_k theta_k X(lam_k) with usage <= R is feasible, and since every
 * u_i is concave its utility is at least sum_k theta_k U(X(lam_k))):
 *   t_i = sum_k theta_k sum_j a_ij x_ij(lam_k) sc_k[j],   U = sum_i u_i(t_i),
 * where sc_k = sc_lin + k*m for jobs with a linear utility (kinds 2, 3) and
 * sc_oth + k*m otherwise (the column scalings applied to allocation k).
 * No dense allocation is formed: each job is solved at every lam_k.  Sums
 * per block of ORA_BLOCK jobs, added in block order. */
int ora_mixture_utility(int64_t n, int m, const float *A, const uint8_t *kind, const float *w,
                        const float *par, int K, const double *theta, const double *lams,
                        const double *sc_oth, const double *sc_lin, int cap, int method,
                        double *U_out, int nthreads)
{
    if (m <= 0 || m > ORA_MAXM || n < 0 || K <= 0) return 1;
    int64_t nb = (n + ORA_BLOCK - 1) / ORA_BLOCK;
    double *part = (double *)calloc((size_t)(nb > 0 ? nb : 1), sizeof(double));
    if (!part) return 2;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads))
    for (int64_t b = 0; b < nb; ++b) {
        double a[ORA_MAXM], o[ORA_NOUT];
        int64_t i1 = (b + 1) * ORA_BLOCK < n ? (b + 1) * ORA_BLOCK : n;
        for (int64_t i = b * ORA_BLOCK; i < i1; ++i) {
            load_row(m, A, i, a);
            double t = 0.0;
            for (int k = 0; k < K; ++k) {
                if (!(theta[k] > 0.0)) continue;
                solve_job(m, a, lams + (size_t)k * m, kind[i], w[i], par[i], cap, method, o);
                const double *sc = (kind[i] >= 2 ? sc_lin : sc_oth) + (size_t)k * m;
                double tk = 0.0;
                if (o[3] >= 0) tk += a[(int)o[3]] * o[5] * sc[(int)o[3]];
                if (o[4] >= 0) tk += a[(int)o[4]] * o[6] * sc[(int)o[4]];
                t += theta[k] * tk;
            }
            part[b] += util(kind[i], w[i], par[i], t);
        }
    }
    double su = 0.0;
    for (int64_t b = 0; b < nb; ++b) su += part[b];
    *U_out = su;
    free(part);
    return 0;
}
