// Feasible allocation at given prices with tie-aware repair.
//
// Section 3 of the paper recovers an allocation from optimal prices by
// solving every job's subproblem; where a subproblem has several optimal
// solutions (near ties of effective prices, of hull segments, or of the
// target throughput) any choice is optimal for the job, but only some
// mixtures of those choices meet the resource limits.  The paper is silent on
// which.  This file:
//
//   1. solves every job at lambda (Algorithm 1) and measures how close its
//      optimum is to a tie: the relative gap between the two best effective
//      prices (no per-job cap), the distance of the closest other cost-curve
//      point to the supporting line of the segment holding t* (with the cap),
//      and |w - alpha| / alpha for linear utilities;
//   2. picks the jobs closest to a tie (at most max_flex, margins below
//      tie_rel) from a histogram of the margins;
//   3. on the host, in FP64, lists each picked job's optimal extreme
//      allocations and solves a small LP for convex weights that maximise
//      their weighted utility minus the overuse sum_j max(r_j - R_j, 0)
//      priced at lambda_j -- about the utility that scaling the overuse away
//      would cost (ra_lp.cpp);
//   4. applies the column scaling of Section 5 to what is left of any
//      overuse (and, without the cap, scales under-used columns up), and
//      writes the allocation with its utility U -- a lower bound on U*.
//
// The per-job records of step 1 use the problem's lower-bound record buffers
// (the ones ra_eval_records reads).

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ra_kernels.cuh"
#include "ra_lp.h"

namespace ra {
namespace {

constexpr int kHistBins = 64;       // quarter decades of the tie margin from 1e-12 to 1e4
constexpr int kMaxFlex = 4096;      // jobs re-mixed at most
constexpr int kMaxAltPerJob = 8;
constexpr int kStatusOverflow = 2;  // a repaired job uses more than 4 resources

// Histogram bin of a tie margin; -1 = not near a tie (>= 1e4, or no second option).
__device__ __forceinline__ int tie_bin(float tau)
{
    if (!(tau < 1e4f)) return -1;
    if (tau < 1e-12f) return 0;
    const int b = static_cast<int>(floorf(4.0f * (log10f(tau) + 12.0f)));
    return b < 0 ? 0 : (b >= kHistBins ? kHistBins - 1 : b);
}

// Upper edge of bin b (host side, for reporting and for the tie_rel cut).
double bin_upper(int b) { return std::pow(10.0, -12.0 + 0.25 * (b + 1)); }

struct ScanArgs {
    const float *A;
    const uint8_t *kind;
    const float *w;
    const float *param;
    long long n;
    int m;
    const double *lam;
    float2 *rec_t;   // throughput from P and Q
    float2 *rec_x;   // time fractions on P and Q
    uchar2 *rec_j;   // columns P, Q (255 = none)
    float *tie;      // per-job tie margin
    int *hist;       // kHistBins counts
};

// Step 1: every job's optimum at lambda and its tie margin.
template <int MT, bool CAP, typename Real>
__global__ void __launch_bounds__(kTile) repair_scan_kernel(ScanArgs S)
{
    __shared__ Real lam_s[RA_MAX_M];
    __shared__ int h_s[kHistBins];
    const int tid = threadIdx.x;
    const int m = S.m;
    if (tid < kHistBins) h_s[tid] = 0;
    if (tid < RA_MAX_M) lam_s[tid] = tid < m ? static_cast<Real>(S.lam[tid]) : Fn<Real>::inf();
    __syncthreads();
    Real lam_r[MT], mu_r[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        lam_r[k] = lam_s[k];
        mu_r[k] = inv_price<Real>(lam_s[k]);
    }
    const Real tiny = Real(1e-30);
    for (long long i = static_cast<long long>(blockIdx.x) * kTile + tid; i < S.n;
         i += static_cast<long long>(gridDim.x) * kTile) {
        const float *row = S.A + i * m;
        Real a[MT];
#pragma unroll
        for (int k = 0; k < MT; ++k) a[k] = k < m ? static_cast<Real>(__ldg(&row[k])) : Real(0);
        const int kd = S.kind[i];
        const Real wi = S.w[i], pi = S.param[i];
        JobSol<Real> s;
        auto fetch = [&](int k, Real &av, Real &lv) {
            av = static_cast<Real>(__ldg(&row[k]));
            lv = lam_s[k];
        };
        solve_job<MT, CAP, true, Real>(a, lam_r, mu_r, 0, fetch, kd, wi, pi, s);
        S.rec_j[i] = make_uchar2(s.cP >= 0 ? s.cP : 255, s.cQ >= 0 ? s.cQ : 255);
        S.rec_t[i] = make_float2(static_cast<float>(s.tP), static_cast<float>(s.tQ));
        S.rec_x[i] = make_float2(static_cast<float>(s.xP), static_cast<float>(s.xQ));
        Real tau = Fn<Real>::inf();
        if (!CAP) {
            // relative gap of the two cheapest effective prices (best, second
            // are the two largest a_j / lambda_j)
            if (s.best > Real(0) && s.second > Real(0)) tau = s.best / s.second - Real(1);
            if (kd >= RA_U_LINCAP && s.jstar >= 0)
                tau = fmin(tau, fabs(wi - s.alpha) / fmax(s.alpha, tiny));
        } else if (s.segQ >= 0) {
            // distance of the closest other point (origin included) to the
            // supporting line of the segment holding t*
            const int P = s.segP, Q = s.segQ;
            const Real aP = P >= 0 ? static_cast<Real>(__ldg(&row[P])) : Real(0);
            const Real lP = P >= 0 ? lam_s[P] : Real(0);
            const Real al = s.alpha;
            Real d = Fn<Real>::inf(), al_left = -Fn<Real>::inf();
            for (int z = 0; z < m; ++z) {
                if (z == P || z == Q) continue;
                const Real az = static_cast<Real>(__ldg(&row[z]));
                if (!(az > Real(0))) continue;
                const Real lz = lam_s[z];
                const Real line = lP + al * (az - aP);
                d = fmin(d, (lz - line) / fmax(fmax(fabs(line), fabs(lz)), tiny));
                if (P >= 0 && az < aP) al_left = fmax(al_left, (lP - lz) / (aP - az));
            }
            if (P >= 0) {
                const Real line0 = lP - al * aP;
                d = fmin(d, -line0 / fmax(fabs(line0), tiny));
                al_left = fmax(al_left, lP / aP);
            }
            tau = fmax(d, Real(0));
            if (kd >= RA_U_LINCAP) {
                tau = fmin(tau, fabs(wi - al) / fmax(fabs(al), tiny));
                if (P >= 0) tau = fmin(tau, fabs(wi - al_left) / fmax(fabs(al_left), tiny));
            }
        }
        const float tf = static_cast<float>(tau);
        S.tie[i] = tf;
        const int b = tie_bin(tf);
        if (b >= 0) atomicAdd(&h_s[b], 1);
    }
    __syncthreads();
    if (tid < kHistBins && h_s[tid] != 0) atomicAdd(&S.hist[tid], h_s[tid]);
}

struct CollectArgs {
    const uint8_t *kind;
    const float2 *rec_x;
    const uchar2 *rec_j;
    const float *tie;
    long long n;
    int m;
    int bin_cut;          // jobs with tie_bin <= bin_cut are re-mixed
    int cap;              // list capacity
    int *count;
    long long *list;      // their indices (in no particular order)
    double *partials;
    unsigned *ticket;
    double *sums;         // 2m: usage of the other jobs, and of their linear-utility part
};

// Column sums of the warp's records in FP64: one butterfly per column that
// some lane uses (fixed order), lane c keeps column c.  The allocation the
// repair scales is the records' FP32 x in FP64; its usage must be summed
// without an FP32 stage, or the column factors leave it off R by the
// rounding of those partial sums.
__device__ __forceinline__ void warp_rsum_f64(int lane, int cP, double xP, int cQ, double xQ,
                                              bool lin, double &racc, double &rlin)
{
    unsigned cols = (cP >= 0 ? 1u << cP : 0u) | (cQ >= 0 ? 1u << cQ : 0u);
    cols = __reduce_or_sync(kFull, cols);
    while (cols) {
        const int c = __ffs(cols) - 1;
        cols &= cols - 1;
        double v = (cP == c ? xP : 0.0) + (cQ == c ? xQ : 0.0);
        double vl = lin ? v : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            v += __shfl_xor_sync(kFull, v, off);
            vl += __shfl_xor_sync(kFull, vl, off);
        }
        if (lane == c) {
            racc += v;
            rlin += vl;
        }
    }
}

// Step 2: list the jobs to re-mix; usage of all the others (fixed order).
template <bool CAP>
__global__ void __launch_bounds__(kTile) repair_collect_kernel(CollectArgs C)
{
    __shared__ double red[kWarps][kPartW];
    const int tid = threadIdx.x, lane = tid & 31;
    const int m = C.m;
    double racc = 0.0, rlin = 0.0;
    const long long stride = static_cast<long long>(gridDim.x) * kTile;
    const long long nround = (C.n + stride - 1) / stride;
    for (long long rr = 0; rr < nround; ++rr) {
        const long long i = rr * stride + static_cast<long long>(blockIdx.x) * kTile + tid;
        JobSol<float> s;
        s.cP = s.cQ = -1;
        s.xP = s.xQ = 0.f;
        bool lin = false;
        if (i < C.n) {
            const int b = tie_bin(C.tie[i]);
            if (b >= 0 && b <= C.bin_cut) {
                const int slot = atomicAdd(C.count, 1);
                if (slot < C.cap) C.list[slot] = i;
            } else {
                const uchar2 j = C.rec_j[i];
                const float2 x = C.rec_x[i];
                s.cP = j.x != 255 ? j.x : -1;
                s.xP = x.x;
                s.cQ = j.y != 255 ? j.y : -1;
                s.xQ = x.y;
                lin = C.kind[i] >= RA_U_LINCAP;
            }
        }
        warp_rsum_f64(lane, s.cP, s.xP, s.cQ, s.xQ, !CAP && lin, racc, rlin);
    }
    if (grid_reduce(0.0, 0.0, 0.0, racc, rlin, m, !CAP, true, C.partials, C.ticket, red) && tid < m) {
        C.sums[tid] = red[0][4 + tid];
        C.sums[m + tid] = CAP ? 0.0 : red[0][4 + m + tid];
    }
}

// The picked jobs' data for the host: m efficiencies, kind, w, param.
__global__ void repair_gather_kernel(const float *A, const uint8_t *kind, const float *w,
                                     const float *param, int m, const long long *idx, int F,
                                     float *out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < F; k += gridDim.x * blockDim.x) {
        const long long i = idx[k];
        float *o = out + static_cast<size_t>(k) * (m + 3);
        for (int j = 0; j < m; ++j) o[j] = A[i * m + j];
        o[m] = static_cast<float>(kind[i]);
        o[m + 1] = w[i];
        o[m + 2] = param[i];
    }
}

struct ApplyArgs {
    const float *A;
    const uint8_t *kind;
    const float *w;
    const float *param;
    const float2 *rec_t;
    const float2 *rec_x;
    const uchar2 *rec_j;
    const float *tie;
    long long n;
    int m;
    int bin_cut;
    const long long *flex_idx;  // sorted
    int F;
    const double *flex_x;       // F x m re-mixed allocations
    const double *flex_ax;      // F x m throughput a_ij x_ij of each entry
    const double *fac;          // 2m column factors: other jobs, linear-utility jobs
    int32_t *jk;                // 4n or NULL
    float *xk;                  // 4n or NULL
    float *X;                   // n m or NULL
    int *status;
    double *partials;
    unsigned *ticket;
    double *out;                // U, then usage[m] of the written allocation
};

// Step 4: the allocation (records, or the re-mixed rows for the picked jobs)
// times the column factors; its utility and usage.  The utility is that of
// the allocation x_ij f_j in FP64 (x the FP32 record, f the FP64 factor, the
// throughput recomputed as sum_j A_ij x_ij f_j), whose usage is f_j times the
// FP64 usage the factors were computed from: feasible to FP64 rounding, so
// the utility is a lower bound on U* at any tolerance.  The allocation written
// out (and its usage in out[1..m]) is that one rounded to FP32.
template <typename Real>
__global__ void __launch_bounds__(kTile) repair_apply_kernel(ApplyArgs Ap)
{
    __shared__ float rows[kTile * RA_MAX_M];
    __shared__ double red[kWarps][kPartW];
    __shared__ double fo[RA_MAX_M], fl[RA_MAX_M];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = Ap.m;
    if (tid < RA_MAX_M) {
        fo[tid] = tid < m ? Ap.fac[tid] : 1.0;
        fl[tid] = tid < m ? Ap.fac[m + tid] : 1.0;
    }
    __syncthreads();
    double uacc = 0.0, racc = 0.0;
    const long long stride = static_cast<long long>(gridDim.x) * kTile;
    const long long nround = (Ap.n + stride - 1) / stride;
    float *row = rows + tid * m;
    for (long long rr = 0; rr < nround; ++rr) {
        const long long i = rr * stride + static_cast<long long>(blockIdx.x) * kTile + tid;
        for (int j = 0; j < m; ++j) row[j] = 0.f;
        if (i < Ap.n) {
            const int kd = Ap.kind[i];
            const double *f = kd >= RA_U_LINCAP ? fl : fo;
            int jj[4] = {-1, -1, -1, -1};
            float xx[4] = {0.f, 0.f, 0.f, 0.f};
            int ne = 0;
            Real t = Real(0);
            const int b = tie_bin(Ap.tie[i]);
            int slot = -1;
            if (b >= 0 && b <= Ap.bin_cut) {
                int lo = 0, hi = Ap.F;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (Ap.flex_idx[mid] < i) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < Ap.F && Ap.flex_idx[lo] == i) slot = lo;
            }
            if (slot >= 0) {
                const double *fx = Ap.flex_x + static_cast<size_t>(slot) * m;
                const double *fa = Ap.flex_ax + static_cast<size_t>(slot) * m;
                for (int j = 0; j < m; ++j) {
                    if (fx[j] == 0.0) continue;
                    const float xo = static_cast<float>(fx[j] * f[j]);
                    row[j] = xo;
                    t += static_cast<Real>(fa[j] * f[j]);
                    if (ne < 4) {
                        jj[ne] = j;
                        xx[ne] = xo;
                    }
                    ++ne;
                }
            } else {
                const uchar2 jp = Ap.rec_j[i];
                const float2 xr = Ap.rec_x[i];
                const float *arow = Ap.A + i * m;
                if (jp.x != 255) {
                    const float xo = static_cast<float>(xr.x * f[jp.x]);
                    row[jp.x] = xo;
                    t += static_cast<Real>(static_cast<double>(arow[jp.x]) * xr.x * f[jp.x]);
                    jj[ne] = jp.x;
                    xx[ne] = xo;
                    ++ne;
                }
                if (jp.y != 255) {
                    const float xo = static_cast<float>(xr.y * f[jp.y]);
                    row[jp.y] = xo;
                    t += static_cast<Real>(static_cast<double>(arow[jp.y]) * xr.y * f[jp.y]);
                    jj[ne] = jp.y;
                    xx[ne] = xo;
                    ++ne;
                }
            }
            if (ne > 4) atomicOr(Ap.status, kStatusOverflow);
            uacc += static_cast<double>(util<Real>(kd, Ap.w[i], Ap.param[i], t));
            if (Ap.jk) {
                for (int e = 0; e < 4; ++e) {
                    Ap.jk[4 * i + e] = jj[e];
                    Ap.xk[4 * i + e] = xx[e];
                }
            }
            if (Ap.X)
                for (int j = 0; j < m; ++j) Ap.X[i * m + j] = row[j];
        }
        __syncwarp();
        warp_colsum<32, float, double>(rows + warp * 32 * m, m, lane, false, racc);
    }
    if (grid_reduce(uacc, 0.0, 0.0, racc, 0.0, m, false, true, Ap.partials, Ap.ticket, red)) {
        if (tid == 0) Ap.out[0] = red[0][0];
        if (tid < m) Ap.out[1 + tid] = red[0][4 + tid];
    }
}

template <int MT, bool CAP, typename Real>
cudaError_t launch_scan_t(const ScanArgs &a, int blocks, cudaStream_t s)
{
    repair_scan_kernel<MT, CAP, Real><<<blocks, kTile, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const ra_problem *p, const ScanArgs &a, int blocks, cudaStream_t s)
{
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    const bool f64 = (p->flags & RA_FP64_JOBMATH) != 0;
#define RA_SCAN(MT)                                                                                \
    if (f64) return cap ? launch_scan_t<MT, true, double>(a, blocks, s)                           \
                        : launch_scan_t<MT, false, double>(a, blocks, s);                         \
    return cap ? launch_scan_t<MT, true, float>(a, blocks, s) : launch_scan_t<MT, false, float>(a, blocks, s);
    switch (p->mt) {
    case 4: RA_SCAN(4)
    case 8: RA_SCAN(8)
    case 16: RA_SCAN(16)
    default: RA_SCAN(32)
    }
#undef RA_SCAN
}

// ---------------------------------------------------------------------------- host side

// u(t) in FP64 (Section 2.2).
double util_h(int kind, double w, double p, double t)
{
    switch (kind) {
    case RA_U_LOG: return w * std::log(t);
    case RA_U_POWER:
        if (!(t > 0.0)) return p > 0.0 ? 0.0 : -INFINITY;
        return p > 0.0 ? w * std::pow(t, p) : -w * std::pow(t, p);
    case RA_U_LINCAP: return w * std::fmin(t, p);
    default: return w * std::fmin(t - p, 0.0);
    }
}

struct Alt {
    double t, u, v;   // throughput, utility, net utility u - cost
    int j[2];         // resources (-1 = none)
    double x[2];      // their time fractions
};

// Optimal extreme allocations of one subproblem within a relative value
// tolerance: every segment of the cost curve through the points (0,0),
// (a_j, lambda_j) -- all pairs with the cap, the rays from the origin
// without it (Section 4.1) -- with the maximiser of u minus that segment
// (Eqs. e-opt-t-log, e-opt-t-target) and, where the linear utilities' slope
// ties w, both ends of the maximising interval.
void job_alternatives(int m, const double *a, const double *lam, int kind, double w, double par,
                      bool cap, double rel, std::vector<Alt> &out)
{
    out.clear();
    std::vector<Alt> cand;
    const double inf = INFINITY;
    for (int Q = 0; Q < m; ++Q) {
        if (!(a[Q] > 0.0)) continue;
        for (int P = -1; P < (cap ? m : 0); ++P) {
            const double aP = P < 0 ? 0.0 : a[P], lP = P < 0 ? 0.0 : lam[P];
            if (P >= 0 && !(aP > 0.0)) continue;
            if (!(aP < a[Q])) continue;
            const double al = (lam[Q] - lP) / (a[Q] - aP);
            const double be = lP - al * aP;
            const double hi = cap ? a[Q] : inf;
            double ts[2];
            int nt = 0;
            if (kind <= RA_U_POWER) {
                double t;
                if (!(al > 0.0)) t = hi;
                else t = kind == RA_U_LOG ? w / al : std::pow(w * std::fabs(par) / al, 1.0 / (1.0 - par));
                ts[nt++] = std::fmin(std::fmax(t, aP), hi);
            } else {
                const double T = std::fmin(std::fmax(par, aP), hi);
                if (w < al * (1.0 - rel)) ts[nt++] = aP;
                else if (w <= al * (1.0 + rel)) {
                    ts[nt++] = aP;
                    ts[nt++] = T;
                } else if (al < 0.0) ts[nt++] = hi;
                else ts[nt++] = T;
            }
            for (int k = 0; k < nt; ++k) {
                const double t = ts[k];
                if (!std::isfinite(t)) continue;
                Alt A;
                A.t = t;
                A.u = util_h(kind, w, par, t);
                A.v = A.u - (al * t + be);
                A.j[0] = A.j[1] = -1;
                A.x[0] = A.x[1] = 0.0;
                int e = 0;
                if (cap) {
                    const double xQ = (t - aP) / (a[Q] - aP), xP = (a[Q] - t) / (a[Q] - aP);
                    if (P >= 0 && xP > 0.0) {
                        A.j[e] = P;
                        A.x[e++] = xP;
                    }
                    if (xQ > 0.0) {
                        A.j[e] = Q;
                        A.x[e++] = xQ;
                    }
                } else if (t > 0.0) {
                    A.j[e] = Q;
                    A.x[e++] = t / a[Q];
                }
                if (std::isfinite(A.v)) cand.push_back(A);
            }
        }
    }
    if (cand.empty()) {
        Alt A{0.0, util_h(kind, w, par, 0.0), 0.0, {-1, -1}, {0.0, 0.0}};
        out.push_back(A);
        return;
    }
    std::stable_sort(cand.begin(), cand.end(), [](const Alt &x, const Alt &y) { return x.v > y.v; });
    const Alt &b = cand[0];
    const double scale = std::fabs(b.u) + std::fabs(b.u - b.v) + 1e-300;
    for (const Alt &A : cand) {
        if (A.v < b.v - rel * scale) break;
        bool dup = false;
        for (const Alt &B : out) {
            double d = 0.0;
            for (int j = 0; j < m && !dup; ++j) {
                const double xa = (A.j[0] == j ? A.x[0] : 0.0) + (A.j[1] == j ? A.x[1] : 0.0);
                const double xb = (B.j[0] == j ? B.x[0] : 0.0) + (B.j[1] == j ? B.x[1] : 0.0);
                d = std::fmax(d, std::fabs(xa - xb));
            }
            if (d <= 1e-13) dup = true;
        }
        if (!dup) out.push_back(A);
        if (static_cast<int>(out.size()) >= kMaxAltPerJob) break;
    }
}

struct Work {
    int cap_flex = 0;
    int m = 0;
    float *tie = nullptr;
    int *hist = nullptr;      // kHistBins + 1 (count)
    long long *list = nullptr;
    long long *flex_idx = nullptr;
    float *gather = nullptr;  // cap x (m + 3)
    double *flex_x = nullptr;
    double *flex_ax = nullptr;
    double *sums = nullptr;   // 2m
    double *fac = nullptr;    // 2m
    double *out = nullptr;    // 1 + m
};

ra_status ensure_work(ra_problem *p, Work **out)
{
    if (p->rep) {
        *out = static_cast<Work *>(p->rep);
        return RA_OK;
    }
    Work *W = new (std::nothrow) Work();
    if (!W) return fail(RA_ENOMEM, "host allocation failed");
    W->cap_flex = kMaxFlex;
    W->m = p->m;
    const int m = p->m;
    bool ok = true;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (ok && cudaMalloc(ptr, bytes) != cudaSuccess) ok = false;
    };
    alloc(reinterpret_cast<void **>(&W->tie), sizeof(float) * p->n);
    alloc(reinterpret_cast<void **>(&W->hist), sizeof(int) * (kHistBins + 1));
    alloc(reinterpret_cast<void **>(&W->list), sizeof(long long) * kMaxFlex);
    alloc(reinterpret_cast<void **>(&W->flex_idx), sizeof(long long) * kMaxFlex);
    alloc(reinterpret_cast<void **>(&W->gather), sizeof(float) * kMaxFlex * (m + 3));
    alloc(reinterpret_cast<void **>(&W->flex_x), sizeof(double) * kMaxFlex * m);
    alloc(reinterpret_cast<void **>(&W->flex_ax), sizeof(double) * kMaxFlex * m);
    alloc(reinterpret_cast<void **>(&W->sums), sizeof(double) * 2 * m);
    alloc(reinterpret_cast<void **>(&W->fac), sizeof(double) * 2 * m);
    alloc(reinterpret_cast<void **>(&W->out), sizeof(double) * (1 + m));
    p->rep = W;  // freed by release_repair_work, also on failure
    if (!ok) {
        (void)cudaGetLastError();
        return fail(RA_ENOMEM, "repair workspace (about %lld bytes) could not be allocated",
                    static_cast<long long>(4 * p->n));
    }
    *out = W;
    return RA_OK;
}

#define RA_CHECK(expr, what)                                                                       \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return fail(RA_ECUDA, "%s: %s", what, cudaGetErrorString(e_));     \
    } while (0)

}  // namespace

void release_repair_work(ra_problem *p)
{
    Work *W = static_cast<Work *>(p->rep);
    if (!W) return;
    cudaFree(W->tie);
    cudaFree(W->hist);
    cudaFree(W->list);
    cudaFree(W->flex_idx);
    cudaFree(W->gather);
    cudaFree(W->flex_x);
    cudaFree(W->flex_ax);
    cudaFree(W->sums);
    cudaFree(W->fac);
    cudaFree(W->out);
    delete W;
    p->rep = nullptr;
}

ra_status repair_allocation(ra_problem *p, const double *lam, const ra_repair_opts &o,
                            int32_t *jk, float *xk, float *X, ra_repair_info *info)
{
    Work *W = nullptr;
    ra_status st = ensure_work(p, &W);
    if (st != RA_OK) return st;
    const int m = p->m;
    const long long n = p->n;
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    cudaStream_t s = p->stream;
    long long blocks = (n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    const int nb = static_cast<int>(blocks);

    // 1. per-job optimum and tie margin
    RA_CHECK(cudaMemsetAsync(W->hist, 0, sizeof(int) * (kHistBins + 1), s), "repair reset");
    RA_CHECK(cudaMemsetAsync(p->status, 0, sizeof(int), s), "status reset");
    ScanArgs sa{p->A, p->kind, p->w, p->param, n, m, lam, p->lbt[0], p->lbt[1], p->lbj[0], W->tie,
                W->hist};
    RA_CHECK(launch_scan(p, sa, nb, s), "repair scan");
    int hist[kHistBins];
    RA_CHECK(cudaMemcpyAsync(hist, W->hist, sizeof(hist), cudaMemcpyDeviceToHost, s), "histogram");
    RA_CHECK(cudaStreamSynchronize(s), "repair scan");

    // 2. the jobs closest to a tie: whole bins, at most max_flex jobs, margins < tie_rel
    const int target = std::min(o.max_flex > 0 ? o.max_flex : 512, kMaxFlex);
    int bin_cut = -1, cum = 0;
    for (int b = 0; b < kHistBins; ++b) {
        if (bin_upper(b) > o.tie_rel * 1.0000001) break;
        if (cum + hist[b] > target) break;
        cum += hist[b];
        bin_cut = b;
    }
    int *d_count = W->hist + kHistBins;
    CollectArgs ca{p->kind, p->lbt[1], p->lbj[0], W->tie, n, m, bin_cut, W->cap_flex, d_count,
                   W->list, p->partials, p->ticket + 4, W->sums};
    if (cap) repair_collect_kernel<true><<<nb, kTile, 0, s>>>(ca);
    else repair_collect_kernel<false><<<nb, kTile, 0, s>>>(ca);
    RA_CHECK(cudaGetLastError(), "repair collect");
    int F = 0;
    std::vector<double> sums(2 * m), lam_h(m), R(m);
    RA_CHECK(cudaMemcpyAsync(&F, d_count, sizeof(int), cudaMemcpyDeviceToHost, s), "flex count");
    RA_CHECK(cudaMemcpyAsync(sums.data(), W->sums, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s), "usage");
    RA_CHECK(cudaMemcpyAsync(lam_h.data(), lam, sizeof(double) * m, cudaMemcpyDeviceToHost, s), "prices");
    RA_CHECK(cudaMemcpyAsync(R.data(), p->R, sizeof(double) * m, cudaMemcpyDeviceToHost, s), "limits");
    RA_CHECK(cudaStreamSynchronize(s), "repair collect");
    if (F > W->cap_flex) return fail(RA_ECUDA, "repair: %d jobs listed, capacity %d", F, W->cap_flex);
    std::vector<long long> idx(F);
    if (F > 0) {
        RA_CHECK(cudaMemcpy(idx.data(), W->list, sizeof(long long) * F, cudaMemcpyDeviceToHost), "flex list");
        std::sort(idx.begin(), idx.end());
        RA_CHECK(cudaMemcpyAsync(W->flex_idx, idx.data(), sizeof(long long) * F, cudaMemcpyHostToDevice, s),
                 "flex list");
        repair_gather_kernel<<<(F + 255) / 256, 256, 0, s>>>(p->A, p->kind, p->w, p->param, m,
                                                             W->flex_idx, F, W->gather);
        RA_CHECK(cudaGetLastError(), "repair gather");
    }
    std::vector<float> gat(static_cast<size_t>(F) * (m + 3));
    if (F > 0) {
        RA_CHECK(cudaMemcpyAsync(gat.data(), W->gather, sizeof(float) * gat.size(), cudaMemcpyDeviceToHost, s),
                 "flex data");
        RA_CHECK(cudaStreamSynchronize(s), "flex data");
    }

    // 3. alternatives and the LP (FP64, host)
    std::vector<std::vector<Alt>> alts(F);
    std::vector<int> kinds(F);
    std::vector<double> arow(static_cast<size_t>(F) * m);
    int n_alt = 0;
    for (int k = 0; k < F; ++k) {
        const float *g = &gat[static_cast<size_t>(k) * (m + 3)];
        for (int j = 0; j < m; ++j) arow[static_cast<size_t>(k) * m + j] = g[j];
        kinds[k] = static_cast<int>(g[m]);
        job_alternatives(m, &arow[static_cast<size_t>(k) * m], lam_h.data(), kinds[k], g[m + 1],
                         g[m + 2], cap, o.tie_rel, alts[k]);
        n_alt += static_cast<int>(alts[k].size());
    }
    auto xdense = [&](const Alt &A, int j) {
        return (A.j[0] == j ? A.x[0] : 0.0) + (A.j[1] == j ? A.x[1] : 0.0);
    };
    // base: alternative 0 of every job; variables theta_{k,e} (e >= 1) in [0, 1]
    std::vector<double> base(m, 0.0), base_lin(m, 0.0);
    for (int k = 0; k < F; ++k)
        for (int j = 0; j < m; ++j) {
            const double x = xdense(alts[k][0], j);
            base[j] += x;
            if (kinds[k] >= RA_U_LINCAP) base_lin[j] += x;
        }
    std::vector<int> vjob, valt;    // variable -> (job, alternative)
    std::vector<int> grow(F, -1);   // convexity row of a job with more than two alternatives
    int G = 0;
    for (int k = 0; k < F; ++k) {
        for (int e = 1; e < static_cast<int>(alts[k].size()); ++e) {
            vjob.push_back(k);
            valt.push_back(e);
        }
        if (alts[k].size() > 2) grow[k] = G++;
    }
    const int V = static_cast<int>(vjob.size());
    const int rows = m + G, cols = V + 2 * m + G;
    std::vector<double> theta(V, 0.0);
    int lp_status = -1;
    double lam_floor_w = 0.0;
    for (int j = 0; j < m; ++j) lam_floor_w = std::fmax(lam_floor_w, lam_h[j]);
    lam_floor_w *= 1e-6;
    double overuse = 0.0;
    if (V > 0) {
        std::vector<double> A(static_cast<size_t>(rows) * cols, 0.0), b(rows, 0.0), c(cols, 0.0),
            ub(cols, INFINITY);
        std::vector<int> basis(rows);
        for (int v = 0; v < V; ++v) {
            const Alt &A1 = alts[vjob[v]][valt[v]], &A0 = alts[vjob[v]][0];
            for (int j = 0; j < m; ++j) A[static_cast<size_t>(j) * cols + v] = xdense(A1, j) - xdense(A0, j);
            if (grow[vjob[v]] >= 0) A[static_cast<size_t>(m + grow[vjob[v]]) * cols + v] = 1.0;
            ub[v] = 1.0;
        }
        for (int j = 0; j < m; ++j) {
            A[static_cast<size_t>(j) * cols + V + j] = 1.0;       // s_j: capacity left
            A[static_cast<size_t>(j) * cols + V + m + j] = -1.0;  // v_j: overuse
            b[j] = R[j] - sums[j] - base[j];
            if (b[j] < 0.0) {
                for (int q = 0; q < cols; ++q) A[static_cast<size_t>(j) * cols + q] *= -1.0;
                b[j] = -b[j];
                basis[j] = V + m + j;
            } else {
                basis[j] = V + j;
            }
            // overuse costs its price: scaling a column down by v_j gives up
            // about lambda_j v_j of utility, so the LP trades overuse against
            // the alternatives' utility in one objective (Lagrangian weights)
            c[V + m + j] = std::fmax(lam_h[j], lam_floor_w);
        }
        for (int g = 0; g < G; ++g) {
            A[static_cast<size_t>(m + g) * cols + V + 2 * m + g] = 1.0;
            b[m + g] = 1.0;
            basis[m + g] = V + 2 * m + g;
        }
        for (int v = 0; v < V; ++v) c[v] = -(alts[vjob[v]][valt[v]].u - alts[vjob[v]][0].u);
        lp::Simplex S(rows, cols, A, b, c, ub, basis);
        lp::Result r = S.solve(20000);
        lp_status = static_cast<int>(r);
        if (r == lp::kOptimal || r == lp::kIterLimit) {
            std::vector<double> x = S.x();
            for (int v = 0; v < V; ++v) theta[v] = std::fmin(std::fmax(x[v], 0.0), 1.0);
            for (int j = 0; j < m; ++j) overuse += x[V + m + j] / std::fmax(R[j], 1e-300);
        }
    }

    // mixtures of the picked jobs, total usage and the column factors
    std::vector<double> fx(static_cast<size_t>(F) * m, 0.0), fax(static_cast<size_t>(F) * m, 0.0);
    std::vector<double> usage(m), usage_lin(m);
    for (int j = 0; j < m; ++j) {
        usage[j] = sums[j];
        usage_lin[j] = sums[m + j];
    }
    {
        std::vector<double> wsum(F, 0.0);
        std::vector<double> xr(static_cast<size_t>(F) * m, 0.0);
        for (int v = 0; v < V; ++v) {
            const Alt &A1 = alts[vjob[v]][valt[v]];
            wsum[vjob[v]] += theta[v];
            for (int e = 0; e < 2; ++e)
                if (A1.j[e] >= 0) xr[static_cast<size_t>(vjob[v]) * m + A1.j[e]] += theta[v] * A1.x[e];
        }
        for (int k = 0; k < F; ++k) {
            const double t0 = std::fmax(1.0 - wsum[k], 0.0);
            const Alt &A0 = alts[k][0];
            for (int e = 0; e < 2; ++e)
                if (A0.j[e] >= 0) xr[static_cast<size_t>(k) * m + A0.j[e]] += t0 * A0.x[e];
            for (int j = 0; j < m; ++j) {
                const double x = xr[static_cast<size_t>(k) * m + j];
                fx[static_cast<size_t>(k) * m + j] = x;
                fax[static_cast<size_t>(k) * m + j] = x * arow[static_cast<size_t>(k) * m + j];
                usage[j] += x;
                if (kinds[k] >= RA_U_LINCAP) usage_lin[j] += x;
            }
        }
    }
    std::vector<double> fac(2 * m);
    for (int j = 0; j < m; ++j) column_scales(R[j], usage[j], usage_lin[j], cap, fac[j], fac[m + j]);

    // 4. write the allocation; its utility and usage
    if (F > 0) {
        RA_CHECK(cudaMemcpyAsync(W->flex_x, fx.data(), sizeof(double) * fx.size(), cudaMemcpyHostToDevice, s), "flex rows");
        RA_CHECK(cudaMemcpyAsync(W->flex_ax, fax.data(), sizeof(double) * fax.size(), cudaMemcpyHostToDevice, s), "flex rows");
    }
    RA_CHECK(cudaMemcpyAsync(W->fac, fac.data(), sizeof(double) * 2 * m, cudaMemcpyHostToDevice, s), "factors");
    ApplyArgs ap{p->A, p->kind, p->w, p->param, p->lbt[0], p->lbt[1], p->lbj[0], W->tie, n, m, bin_cut,
                 W->flex_idx, F, W->flex_x, W->flex_ax, W->fac, jk, xk, X, p->status, p->partials,
                 p->ticket + 5, W->out};
    // the utility of the FP64 allocation in FP64 (a lower bound on U* to FP64
    // rounding, whichever per-job arithmetic the evaluations use)
    repair_apply_kernel<double><<<nb, kTile, 0, s>>>(ap);
    RA_CHECK(cudaGetLastError(), "repair apply");
    std::vector<double> res(1 + m);
    int kst = 0;
    RA_CHECK(cudaMemcpyAsync(res.data(), W->out, sizeof(double) * (1 + m), cudaMemcpyDeviceToHost, s), "repair result");
    RA_CHECK(cudaMemcpyAsync(&kst, p->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
    RA_CHECK(cudaStreamSynchronize(s), "repair apply");
    if (kst & kStatusOverflow) {
        if (jk || xk)
            return fail(RA_EINVAL, "a repaired job uses more than 4 resources: request the dense X");
    }
    if (info) {
        info->n_flex = F;
        info->n_alt = n_alt;
        info->lp_status = lp_status;
        info->tie_cut = bin_cut >= 0 ? bin_upper(bin_cut) : 0.0;
        info->overuse = overuse;
        info->U = res[0];
        double mu = 0.0;
        for (int j = 0; j < m; ++j) mu = std::fmax(mu, R[j] > 0.0 ? res[1 + j] / R[j] : (res[1 + j] > 0.0 ? INFINITY : 0.0));
        info->max_usage_over_R = mu;
    }
    return RA_OK;
}

}  // namespace ra
