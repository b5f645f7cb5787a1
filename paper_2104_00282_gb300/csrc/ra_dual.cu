// Fused dual evaluation for the price-discovery method (arXiv 2104.00282).
//
// One pass over the jobs computes, at prices lambda (Section 3):
//   g(lambda) = lambda^T R + sum_i h_i,   r = sum_i x_i,   U(X) = sum_i u_i(t_i),
// where (t_i, x_i, h_i) solve job i's subproblem (Eq. e-subprob) by the
// lower-hull walk of Section 4 (Algorithm 1): the first segment leaves the
// origin towards argmin_j lambda_j/A_ij; while the unconstrained optimum of
// u - c lies beyond the segment's right end, step to the next hull vertex
// (the minimum slope among points further right) and solve again with
// Eq. e-opt-t-log / e-opt-t-target.
//
// Layout and data movement (GB300): A is n x m FP32 row-major.  Each CTA owns
// 256-job tiles (one thread per job); a tile's rows (256*m*4 bytes), weights,
// parameters and kinds are contiguous, so one elected thread moves each with
// a 1-D bulk TMA copy (cp.async.bulk) into a multi-stage shared-memory ring
// completed on mbarriers.  Threads read their row with 128-bit shared loads
// in a per-thread rotated chunk order (conflict-free) against the prices and
// inverse prices in shared memory (broadcast reads), so the argmin and hull
// loops hold no per-job register array.  The per-resource sums r_j use the
// tile's own rows as a warp-private dense 32 x m scratch (each job writes its
// <= 2 nonzeros; transposed when m = 32), reduced in a fixed order.
// Compensated FP32 per-thread accumulators, a fixed-order float-float block
// stage and a last-block-done grid stage make every output bitwise
// deterministic for a given GPU.  The FP64 job-math kernel keeps FP64
// accumulators and stages.

#include <cstdio>

#include "ra_internal.cuh"

namespace ra {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kTile / 32;

// ---------------------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for completion of phase `parity`; gives up after limit_ns of device
// time (ra_set_wait_timeout; two seconds by default).  A zero limit gives up
// at once, without polling.
__device__ __noinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (limit_ns == 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 31 && globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

// Bound of the waits that let copies still in flight land before a CTA that
// gave up exits: independent of the caller's limit, since the copies are
// valid and complete within microseconds.
constexpr uint64_t kDrainNs = 2000000000ull;

// ---------------------------------------------------------------------------- utilities

template <typename Real> struct Fn;
template <> struct Fn<float> {
    static __device__ __forceinline__ float log(float x) { return logf(x); }
    static __device__ __forceinline__ float log2(float x) { return log2f(x); }
    static __device__ __forceinline__ float exp2(float x) { return exp2f(x); }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
};
template <> struct Fn<double> {
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double log2(double x) { return ::log2(x); }
    static __device__ __forceinline__ double exp2(double x) { return ::exp2(x); }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};

// mu = 1/lambda for the effective-price argmax (argmax_j a_j mu_j).  An exact
// zero price becomes a huge finite mu instead of +inf, so that zero-price
// resources still compare by efficiency: the lower hull then leaves the
// origin along lambda = 0 straight to the most efficient free resource (the
// farthest collinear point), and no two free resources tie at +inf.  In FP32
// prices below 1e-30 count as zero (their inverse would overflow).
template <typename Real> __device__ __forceinline__ Real inv_price(Real lam);
template <> __device__ __forceinline__ float inv_price<float>(float lam)
{
    return lam > 1e-30f ? 1.0f / lam : (lam >= 0.0f ? 5.192296858534828e33f /* 2^112 */ : 0.0f);
}
template <> __device__ __forceinline__ double inv_price<double>(double lam)
{
    return lam > 0.0 ? 1.0 / lam : (lam == 0.0 ? 0x1p960 : 0.0);
}

// u(t), Section 2.2.
template <typename Real>
__device__ __forceinline__ Real util(int kind, Real w, Real p, Real t)
{
    if (kind == RA_U_LOG) return w * Fn<Real>::log(t);
    if (kind == RA_U_POWER) return t > Real(0) ? w * Fn<Real>::exp2(p * Fn<Real>::log2(t)) : Real(0);
    if (kind == RA_U_LINCAP) return w * fmin(t, p);
    return w * fmin(t - p, Real(0));
}

// FP32: every kind is evaluated with one logarithm and one exponential
// (CUDA's fast intrinsics __logf/__expf, absolute error about 2^-21 in the
// logarithm) and the result selected by kind, so a warp holding mixed kinds
// does not serialise one code path per kind.
template <>
__device__ __forceinline__ float util<float>(int kind, float w, float p, float t)
{
    const float L = __logf(t);
    const float ul = w * L;
    const float up = t > 0.0f ? w * __expf(p * L) : 0.0f;
    const float uc = w * fminf(t, p);
    const float ut = w * fminf(t - p, 0.0f);
    return kind == RA_U_LOG ? ul : kind == RA_U_POWER ? up : kind == RA_U_LINCAP ? uc : ut;
}

// Smallest maximiser of u(t) - alpha t on [lo, hi]:
//   strictly concave kinds: Pi_[lo,hi] (u')^{-1}(alpha)        (Eq. e-opt-t-log)
//   piecewise-linear kinds: case analysis of Eq. e-opt-t-target.
template <typename Real>
__device__ __forceinline__ Real topt(int kind, Real w, Real p, Real alpha, Real lo, Real hi)
{
    Real t;
    if (kind <= RA_U_POWER) {
        if (!(alpha > Real(0))) return hi;
        if (kind == RA_U_LOG) t = w / alpha;
        else t = Fn<Real>::exp2(Fn<Real>::log2(w * p / alpha) / (Real(1) - p));
    } else {
        if (w <= alpha) return lo;
        if (alpha < Real(0)) return hi;
        t = p;
    }
    return fmin(fmax(t, lo), hi);
}

// FP32 variant of topt with the same selection structure: log w/alpha,
// power exp(log(w p / alpha) / (1 - p)), both through the fast intrinsics.
template <>
__device__ __forceinline__ float topt<float>(int kind, float w, float p, float alpha, float lo,
                                             float hi)
{
    const float tl = __fdividef(w, alpha);
    const float tp = __expf(__fdividef(__logf(__fdividef(w * p, alpha)), 1.0f - p));
    float t;
    if (kind <= RA_U_POWER) {
        if (!(alpha > 0.0f)) return hi;
        t = kind == RA_U_LOG ? tl : tp;
    } else {
        if (w <= alpha) return lo;
        if (alpha < 0.0f) return hi;
        t = p;
    }
    return fminf(fmaxf(t, lo), hi);
}

// Slot k of a per-thread register array holds column colof(k): rows are read
// in 16-byte chunks rotated by `rot` so that a warp's 128-bit shared loads hit
// distinct banks.  rot = 0 is the identity mapping.
template <int MT>
__device__ __forceinline__ int colof(int k, int rot)
{
    constexpr int C = MT / 4;
    return ((((k >> 2) + rot) & (C - 1)) << 2) | (k & 3);
}

template <typename Real>
struct JobSol {
    Real t, h;
    Real u;           // u(t): the job's utility at the optimum
    Real xP, xQ;      // time fractions on the segment ends (P may be the origin)
    Real tP, tQ;      // throughput delivered by P and by Q
    int cP, cQ;       // columns, -1 = none
    int jstar;        // argmin_j lambda_j / A_ij, -1 = none
    Real second;      // runner-up of a_j / lambda_j (near-tie detection)
    Real best;
};

// Algorithm 1 for one job.  a/lam/mu are register arrays in slot order
// (mu = 1/lam); fetch(k, &a, &lam) re-reads slot k's pair by column from
// memory so that no register array is indexed dynamically.
template <int MT, bool CAP, bool TIES, typename Real, class Fetch>
__device__ __forceinline__ void solve_job(const Real (&a)[MT], const Real (&lam)[MT],
                                          const Real (&mu)[MT], int rot, Fetch fetch, int kind,
                                          Real w, Real p, JobSol<Real> &s)
{
    // A1: cheapest effective price, argmax_j a_j / lambda_j, in four
    // independent chains (ILP); ties go to the lower column.
    Real bv[4] = {Real(0), Real(0), Real(0), Real(0)};
    int bk[4] = {-1, -1, -1, -1};
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        const Real v = a[k] * mu[k];
        if (v > bv[k & 3]) {
            bv[k & 3] = v;
            bk[k & 3] = k;
        }
    }
    Real vb = bv[0];
    int kb = bk[0];
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        const bool take = bv[c] > vb || (bv[c] == vb && bk[c] >= 0 &&
                                         (kb < 0 || colof<MT>(bk[c], rot) < colof<MT>(kb, rot)));
        if (take) {
            vb = bv[c];
            kb = bk[c];
        }
    }
    s.best = vb;
    s.second = Real(0);
    if (TIES) {
        Real sec = Real(0);
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            const Real v = a[k] * mu[k];
            if (k != kb && v > sec) sec = v;
        }
        s.second = sec;
    }
    s.cP = -1;
    s.xP = Real(0);
    s.tP = Real(0);
    if (kb < 0) {  // no usable resource
        s.jstar = -1;
        s.cQ = -1;
        s.t = Real(0);
        s.xQ = Real(0);
        s.tQ = Real(0);
        s.h = util<Real>(kind, w, p, Real(0));
        s.u = s.h;
        return;
    }
    Real aQ, lQ;
    fetch(kb, aQ, lQ);
    s.jstar = colof<MT>(kb, rot);
    int kQ = kb;
    Real aP = Real(0), lP = Real(0);
    int kP = -1;
    Real alpha = lQ / aQ;
    Real t;
    if (!CAP) {
        t = topt<Real>(kind, w, p, alpha, Real(0), Fn<Real>::inf());
    } else {
        // A3: walk the lower hull until the segment holds the optimum.
        for (int step = 0; step < MT; ++step) {
            t = topt<Real>(kind, w, p, alpha, aP, aQ);
            if (t < aQ) break;
            // next vertex: minimum slope (lam_k - lQ)/(a_k - aQ) over a_k > aQ,
            // compared division-free, in four independent chains
            Real cdl[4] = {Real(1), Real(1), Real(1), Real(1)};
            Real cda[4] = {Real(0), Real(0), Real(0), Real(0)};
            int ckn[4] = {-1, -1, -1, -1};
#pragma unroll
            for (int k = 0; k < MT; ++k) {
                const Real da = a[k] - aQ;
                const Real dl = lam[k] - lQ;
                if (da > Real(0) && dl * cda[k & 3] < cdl[k & 3] * da) {
                    cdl[k & 3] = dl;
                    cda[k & 3] = da;
                    ckn[k & 3] = k;
                }
            }
            Real bdl = cdl[0], bda = cda[0];
            int kn = ckn[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                if (ckn[c] < 0) continue;
                const Real lhs = cdl[c] * bda, rhs = bdl * cda[c];
                if (kn < 0 || lhs < rhs ||
                    (lhs == rhs && colof<MT>(ckn[c], rot) < colof<MT>(kn, rot))) {
                    bdl = cdl[c];
                    bda = cda[c];
                    kn = ckn[c];
                }
            }
            if (kn < 0) {  // aQ = max_j a_j: right end of the domain
                t = aQ;
                break;
            }
            kP = kQ;
            aP = aQ;
            lP = lQ;
            kQ = kn;
            fetch(kn, aQ, lQ);
            alpha = bdl / bda;
        }
    }
    s.t = t;
    const Real u = util<Real>(kind, w, p, t);
    s.u = u;
    s.h = u - (lP + alpha * (t - aP));
    if (!CAP && kind <= RA_U_POWER) {
        // interior optimum t = (u')^{-1}(alpha) on [0, inf): alpha t = w for
        // log and alpha t = p u(t) for power, so h = u(t) - alpha t is formed
        // without the cancellation of two huge terms (t overflows FP32 for
        // prices near zero; h is then +inf, never inf - inf).  Selects only:
        // u is evaluated once for every kind of a warp.
        s.h = !(alpha > Real(0)) ? Fn<Real>::inf() : kind == RA_U_LOG ? u - w : (Real(1) - p) * u;
    }
    Real xQ, xP;
    if (CAP) {
        const Real den = aQ - aP;
        xQ = (t - aP) / den;
        xP = (kP >= 0) ? (aQ - t) / den : Real(0);
    } else {
        xQ = t / aQ;
        xP = Real(0);
    }
    s.cQ = xQ > Real(0) ? colof<MT>(kQ, rot) : -1;
    s.xQ = xQ > Real(0) ? xQ : Real(0);
    s.tQ = s.xQ * aQ;
    if (kP >= 0 && xP > Real(0)) {
        s.cP = colof<MT>(kP, rot);
        s.xP = xP;
        s.tP = xP * aP;
    }
}

// Algorithm 1 in FP32 for a job whose m efficiencies are at `row` (shared or
// global memory; 16-byte aligned when grouped), prices and inverse prices in
// shared memory.  The cheapest effective price is found while streaming the
// row in 16-byte chunks (rotated by `rot` as in load_row) against the
// inverse prices; with the cap, each hull step streams the row and the prices
// again.  No per-job register array is held -- the register footprint that
// lets a third CTA share the SM.  Chains, their order, tie rules and the
// closed forms are those of solve_job<MT, CAP, false, float>, so both give
// the same bits.
template <int MT, bool CAP>
__device__ __forceinline__ void solve_job_sm(const float *row, const float *mu_s, const float *lam_s,
                                             int m, bool grouped, int rot, int kind, float w,
                                             float p, JobSol<float> &s)
{
    constexpr int C = MT / 4;
    float bv[4] = {0.f, 0.f, 0.f, 0.f};
    int bc[4] = {-1, -1, -1, -1};    // column of each chain's best
    if (grouped) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int q = (c + rot) & (C - 1);
            const float4 av = reinterpret_cast<const float4 *>(row)[q];
            const float4 mv = reinterpret_cast<const float4 *>(mu_s)[q];
            const float v0 = av.x * mv.x, v1 = av.y * mv.y, v2 = av.z * mv.z, v3 = av.w * mv.w;
            if (v0 > bv[0]) { bv[0] = v0; bc[0] = 4 * q; }
            if (v1 > bv[1]) { bv[1] = v1; bc[1] = 4 * q + 1; }
            if (v2 > bv[2]) { bv[2] = v2; bc[2] = 4 * q + 2; }
            if (v3 > bv[3]) { bv[3] = v3; bc[3] = 4 * q + 3; }
        }
    } else {
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            if (k < m) {
                const float v = row[k] * mu_s[k];
                if (v > bv[k & 3]) {
                    bv[k & 3] = v;
                    bc[k & 3] = k;
                }
            }
        }
    }
    float vb = bv[0];
    int cb = bc[0];
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        const bool take = bv[c] > vb || (bv[c] == vb && bc[c] >= 0 && (cb < 0 || bc[c] < cb));
        if (take) {
            vb = bv[c];
            cb = bc[c];
        }
    }
    s.best = vb;
    s.second = 0.f;
    s.cP = -1;
    s.xP = 0.f;
    s.tP = 0.f;
    if (cb < 0) {  // no usable resource
        s.jstar = -1;
        s.cQ = -1;
        s.t = 0.f;
        s.xQ = 0.f;
        s.tQ = 0.f;
        s.h = util<float>(kind, w, p, 0.f);
        s.u = s.h;
        return;
    }
    s.jstar = cb;
    int cQ = cb, cP = -1;
    float aQ = row[cb], lQ = lam_s[cb];
    float aP = 0.f, lP = 0.f;
    float alpha = lQ / aQ;
    float t;
    if (!CAP) {
        t = topt<float>(kind, w, p, alpha, 0.f, Fn<float>::inf());
    } else {
        // A3: walk the lower hull until the segment holds the optimum
        for (int step = 0; step < MT; ++step) {
            t = topt<float>(kind, w, p, alpha, aP, aQ);
            if (t < aQ) break;
            // next vertex: minimum slope (lam_k - lQ)/(a_k - aQ) over a_k > aQ,
            // compared division-free, in four independent chains
            float cdl[4] = {1.f, 1.f, 1.f, 1.f};
            float cda[4] = {0.f, 0.f, 0.f, 0.f};
            int ckn[4] = {-1, -1, -1, -1};
            auto consider = [&](int ch, float ak, float lk, int col) {
                const float da = ak - aQ, dl = lk - lQ;
                if (da > 0.f && dl * cda[ch] < cdl[ch] * da) {
                    cdl[ch] = dl;
                    cda[ch] = da;
                    ckn[ch] = col;
                }
            };
            if (grouped) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int q = (c + rot) & (C - 1);
                    const float4 av = reinterpret_cast<const float4 *>(row)[q];
                    const float4 lv = reinterpret_cast<const float4 *>(lam_s)[q];
                    consider(0, av.x, lv.x, 4 * q);
                    consider(1, av.y, lv.y, 4 * q + 1);
                    consider(2, av.z, lv.z, 4 * q + 2);
                    consider(3, av.w, lv.w, 4 * q + 3);
                }
            } else {
#pragma unroll
                for (int k = 0; k < MT; ++k)
                    if (k < m) consider(k & 3, row[k], lam_s[k], k);
            }
            float bdl = cdl[0], bda = cda[0];
            int kn = ckn[0];
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                if (ckn[c] < 0) continue;
                const float lhs = cdl[c] * bda, rhs = bdl * cda[c];
                if (kn < 0 || lhs < rhs || (lhs == rhs && ckn[c] < kn)) {
                    bdl = cdl[c];
                    bda = cda[c];
                    kn = ckn[c];
                }
            }
            if (kn < 0) {  // aQ = max_j a_j: right end of the domain
                t = aQ;
                break;
            }
            cP = cQ;
            aP = aQ;
            lP = lQ;
            cQ = kn;
            aQ = row[kn];
            lQ = lam_s[kn];
            alpha = bdl / bda;
        }
    }
    s.t = t;
    const float u = util<float>(kind, w, p, t);
    s.u = u;
    s.h = u - (lP + alpha * (t - aP));
    if (!CAP && kind <= RA_U_POWER)   // interior optimum: see solve_job
        s.h = !(alpha > 0.f) ? Fn<float>::inf() : kind == RA_U_LOG ? u - w : (1.f - p) * u;
    float xQ, xP;
    if (CAP) {
        const float den = aQ - aP;
        xQ = (t - aP) / den;
        xP = (cP >= 0) ? (aQ - t) / den : 0.f;
    } else {
        xQ = t / aQ;
        xP = 0.f;
    }
    s.cQ = xQ > 0.f ? cQ : -1;
    s.xQ = xQ > 0.f ? xQ : 0.f;
    s.tQ = s.xQ * aQ;
    if (cP >= 0 && xP > 0.f) {
        s.cP = cP;
        s.xP = xP;
        s.tP = xP * aP;
    }
}

// Per-thread running sums of the FP32 path: compensated FP32 (Kahan), error
// about 2^-23 of the sum of magnitudes however many terms, so the per-job
// adds stay off the FP64 pipe (a small fraction of the FP32 rate on this
// GPU); converted to FP64 once, before the block and grid stages.  An
// infinite term leaves the sum infinite (the compensation is dropped).
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = isfinite(t) ? (t - s) - y : 0.0f;
        s = t;
    }
    __device__ __forceinline__ double value() const
    {
        return static_cast<double>(s) - static_cast<double>(c);
    }
};
__device__ __forceinline__ void acc_add(double &a, double x) { a += x; }
__device__ __forceinline__ void acc_add(KahanF &a, float x) { a.add(x); }

template <int MT, typename Real, typename Acc>
__device__ __forceinline__ void warp_colsum(const Real *warp_rows, int m, int lane, bool grouped,
                                            Acc &racc);

// Column sums of the warp's 32 x 32 FP32 block when m = 32, transposed: lane
// l zeroes row l, writes its job's x into slot l of rows cQ and cP, and lane
// c sums row c (the column-c usage of the warp's 32 jobs) with eight 128-bit
// loads in rotated chunk order (four lanes per 16-byte bank group, the
// minimum for a 512-byte warp access) -- a quarter of the load instructions
// of a column walk.  Returns the four partial sums of lane `lane`'s row;
// with `lm` non-zero, cl gets the partial sums of the slots whose lane bit
// is set in lm.
template <bool LIN>
__device__ __forceinline__ void warp_rows_t32(float *warp_rows, int lane, int rot, int cP, float xP,
                                              int cQ, float xQ, unsigned lm, float (&cs)[4],
                                              float (&cl)[4])
{
    float *row = warp_rows + lane * 32;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        reinterpret_cast<float4 *>(row)[(c + rot) & 7] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    if (cP >= 0) warp_rows[cP * 32 + lane] = xP;
    if (cQ >= 0) warp_rows[cQ * 32 + lane] = xQ;
    __syncwarp();
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int q = (c + rot) & 7;
        const float4 v = reinterpret_cast<const float4 *>(row)[q];
        cs[0] += v.x;
        cs[1] += v.y;
        cs[2] += v.z;
        cs[3] += v.w;
        if (LIN) {
            const unsigned b = lm >> (4 * q);
            cl[0] += (b & 1u) ? v.x : 0.f;
            cl[1] += (b & 2u) ? v.y : 0.f;
            cl[2] += (b & 4u) ? v.z : 0.f;
            cl[3] += (b & 8u) ? v.w : 0.f;
        }
    }
    __syncwarp();
}

// Warp-cooperative r accumulation: each lane's `row` (m entries of shared
// memory that the lane alone owns) becomes its dense x_i; the 32 x m block is
// then summed column-wise in a fixed order.  `racc` of lane c (< m) gains the
// column-c sum.  `grouped` selects the lane-split column sum used when
// m == MT is a power of two >= 4 (and the transposed sum when m = 32).
template <int MT, typename Real, typename Acc>
__device__ __forceinline__ void warp_rsum(Real *warp_rows, int m, int lane, bool grouped,
                                          int rot, const JobSol<Real> &s, Acc &racc)
{
    Real *row = warp_rows + lane * m;
    if (MT == 32 && grouped && sizeof(Real) == 4) {
        float cs[4] = {0.f, 0.f, 0.f, 0.f}, cl[4];
        warp_rows_t32<false>(reinterpret_cast<float *>(warp_rows), lane, rot, s.cP,
                             static_cast<float>(s.xP), s.cQ, static_cast<float>(s.xQ), 0u, cs, cl);
        acc_add(racc, static_cast<Real>((cs[0] + cs[1]) + (cs[2] + cs[3])));
        return;
    }
    if (grouped && sizeof(Real) == 4) {
        constexpr int C = MT / 4;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int q = (c + rot) & (C - 1);
            reinterpret_cast<float4 *>(row)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int j = 0; j < m; ++j) row[j] = Real(0);
    }
    if (s.cP >= 0) row[s.cP] = s.xP;
    if (s.cQ >= 0) row[s.cQ] = s.xQ;
    __syncwarp();
    warp_colsum<MT, Real, Acc>(warp_rows, m, lane, grouped, racc);
}

// Column sums of a warp's 32 x m block of shared memory, in a fixed order with
// four independent partial sums; lane c (< m) adds column c's total to racc.
template <int MT, typename Real, typename Acc>
__device__ __forceinline__ void warp_colsum(const Real *warp_rows, int m, int lane, bool grouped,
                                            Acc &racc)
{
    if (grouped) {
        constexpr int G = 32 / MT;
        const int c = lane % MT, g = lane / MT;
        Real cs[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int k = 0; k < MT; ++k) cs[k & 3] += warp_rows[(g + k * G) * MT + c];
        Real t = (cs[0] + cs[1]) + (cs[2] + cs[3]);
#pragma unroll
        for (int off = MT; off < 32; off <<= 1) t += __shfl_xor_sync(kFull, t, off);
        if (g == 0) acc_add(racc, t);
    } else if (lane < m) {
        Real cs[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll 8
        for (int r = 0; r < 32; ++r) cs[r & 3] += warp_rows[r * m + lane];
        acc_add(racc, (cs[0] + cs[1]) + (cs[2] + cs[3]));
    }
    __syncwarp();
}

// warp_rsum that also sums the linear-utility jobs' part of each column
// (lanes flagged by `lin`): the same fixed-order column sums, with a second
// set of partial sums fed from the rows whose bit is set in the warp's lane
// mask -- no extra shared-memory traffic.  r is bitwise what warp_rsum gives.
template <int MT, typename Acc>
__device__ __forceinline__ void warp_rsum_lin(float *warp_rows, int m, int lane, bool grouped,
                                              int rot, const JobSol<float> &s, bool lin, Acc &racc,
                                              Acc &rlin)
{
    const unsigned lm = __ballot_sync(kFull, lin);
    if (MT == 32 && grouped) {
        float cs[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
        warp_rows_t32<true>(warp_rows, lane, rot, s.cP, s.xP, s.cQ, s.xQ, lm, cs, cl);
        acc_add(racc, (cs[0] + cs[1]) + (cs[2] + cs[3]));
        acc_add(rlin, (cl[0] + cl[1]) + (cl[2] + cl[3]));
        return;
    }
    float *row = warp_rows + lane * m;
    if (grouped) {
        constexpr int C = MT / 4;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int q = (c + rot) & (C - 1);
            reinterpret_cast<float4 *>(row)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int j = 0; j < m; ++j) row[j] = 0.f;
    }
    if (s.cP >= 0) row[s.cP] = s.xP;
    if (s.cQ >= 0) row[s.cQ] = s.xQ;
    __syncwarp();
    if (grouped) {
        constexpr int G = 32 / MT;
        const int c = lane % MT, g = lane / MT;
        float cs[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            const int r = g + k * G;
            const float v = warp_rows[r * MT + c];
            cs[k & 3] += v;
            cl[k & 3] += ((lm >> r) & 1u) ? v : 0.f;
        }
        float t = (cs[0] + cs[1]) + (cs[2] + cs[3]);
        float tl = (cl[0] + cl[1]) + (cl[2] + cl[3]);
#pragma unroll
        for (int off = MT; off < 32; off <<= 1) {
            t += __shfl_xor_sync(kFull, t, off);
            tl += __shfl_xor_sync(kFull, tl, off);
        }
        if (g == 0) {
            acc_add(racc, t);
            acc_add(rlin, tl);
        }
    } else if (lane < m) {
        float cs[4] = {0.f, 0.f, 0.f, 0.f}, cl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const float v = warp_rows[r * m + lane];
            cs[r & 3] += v;
            cl[r & 3] += ((lm >> r) & 1u) ? v : 0.f;
        }
        acc_add(racc, (cs[0] + cs[1]) + (cs[2] + cs[3]));
        acc_add(rlin, (cl[0] + cl[1]) + (cl[2] + cl[3]));
    }
    __syncwarp();
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Float-float: the unevaluated sum hi + lo of two FP32 numbers (about 44
// significant bits), the type of the block and grid stages of the FP32
// path's reductions.  FP64 arithmetic issues at a small fraction of the FP32
// rate on this GPU; the CTA that summed a grid's FP64 block partials took
// about 20 us, which the same sum in float-float arithmetic does not.
struct __align__(8) FF {
    float hi, lo;
};

// hi + lo of a + b: Knuth's two-sum of the high parts (its error term is
// exact and the same in either operand order, so the butterfly below leaves
// every lane with bitwise the same value), plus the low parts, renormalised.
// A non-finite sum is returned as (sum, 0).  Branch-free, so that loads
// after it in a loop are not held behind it.
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float hi = s + e;
    const float lo = e - (hi - s);
    const bool fin = isfinite(s);
    return FF{fin ? hi : s, fin ? lo : 0.0f};
}
__device__ __forceinline__ FF ff_of(const KahanF &k) { return FF{k.s, -k.c}; }

// Reduction-stage arithmetic on FP64 values (the FP64 job-math kernel) and
// on float-float values (the FP32 kernels).
__device__ __forceinline__ double red_add(double a, double b) { return a + b; }
__device__ __forceinline__ FF red_add(FF a, FF b) { return ff_add(a, b); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(FF a)
{
    return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}
__device__ __forceinline__ double ldcg_red(const double *p) { return __ldcg(p); }
__device__ __forceinline__ FF ldcg_red(const FF *p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return FF{v.x, v.y};
}
template <typename T> __device__ __forceinline__ T red_zero();
template <> __device__ __forceinline__ double red_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ FF red_zero<FF>() { return FF{0.0f, 0.0f}; }
__device__ __forceinline__ double warp_sum(double v) { return warp_sum_d(v); }
__device__ __forceinline__ FF warp_sum(FF v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        FF o;
        o.hi = __shfl_xor_sync(kFull, v.hi, off);
        o.lo = __shfl_xor_sync(kFull, v.lo, off);
        v = ff_add(v, o);
    }
    return v;
}
static_assert(sizeof(FF) == sizeof(double), "partial slots hold either type");

// Usage of the warp's linear-utility jobs per column (no-cap mode, where a
// job uses one column, cQ): one butterfly sum per distinct column among
// those lanes, taken in lane order; lane c adds column c's sum to acc.
template <typename Real, typename Acc>
__device__ __forceinline__ void warp_rlin(bool lin, int lane, const JobSol<Real> &s, Acc &acc)
{
    const bool on = lin && s.cQ >= 0;
    unsigned mask = __ballot_sync(kFull, on);
    while (mask) {
        const int c = __shfl_sync(kFull, s.cQ, __ffs(mask) - 1);
        const bool mine = on && s.cQ == c;
        Real v = mine ? s.xQ : Real(0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == c) acc_add(acc, v);
        mask &= ~__ballot_sync(kFull, mine);
    }
}

// Column sums of the first nv entries of G rows of kPartW FP64 partials, by
// the whole CTA: warp w adds rows w, w + kWarps, ... (lane l holds entries l,
// l + 32, l + 64; one row is a coalesced read), eight rows' loads in flight
// per trip, then the warps' sums are added in warp order -- a fixed order
// whatever the timing.  red[0][c] receives column c's total; red is
// overwritten, and every thread of the CTA must call this.
static_assert(kPartW <= 96, "three entries per lane");
template <typename T>
__device__ __forceinline__ void sum_partial_rows(const T *partials, unsigned G, int nv,
                                                 T (*red)[kPartW])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool h0 = lane < nv, h1 = lane + 32 < nv, h2 = lane + 64 < nv;
    const T zero = red_zero<T>();
    T a0 = zero, a1 = zero, a2 = zero;
    constexpr int U = 8;  // rows per warp whose loads are issued before any add
    for (unsigned b0 = warp; b0 < G; b0 += U * kWarps) {
        T v0[U], v1[U], v2[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned b = b0 + u * kWarps;
            const T *row = partials + static_cast<size_t>(b) * kPartW + lane;
            v0[u] = (b < G && h0) ? ldcg_red(row) : zero;
            v1[u] = (b < G && h1) ? ldcg_red(row + 32) : zero;
            v2[u] = (b < G && h2) ? ldcg_red(row + 64) : zero;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned b = b0 + u * kWarps;
            if (b < G) {
                a0 = red_add(a0, v0[u]);
                a1 = red_add(a1, v1[u]);
                a2 = red_add(a2, v2[u]);
            }
        }
    }
    __syncthreads();  // red's earlier contents have been read
    if (h0) red[warp][lane] = a0;
    if (h1) red[warp][lane + 32] = a1;
    if (h2) red[warp][lane + 64] = a2;
    __syncthreads();
    if (tid < nv) {
        T v = red[0][tid];
        for (int w = 1; w < kWarps; ++w) v = red_add(v, red[w][tid]);
        red[0][tid] = v;
    }
}

// Block stage + grid stage: per-thread FP64 values -> per-block partials
// (fixed warp order) -> the last CTA to finish sums the partials in block
// order.  Returns true in that CTA only, where red[0][0 .. m+4) then holds the
// totals (h, U(X), lagged U_lb, spare, r_0..r_{m-1}, then r_lin_0..r_lin_{m-1}
// when lin is set).  red is kWarps x kPartW.
template <typename T>
__device__ __noinline__ bool grid_reduce(T hsum, T uxsum, T lbsum, T racc, T rlin, int m, bool lin,
                            bool lane_owns_col, double *partial_slots, unsigned *ticket,
                            T (*red)[kPartW])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ int is_last;
    T *partials = reinterpret_cast<T *>(partial_slots);
    const int nv = lin ? 2 * m + 4 : m + 4;
    const T zero = red_zero<T>();
    __syncthreads();  // red may alias tile memory that other warps still read
    hsum = warp_sum(hsum);
    uxsum = warp_sum(uxsum);
    lbsum = warp_sum(lbsum);
    if (lane == 0) {
        red[warp][0] = hsum;
        red[warp][1] = uxsum;
        red[warp][2] = lbsum;
        red[warp][3] = zero;
    }
    if (lane < m) red[warp][4 + lane] = lane_owns_col ? racc : zero;
    if (lin && lane < m) red[warp][4 + m + lane] = rlin;
    __syncthreads();
    if (tid < nv) {
        T v = red[0][tid];
        for (int w = 1; w < kWarps; ++w) v = red_add(v, red[w][tid]);
        partials[static_cast<size_t>(blockIdx.x) * kPartW + tid] = v;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    sum_partial_rows(partials, gridDim.x, nv, red);
    if (tid == 0) *ticket = 0u;  // ready for the next launch
    __syncthreads();
    return true;
}

// The status word as the last CTA sees it after the grid stage's fences.
__device__ __forceinline__ int ld_status(const int *status) { return __ldcg(status); }
__device__ __forceinline__ double nan_d() { return __longlong_as_double(0x7ff8000000000000ll); }

// Dual outputs (Section 3): g = lambda^T R + sum h_i, q = R - r.
// lambda^T R, summed in column order by one thread.  The streaming kernels
// stage lambda and R in shared memory in their prologue and have a thread of
// warp 1 take the sum while the first tiles are in flight (the loop is a
// chain of dependent FP64 multiply-adds; from global memory under a full
// stream every step would also wait for a load).
__device__ __forceinline__ double lam_dot_R(const double *lam, const double *R, int m)
{
    double lr = 0.0;
    for (int j = 0; j < m; ++j) lr += lam[j] * R[j];
    return lr;
}

template <typename T>
__device__ void reduce_and_finalize(T hsum, T uxsum, T lbsum, T racc, T rlin, int m, bool lin,
                                    bool lane_owns_col, const DualParams &P, T (*red)[kPartW],
                                    const double *lr_s)
{
    if (!grid_reduce(hsum, uxsum, lbsum, racc, rlin, m, lin, lane_owns_col, P.partials, P.ticket,
                     red))
        return;
    const int tid = threadIdx.x;
    // a CTA whose bounded wait gave up left its jobs out of the sums: the
    // outputs become NaN, so that a caller who cannot read the status word
    // (ra_eval_dual_static) still sees that the evaluation is incomplete
    const bool bad = (ld_status(P.status) & kStatusTimeout) != 0;
    if (tid < m) {
        const double r = bad ? nan_d() : to_double(red[0][4 + tid]);
        P.out->r[tid] = r;
        P.out->q[tid] = P.R[tid] - r;
        P.out->r_lin[tid] = bad ? nan_d() : lin ? to_double(red[0][4 + m + tid]) : 0.0;
    }
    if (tid == 0) {
        const double sumh = bad ? nan_d() : to_double(red[0][0]);
        P.out->sumh = sumh;
        P.out->g = *lr_s + sumh;
        P.out->Ux = bad ? nan_d() : to_double(red[0][1]);
        P.out->Ulb_prev = bad ? nan_d() : to_double(red[0][2]);
    }
}

// ---------------------------------------------------------------------------- TMA kernel

template <int MT>
struct StageLayout {
    static __host__ __device__ size_t a_bytes(int m) { return static_cast<size_t>(kTile) * m * 4; }
    static __host__ __device__ size_t bytes(int m) { return a_bytes(m) + kTile * 9; }
};

// A stage of the single-problem streaming ring also has room for the tile's
// records of the previous evaluation (kTile float2 then kTile uchar2), which
// the solver's evaluation loads with the tile instead of per thread.
constexpr size_t kRecBytes = kTile * (sizeof(float2) + sizeof(uchar2));
constexpr int kRingSmemMax = 112 * 1024;  // dynamic allowance of the single-problem streaming kernels
__host__ __device__ inline size_t ring_stage_bytes(int m) { return StageLayout<4>::bytes(m) + kRecBytes; }

// The block stage's rows of the single-problem streaming kernels live in the
// tile ring, idle by then (one row of kPartW per warp).
__device__ __forceinline__ FF (*ring_red(unsigned char *smem))[kPartW]
{
    return reinterpret_cast<FF (*)[kPartW]>(smem);
}

// Per-job stream over this CTA's share of the jobs.  Full 256-job tiles come
// in through a ring of `stages` shared-memory buffers (ring_stage_bytes(m)
// apart) filled by 1-D bulk TMA copies (one elected thread issues A's rows,
// w, param and kind of a tile -- and, when rec_t is set, the tile's records
// rec_t / rec_j -- and arms the stage's mbarrier with the byte count); the
// ragged tail (n mod 256 jobs) is handled by one CTA, its rows staged in the
// idle stage 0.  For every job the callee receives job(i, valid, row, kind,
// w, p, warp_rows, rec): row points at the job's m efficiencies in shared
// memory, warp_rows at the 32 x m block of rows the calling warp owns (tile
// rows or idle stage-0 space), which the callee may overwrite once it has
// read its own row, and rec at the tile's staged records (NULL for the tail
// or without records).  All 256 threads call job for every tile, valid or
// not, so warp collectives work.  Returns false if a bounded wait gave up
// (the status word is then set).
struct NoPrologue {
    __device__ void operator()() const {}
};
template <int MT, class Job, class Pre = NoPrologue>
__device__ bool stream_jobs(const float *A, const float *W, const float *Par, const uint8_t *Kind,
                            const float2 *rec_t, const uchar2 *rec_j, long long n, int m,
                            int stages, long long num_full, unsigned char *smem, uint64_t *bars,
                            int *status, uint64_t wait_ns, Job &&job, Pre &&pre = Pre{})
{
    const int tid = threadIdx.x, warp = tid >> 5;
    const size_t a_bytes = StageLayout<MT>::a_bytes(m);
    const size_t core_bytes = StageLayout<MT>::bytes(m);
    const size_t st_bytes = ring_stage_bytes(m);
    const bool recs = rec_t != nullptr;
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const long long G = gridDim.x;
    const long long n_my = (num_full > blockIdx.x) ? (num_full - blockIdx.x + G - 1) / G : 0;
    auto issue = [&](long long it) {
        if (it >= n_my) return;
        const long long tile = blockIdx.x + it * G;
        const int st = static_cast<int>(it % stages);
        unsigned char *base = smem + st * st_bytes;
        const long long j0 = tile * kTile;
        mbar_arrive_expect_tx(&bars[st], static_cast<uint32_t>(core_bytes + (recs ? kRecBytes : 0)));
        bulk_load(base, A + j0 * m, static_cast<uint32_t>(a_bytes), &bars[st]);
        bulk_load(base + a_bytes, W + j0, kTile * 4, &bars[st]);
        bulk_load(base + a_bytes + kTile * 4, Par + j0, kTile * 4, &bars[st]);
        bulk_load(base + a_bytes + kTile * 8, Kind + j0, kTile, &bars[st]);
        if (recs) {
            bulk_load(base + core_bytes, rec_t + j0, kTile * sizeof(float2), &bars[st]);
            bulk_load(base + core_bytes + kTile * sizeof(float2), rec_j + j0, kTile * sizeof(uchar2),
                      &bars[st]);
        }
    };
    if (tid == 0)
        for (int s = 0; s < stages; ++s) issue(s);
    pre();  // while the first tiles are in flight (no barrier before the first tile's end)

    for (long long it = 0; it < n_my; ++it) {
        const int st = static_cast<int>(it % stages);
        const uint32_t parity = static_cast<uint32_t>((it / stages) & 1);
        const bool ok = mbar_wait_bounded(&bars[st], parity, wait_ns);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(status, kStatusTimeout);
                // let copies already in flight land before the CTA exits (bounded)
                for (long long it2 = it; it2 < n_my && it2 < it + stages; ++it2)
                    (void)mbar_wait_bounded(&bars[it2 % stages], static_cast<uint32_t>((it2 / stages) & 1),
                                            kDrainNs);
            }
            __syncthreads();
            return false;
        }
        unsigned char *base = smem + st * st_bytes;
        float *a_s = reinterpret_cast<float *>(base);
        const float *w_s = reinterpret_cast<const float *>(base + a_bytes);
        const float *p_s = reinterpret_cast<const float *>(base + a_bytes + kTile * 4);
        const uint8_t *k_s = base + a_bytes + kTile * 8;
        const long long i = (blockIdx.x + it * G) * kTile + tid;
        job(i, true, a_s + tid * m, static_cast<int>(k_s[tid]), w_s[tid], p_s[tid],
            a_s + warp * 32 * m, recs ? base + core_bytes : nullptr);
        __syncthreads();  // stage fully consumed
        if (tid == 0) {
            fence_proxy_async();
            issue(it + stages);
        }
    }
    // ragged tail: jobs [num_full * 256, n), one CTA, direct loads
    const long long tail0 = num_full * kTile;
    if (tail0 < n && blockIdx.x == static_cast<unsigned>(num_full % G)) {
        const long long i = tail0 + tid;
        const bool valid = i < n;
        float *scratch = reinterpret_cast<float *>(smem);  // stage 0 is idle now
        float *own = scratch + tid * m;                     // the tail's rows, staged like a tile
        for (int k = 0; k < m; ++k) own[k] = valid ? A[i * m + k] : 0.0f;
        __syncthreads();
        job(i, valid, own, valid ? static_cast<int>(Kind[i]) : RA_U_LINCAP,
            valid ? W[i] : 1.0f, valid ? Par[i] : 0.0f, scratch + warp * 32 * m,
            static_cast<const unsigned char *>(nullptr));
    }
    return true;
}

// Load job i's efficiencies into register slots (slot k = column colof(k, rot)).
template <int MT>
__device__ __forceinline__ void load_row(float (&a)[MT], const float *row, const float *A,
                                         long long i, bool valid, int m, bool grouped, int rot)
{
    constexpr int C = MT / 4;
    if (row != nullptr && grouped) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 v = reinterpret_cast<const float4 *>(row)[(c + rot) & (C - 1)];
            a[4 * c + 0] = v.x;
            a[4 * c + 1] = v.y;
            a[4 * c + 2] = v.z;
            a[4 * c + 3] = v.w;
        }
    } else if (row != nullptr) {
#pragma unroll
        for (int k = 0; k < MT; ++k) a[k] = k < m ? row[k] : 0.0f;
    } else {
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            const int c = colof<MT>(k, rot);
            a[k] = (valid && c < m) ? __ldg(&A[i * m + c]) : 0.0f;
        }
    }
}

template <int MT>
__device__ __forceinline__ unsigned char *align128(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) &
                                             ~static_cast<uintptr_t>(127));
}

// Main streaming kernel, FP32 per-job arithmetic (Sections 3 and 4).
template <int MT, bool CAP, bool LAG, bool REC>
__global__ void __launch_bounds__(kTile, CAP ? 2 : 3)
    dual_tma_kernel(DualParams P, int stages, long long num_full)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ __align__(16) float lam_s[RA_MAX_M];
    __shared__ __align__(16) float mu_s[RA_MAX_M];
    __shared__ float s_s[RA_MAX_M];
    __shared__ float sl_s[RA_MAX_M];
    __shared__ double lamd_s[RA_MAX_M], Rd_s[RA_MAX_M];
    __shared__ double lr_s;

    if (P.skip != nullptr && *P.skip != 0) return;

    const int tid = threadIdx.x, lane = tid & 31;
    const int m = P.m;
    const bool grouped = (m == MT);
    const float2 *lbt_prev = P.lbt_prev;
    const uchar2 *lbj_prev = P.lbj_prev;
    float2 *lbt_out = P.lbt_out;
    uchar2 *lbj_out = P.lbj_out;
    if (P.pingpong != nullptr) {
        const int q = *P.pingpong & 1;
        lbt_prev = P.lbt_buf[q];
        lbj_prev = P.lbj_buf[q];
        lbt_out = P.lbt_buf[q ^ 1];
        lbj_out = P.lbj_buf[q ^ 1];
    }
    const bool lag = LAG && (P.lag_on == nullptr || *P.lag_on != 0);
    constexpr int C = MT / 4;
    const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;

    if (tid < RA_MAX_M) {
        lamd_s[tid] = tid < m ? P.lam[tid] : 0.0;
        Rd_s[tid] = tid < m ? P.R[tid] : 0.0;
        lam_s[tid] = tid < m ? static_cast<float>(lamd_s[tid]) : Fn<float>::inf();
        mu_s[tid] = inv_price<float>(lam_s[tid]);
        s_s[tid] = (LAG && lag && tid < m) ? static_cast<float>(P.s_prev[tid]) : 1.0f;
        sl_s[tid] = (LAG && lag && tid < m)
                        ? static_cast<float>((P.s_lin_prev ? P.s_lin_prev : P.s_prev)[tid])
                        : 1.0f;
    }
    __syncthreads();

    KahanF hsum, uxsum, lbsum, racc, rlin;
    auto job = [&](long long i, bool valid, const float *row, int kind, float w, float p,
                   float *warp_rows, const unsigned char *rec) {
        // the previous evaluation's record: staged with the tile, or (ragged
        // tail) read first so that its latency overlaps this job's solve
        float2 tp = make_float2(0.f, 0.f);
        uchar2 jp = make_uchar2(255, 255);
        if (LAG && lag && valid) {
            if (rec != nullptr) {
                tp = reinterpret_cast<const float2 *>(rec)[tid];
                jp = reinterpret_cast<const uchar2 *>(rec + kTile * sizeof(float2))[tid];
            } else {
                tp = lbt_prev[i];
                jp = lbj_prev[i];
            }
        }
        JobSol<float> s;
        s.cP = s.cQ = -1;
        s.xP = s.xQ = 0.f;
        if (valid) {
            solve_job_sm<MT, CAP>(row, mu_s, lam_s, m, grouped, rot, kind, w, p, s);
            hsum.add(s.h);
            uxsum.add(s.u);
            if (LAG && lag) {
                const float *sc = kind >= RA_U_LINCAP ? sl_s : s_s;
                float tt = 0.f;
                if (jp.x != 255) tt += sc[jp.x] * tp.x;
                if (jp.y != 255) tt += sc[jp.y] * tp.y;
                lbsum.add(util<float>(kind, w, p, tt));
            }
            if (REC) {
                lbt_out[i] = make_float2(s.tP, s.tQ);
                lbj_out[i] = make_uchar2(s.cP >= 0 ? s.cP : 255, s.cQ >= 0 ? s.cQ : 255);
            }
        }
        if (!CAP && REC)
            warp_rsum_lin<MT, KahanF>(warp_rows, m, lane, grouped, rot, s,
                                      valid && kind >= RA_U_LINCAP, racc, rlin);
        else
            warp_rsum<MT, float, KahanF>(warp_rows, m, lane, grouped, rot, s, racc);
    };
    unsigned char *smem = align128<MT>(smem_dyn);
    stream_jobs<MT>(P.A, P.w, P.param, P.kind, (LAG && lag) ? lbt_prev : nullptr,
                    (LAG && lag) ? lbj_prev : nullptr, P.n, m, stages, num_full, smem, bars,
                    P.status, P.wait_ns, job, [&] {
                        if (tid == 32) lr_s = lam_dot_R(lamd_s, Rd_s, m);
                    });
    reduce_and_finalize(ff_of(hsum), ff_of(uxsum), ff_of(lbsum), ff_of(racc), ff_of(rlin), m,
                        !CAP && REC, grouped ? (lane / MT == 0) : true, P, ring_red(smem), &lr_s);
}

// Initial prices, Eq. e-initialization:
//   lambda^1 = (1/n) sum_i u_i'(a_i^T x0) a_i,  x0 = R / (kappa n),
// streamed through the same TMA ring: each job scales its own row in shared
// memory by d_i = u_i'(a_i^T x0) and the warp sums the rows column-wise.
template <int MT>
__global__ void __launch_bounds__(kTile, 2)
    init_tma_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                    const double *R, long long n, int m, int cap, int stages, long long num_full,
                    double *partials, unsigned *ticket, int *status, uint64_t wait_ns, double *lam1)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ float x0_s[RA_MAX_M];
    const int tid = threadIdx.x, lane = tid & 31;
    const bool grouped = (m == MT);
    constexpr int C = MT / 4;
    const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
    if (tid == 0) {
        double kappa = 0.0;
        for (int j = 0; j < m; ++j) kappa += R[j] / static_cast<double>(n);
        const double div = (cap && kappa > 1.0) ? kappa : 1.0;
        for (int j = 0; j < RA_MAX_M; ++j)
            x0_s[j] = j < m ? static_cast<float>(R[j] / (static_cast<double>(n) * div)) : 0.0f;
    }
    __syncthreads();
    float x0_r[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) x0_r[k] = x0_s[colof<MT>(k, rot)];
    KahanF racc;
    auto job = [&](long long i, bool valid, const float *row, int kd, float wi, float pi,
                   float *warp_rows, const unsigned char *) {
        float a[MT];
        load_row<MT>(a, row, A, i, valid, m, grouped, rot);
        float tc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < MT; ++k) tc[k & 3] = fmaf(a[k], x0_r[k], tc[k & 3]);
        const float t = (tc[0] + tc[1]) + (tc[2] + tc[3]);
        float d = 0.0f;
        if (valid) {
            if (kd == RA_U_LOG) d = wi / t;
            else if (kd == RA_U_POWER) d = wi * pi * exp2f((pi - 1.0f) * log2f(t));
            else d = t < pi ? wi : 0.0f;  // supergradient of w min(t, T) (+ const)
        }
        // own row <- d * a, in column order, then warp column sums
        float *own = warp_rows + lane * m;
        if (grouped) {
#pragma unroll
            for (int c = 0; c < C; ++c)
                reinterpret_cast<float4 *>(own)[(c + rot) & (C - 1)] =
                    make_float4(d * a[4 * c], d * a[4 * c + 1], d * a[4 * c + 2], d * a[4 * c + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < MT; ++k)
                if (k < m) own[colof<MT>(k, rot)] = d * a[k];
        }
        __syncwarp();
        warp_colsum<MT, float, KahanF>(warp_rows, m, lane, grouped, racc);
    };
    unsigned char *smem = align128<MT>(smem_dyn);
    stream_jobs<MT>(A, w, param, kind, nullptr, nullptr, n, m, stages, num_full, smem, bars, status,
                    wait_ns, job);
    const FF z = red_zero<FF>();
    FF(*red)[kPartW] = ring_red(smem);
    if (grid_reduce(z, z, z, ff_of(racc), z, m, false, grouped ? (lane / MT == 0) : true, partials,
                    ticket, red)) {
        // a CTA whose wait gave up left its share out of the sums: no prices
        const bool bad = (ld_status(status) & kStatusTimeout) != 0;
        if (tid < m) lam1[tid] = bad ? nan_d() : to_double(red[0][4 + tid]) / static_cast<double>(n);
    }
}

// Dual values g(lambda_a) and g(lambda_b) in one pass over the data (the
// two start points a warm start chooses between): each job is solved at both
// price vectors from the same staged row; only the two sums of h are
// reduced.  g_out[0], g_out[1] receive lambda^T R + sum_i h_i for each.
template <int MT, bool CAP>
__global__ void __launch_bounds__(kTile, CAP ? 2 : 3)
    dual_g2_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                   const double *R, long long n, int m, const double *lam_a, const double *lam_b,
                   int stages, long long num_full, double *partials, unsigned *ticket, int *status,
                   uint64_t wait_ns, double *g_out)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ __align__(16) float la_s[RA_MAX_M], ma_s[RA_MAX_M], lb_s[RA_MAX_M], mb_s[RA_MAX_M];
    __shared__ double lr_s[2];
    __shared__ double lad_s[RA_MAX_M], lbd_s[RA_MAX_M], Rd_s[RA_MAX_M];
    const int tid = threadIdx.x;
    const bool grouped = (m == MT);
    constexpr int C = MT / 4;
    const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
    if (tid < RA_MAX_M) {
        la_s[tid] = tid < m ? static_cast<float>(lam_a[tid]) : Fn<float>::inf();
        lb_s[tid] = tid < m ? static_cast<float>(lam_b[tid]) : Fn<float>::inf();
        lad_s[tid] = tid < m ? lam_a[tid] : 0.0;
        lbd_s[tid] = tid < m ? lam_b[tid] : 0.0;
        Rd_s[tid] = tid < m ? R[tid] : 0.0;
        ma_s[tid] = inv_price<float>(la_s[tid]);
        mb_s[tid] = inv_price<float>(lb_s[tid]);
    }
    __syncthreads();
    KahanF ha, hb;
    auto job = [&](long long i, bool valid, const float *row, int kd, float wi, float pi,
                   float *warp_rows, const unsigned char *) {
        (void)i;
        (void)warp_rows;
        if (!valid) return;
        JobSol<float> sa, sb;
        solve_job_sm<MT, CAP>(row, ma_s, la_s, m, grouped, rot, kd, wi, pi, sa);
        solve_job_sm<MT, CAP>(row, mb_s, lb_s, m, grouped, rot, kd, wi, pi, sb);
        ha.add(sa.h);
        hb.add(sb.h);
    };
    unsigned char *smem = align128<MT>(smem_dyn);
    stream_jobs<MT>(A, w, param, kind, nullptr, nullptr, n, m, stages, num_full, smem, bars, status,
                    wait_ns, job, [&] {
                        if (tid == 32) {
                            lr_s[0] = lam_dot_R(lad_s, Rd_s, m);
                            lr_s[1] = lam_dot_R(lbd_s, Rd_s, m);
                        }
                    });
    const FF z = red_zero<FF>();
    FF(*red)[kPartW] = ring_red(smem);
    if (grid_reduce(ff_of(ha), ff_of(hb), z, z, z, 0, false, true, partials, ticket, red) &&
        tid == 0) {
        const bool bad = (ld_status(status) & kStatusTimeout) != 0;
        g_out[0] = bad ? nan_d() : lr_s[0] + to_double(red[0][0]);
        g_out[1] = bad ? nan_d() : lr_s[1] + to_double(red[0][1]);
    }
}

// ---------------------------------------------------------------------------- batched kernels

// Column sums of a warp's x block without shared memory: column c is summed
// by a butterfly over the lanes' (at most two) nonzeros and lane c adds it.
template <typename Real, typename Acc>
__device__ __forceinline__ void warp_rsum_shfl(int m, int lane, const JobSol<Real> &s, Acc &racc)
{
    for (int c = 0; c < m; ++c) {
        float v = (s.cP == c ? static_cast<float>(s.xP) : 0.f) + (s.cQ == c ? static_cast<float>(s.xQ) : 0.f);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == c) acc_add(racc, v);
    }
}

// Sequence of tiles of this CTA in a batched evaluation: chunks blockIdx.x,
// blockIdx.x + G, ... of the class's chunk list, each a run of up to
// kChunkTiles tiles of one problem; chunks of problems already converged
// are skipped.  The producer (TMA issuer) and the consumers walk the same
// sequence with separate cursors.
struct TileCursor {
    long long c;     // chunk index (>= nchunks: end)
    int k;           // tile within the chunk
};

__device__ __forceinline__ bool chunk_live(const BatchDualArgs &B, long long c)
{
    return B.st[B.chunk_prob[c]].done == 0;
}

__device__ __forceinline__ void cursor_first(const BatchDualArgs &B, TileCursor &cur)
{
    cur.c = blockIdx.x;
    cur.k = 0;
    while (cur.c < B.nchunks && !chunk_live(B, cur.c)) cur.c += gridDim.x;
}

__device__ __forceinline__ void cursor_next(const BatchDualArgs &B, TileCursor &cur)
{
    if (++cur.k < B.chunk_ntiles[cur.c]) return;
    cur.k = 0;
    do {
        cur.c += gridDim.x;
    } while (cur.c < B.nchunks && !chunk_live(B, cur.c));
}

__device__ __forceinline__ bool tile_full(const BatchDualArgs &B, const TileCursor &cur)
{
    const BatchProblem &P = B.probs[B.chunk_prob[cur.c]];
    const long long t = B.chunk_tile0[cur.c] + cur.k;
    return (t + 1) * kTile <= P.n;
}

// Batched dual evaluation for every live problem of one width class.  Per
// tile the work is exactly that of dual_tma_kernel (TMA ring for full tiles,
// direct loads for a problem's ragged last tile); prices are reloaded at each
// chunk start, and each chunk's sums go to its own FP64 partial slot.  The
// last chunk of a problem to finish (per-problem ticket) adds that problem's
// partials in chunk order and writes its EvalOut, so the results equal a
// deterministic single-problem evaluation up to the order of additions.
template <int MT, bool CAP>
__global__ void __launch_bounds__(kTile, CAP ? 2 : 3) batch_dual_kernel(BatchDualArgs B)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ __align__(16) float lam_s[RA_MAX_M];
    __shared__ __align__(16) float mu_s[RA_MAX_M];
    __shared__ float s_s[RA_MAX_M];
    __shared__ float sl_s[RA_MAX_M];
    __shared__ FF red[kWarps][kPartW];
    __shared__ int is_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int C = MT / 4;
    const int stages = B.stages;
    unsigned char *smem = align128<MT>(smem_dyn);
    if (tid == 0) {
        for (int s2 = 0; s2 < stages; ++s2) mbar_init(&bars[s2], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // producer: issue the next full tile of the sequence into its stage
    TileCursor prod;
    long long issued = 0;
    if (tid == 0) cursor_first(B, prod);
    auto issue_next = [&]() {
        while (prod.c < B.nchunks && !tile_full(B, prod)) cursor_next(B, prod);
        if (prod.c >= B.nchunks) return;
        const BatchProblem &P = B.probs[B.chunk_prob[prod.c]];
        const int m = P.m;
        const long long j0 = static_cast<long long>(B.chunk_tile0[prod.c] + prod.k) * kTile;
        const size_t a_bytes = static_cast<size_t>(kTile) * m * 4;
        const size_t st_bytes = a_bytes + kTile * 9;
        const int st = static_cast<int>(issued % stages);
        unsigned char *base = smem + st * StageLayout<MT>::bytes(MT);
        mbar_arrive_expect_tx(&bars[st], static_cast<uint32_t>(st_bytes));
        bulk_load(base, P.A + j0 * m, static_cast<uint32_t>(a_bytes), &bars[st]);
        bulk_load(base + a_bytes, P.w + j0, kTile * 4, &bars[st]);
        bulk_load(base + a_bytes + kTile * 4, P.param + j0, kTile * 4, &bars[st]);
        bulk_load(base + a_bytes + kTile * 8, P.kind + j0, kTile, &bars[st]);
        ++issued;
        cursor_next(B, prod);
    };
    if (tid == 0)
        for (int s2 = 0; s2 < stages; ++s2) issue_next();

    TileCursor cur;
    cursor_first(B, cur);
    long long consumed = 0;
    KahanF hsum, uxsum, lbsum, racc, rlin;
    const int nv_lin = CAP ? 0 : 1;
    while (cur.c < B.nchunks) {
        const int p = B.chunk_prob[cur.c];
        const BatchProblem &P = B.probs[p];
        const int m = P.m;
        const bool grouped = (m == MT);
        const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
        const int pp = B.pingpong[p] & 1;
        const bool lag = B.lag_on[p] != 0;
        const float2 *lbt_prev = P.lbt[pp];
        const uchar2 *lbj_prev = P.lbj[pp];
        float2 *lbt_out = P.lbt[pp ^ 1];
        uchar2 *lbj_out = P.lbj[pp ^ 1];
        if (cur.k == 0) {  // chunk start: this problem's prices
            __syncthreads();
            if (tid < RA_MAX_M) {
                lam_s[tid] = tid < m ? static_cast<float>(B.st[p].lam_trial[tid]) : Fn<float>::inf();
                mu_s[tid] = inv_price<float>(lam_s[tid]);
                s_s[tid] = (lag && tid < m) ? static_cast<float>(B.st[p].s_lag[tid]) : 1.0f;
                sl_s[tid] = (lag && tid < m) ? static_cast<float>(B.st[p].s_lin_lag[tid]) : 1.0f;
            }
            __syncthreads();
            hsum = uxsum = lbsum = racc = rlin = KahanF{};
        }
        const long long t = B.chunk_tile0[cur.c] + cur.k;
        const bool full = (t + 1) * kTile <= P.n;
        const long long i = t * kTile + tid;
        const bool valid = i < P.n;
        const float *row = nullptr;
        float *warp_rows;
        int kind = RA_U_LINCAP;
        float w = 1.0f, pr = 0.0f;
        int st = 0;
        if (full) {
            st = static_cast<int>(consumed % stages);
            const bool ok = mbar_wait_bounded(&bars[st], static_cast<uint32_t>((consumed / stages) & 1),
                                              B.wait_ns);
            if (__syncthreads_or(!ok)) {
                // a copy never completed: record it, let the copies still in
                // flight land (bounded) and give up
                if (tid == 0) {
                    atomicOr(B.status, kStatusTimeout);
                    for (long long it2 = consumed; it2 < issued; ++it2)
                        (void)mbar_wait_bounded(&bars[it2 % stages], static_cast<uint32_t>((it2 / stages) & 1),
                                                kDrainNs);
                }
                __syncthreads();
                return;
            }
            unsigned char *base = smem + st * StageLayout<MT>::bytes(MT);
            const size_t a_bytes = static_cast<size_t>(kTile) * m * 4;
            float *a_s = reinterpret_cast<float *>(base);
            row = a_s + tid * m;
            warp_rows = a_s + warp * 32 * m;
            kind = base[a_bytes + kTile * 8 + tid];
            w = reinterpret_cast<const float *>(base + a_bytes)[tid];
            pr = reinterpret_cast<const float *>(base + a_bytes + kTile * 4)[tid];
        } else {
            // ragged last tile of a problem: direct loads (every stage of the
            // ring may hold a copy in flight, so no shared scratch is used)
            warp_rows = nullptr;
            if (valid) {
                kind = P.kind[i];
                w = P.w[i];
                pr = P.param[i];
            }
        }
        float2 tp = make_float2(0.f, 0.f);
        uchar2 jp = make_uchar2(255, 255);
        if (lag && valid) {
            tp = lbt_prev[i];
            jp = lbj_prev[i];
        }
        JobSol<float> sol;
        sol.cP = sol.cQ = -1;
        sol.xP = sol.xQ = 0.f;
        if (valid) {
            // full tiles read the staged row, a ragged tile the row in HBM
            solve_job_sm<MT, CAP>(row != nullptr ? row : P.A + i * m, mu_s, lam_s, m, grouped, rot,
                                  kind, w, pr, sol);
            hsum.add(sol.h);
            uxsum.add(sol.u);
            if (lag) {
                const float *sc = kind >= RA_U_LINCAP ? sl_s : s_s;
                float tt = 0.f;
                if (jp.x != 255) tt += sc[jp.x] * tp.x;
                if (jp.y != 255) tt += sc[jp.y] * tp.y;
                lbsum.add(util<float>(kind, w, pr, tt));
            }
            lbt_out[i] = make_float2(sol.tP, sol.tQ);
            lbj_out[i] = make_uchar2(sol.cP >= 0 ? sol.cP : 255, sol.cQ >= 0 ? sol.cQ : 255);
        }
        if (full) {
            if (!CAP)
                warp_rsum_lin<MT, KahanF>(warp_rows, m, lane, grouped, rot, sol,
                                          valid && kind >= RA_U_LINCAP, racc, rlin);
            else
                warp_rsum<MT, float, KahanF>(warp_rows, m, lane, grouped, rot, sol, racc);
        } else {
            warp_rsum_shfl<float, KahanF>(m, lane, sol, racc);
            if (!CAP) warp_rlin<float, KahanF>(valid && kind >= RA_U_LINCAP, lane, sol, rlin);
        }
        __syncthreads();  // stage consumed
        if (full) {
            ++consumed;
            if (tid == 0) {
                fence_proxy_async();
                issue_next();
            }
        }
        // chunk end: block sums -> this chunk's partial slot -> per-problem ticket
        const bool chunk_end = cur.k + 1 >= B.chunk_ntiles[cur.c];
        if (chunk_end) {
            const FF h = warp_sum(ff_of(hsum)), ux = warp_sum(ff_of(uxsum)),
                     lb = warp_sum(ff_of(lbsum)), z = red_zero<FF>();
            if (lane == 0) {
                red[warp][0] = h;
                red[warp][1] = ux;
                red[warp][2] = lb;
                red[warp][3] = z;
            }
            if (lane < m) red[warp][4 + lane] = (grouped ? (lane / MT == 0) : true) ? ff_of(racc) : z;
            if (nv_lin && lane < m) red[warp][4 + m + lane] = ff_of(rlin);
            __syncthreads();
            if (tid < (1 + nv_lin) * m + 4) {
                FF v = red[0][tid];
                for (int w2 = 1; w2 < kWarps; ++w2) v = ff_add(v, red[w2][tid]);
                reinterpret_cast<FF *>(B.partials)[static_cast<size_t>(cur.c) * kPartW + tid] = v;
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                const unsigned nch = static_cast<unsigned>(P.chunk_end - P.chunk_begin);
                is_last = (atomicAdd(&B.ticket[p], 1u) == nch - 1);
            }
            __syncthreads();
            if (is_last) {
                __threadfence();
                sum_partial_rows(reinterpret_cast<const FF *>(B.partials) +
                                     static_cast<size_t>(P.chunk_begin) * kPartW,
                                 static_cast<unsigned>(P.chunk_end - P.chunk_begin),
                                 (1 + nv_lin) * m + 4, red);
                __syncthreads();
                EvalOut *out = B.ev + p;
                if (tid < m) {
                    const double r = to_double(red[0][4 + tid]);
                    out->r[tid] = r;
                    out->q[tid] = P.R[tid] - r;
                    out->r_lin[tid] = nv_lin ? to_double(red[0][4 + m + tid]) : 0.0;
                }
                if (tid == 0) {
                    const double sumh = to_double(red[0][0]);
                    out->sumh = sumh;
                    out->g = lam_dot_R(B.st[p].lam_trial, P.R, m) + sumh;
                    out->Ux = to_double(red[0][1]);
                    out->Ulb_prev = to_double(red[0][2]);
                    B.ticket[p] = 0u;
                }
            }
            __syncthreads();
            hsum = uxsum = lbsum = racc = rlin = KahanF{};
        }
        cursor_next(B, cur);
    }
}

// Batched Eq. e-initialization (once per batch solve): direct loads, one
// FP64 partial per chunk, per-problem ticket and fixed-order final sum.
template <int MT>
__global__ void __launch_bounds__(kTile) batch_init_kernel(BatchDualArgs B, double *lam1,
                                                           const long long *lam_off)
{
    __shared__ float x0_s[RA_MAX_M];
    __shared__ FF red[kWarps][kPartW];
    __shared__ int is_last;
    __shared__ float rows[kTile * MT];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (long long c = blockIdx.x; c < B.nchunks; c += gridDim.x) {
        const int p = B.chunk_prob[c];
        const BatchProblem &P = B.probs[p];
        const int m = P.m;
        __syncthreads();
        if (tid == 0) {
            double kappa = 0.0;
            for (int j = 0; j < m; ++j) kappa += P.R[j] / static_cast<double>(P.n);
            const double div = (B.cap && kappa > 1.0) ? kappa : 1.0;
            for (int j = 0; j < RA_MAX_M; ++j)
                x0_s[j] = j < m ? static_cast<float>(P.R[j] / (static_cast<double>(P.n) * div)) : 0.0f;
        }
        __syncthreads();
        KahanF racc;
        for (int k = 0; k < B.chunk_ntiles[c]; ++k) {
            const long long i = static_cast<long long>(B.chunk_tile0[c] + k) * kTile + tid;
            const bool valid = i < P.n;
            float a[MT];
            float tc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                a[j] = (valid && j < m) ? __ldg(&P.A[i * m + j]) : 0.0f;
                tc[j & 3] = fmaf(a[j], x0_s[j], tc[j & 3]);
            }
            const float t = (tc[0] + tc[1]) + (tc[2] + tc[3]);
            float d = 0.0f;
            if (valid) {
                const int kd = P.kind[i];
                const float wi = P.w[i], pi = P.param[i];
                if (kd == RA_U_LOG) d = wi / t;
                else if (kd == RA_U_POWER) d = wi * pi * exp2f((pi - 1.0f) * log2f(t));
                else d = t < pi ? wi : 0.0f;
            }
            float *own = rows + tid * m;
#pragma unroll
            for (int j = 0; j < MT; ++j)
                if (j < m) own[j] = d * a[j];
            __syncwarp();
            warp_colsum<MT, float, KahanF>(rows + warp * 32 * m, m, lane, false, racc);
        }
        if (lane < m) red[warp][4 + lane] = ff_of(racc);
        __syncthreads();
        if (tid < m) {
            FF v = red[0][4 + tid];
            for (int w2 = 1; w2 < kWarps; ++w2) v = ff_add(v, red[w2][4 + tid]);
            reinterpret_cast<FF *>(B.partials)[static_cast<size_t>(c) * kPartW + tid] = v;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) is_last = (atomicAdd(&B.ticket[p], 1u) == static_cast<unsigned>(P.chunk_end - P.chunk_begin) - 1);
        __syncthreads();
        if (is_last) {
            __threadfence();
            sum_partial_rows(reinterpret_cast<const FF *>(B.partials) +
                                 static_cast<size_t>(P.chunk_begin) * kPartW,
                             static_cast<unsigned>(P.chunk_end - P.chunk_begin), m, red);
            if (tid < m) lam1[lam_off[p] + tid] = to_double(red[0][tid]) / static_cast<double>(P.n);
            if (tid == 0) B.ticket[p] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------- simple kernel

// One thread per job with direct global loads; used for FP64 per-job
// arithmetic (the precision study) and as the generic path.
template <int MT, bool CAP, typename Real, bool LAG, bool REC>
__global__ void __launch_bounds__(kTile)
    dual_simple_kernel(DualParams P)
{
    extern __shared__ __align__(16) unsigned char smem_simple[];
    __shared__ Real lam_s[RA_MAX_M];
    __shared__ float s_s[RA_MAX_M];
    __shared__ float sl_s[RA_MAX_M];
    __shared__ double red[kWarps][kPartW];
    __shared__ double lr_s;
    Real *rows = reinterpret_cast<Real *>(smem_simple);  // kTile x m

    if (P.skip != nullptr && *P.skip != 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = P.m;
    const float2 *lbt_prev = P.lbt_prev;
    const uchar2 *lbj_prev = P.lbj_prev;
    float2 *lbt_out = P.lbt_out;
    uchar2 *lbj_out = P.lbj_out;
    if (P.pingpong != nullptr) {
        const int q = *P.pingpong & 1;
        lbt_prev = P.lbt_buf[q];
        lbj_prev = P.lbj_buf[q];
        lbt_out = P.lbt_buf[q ^ 1];
        lbj_out = P.lbj_buf[q ^ 1];
    }
    const bool lag = LAG && (P.lag_on == nullptr || *P.lag_on != 0);
    if (tid < RA_MAX_M) {
        lam_s[tid] = tid < m ? static_cast<Real>(P.lam[tid]) : Fn<Real>::inf();
        s_s[tid] = (lag && tid < m) ? static_cast<float>(P.s_prev[tid]) : 1.0f;
        sl_s[tid] = (lag && tid < m)
                        ? static_cast<float>((P.s_lin_prev ? P.s_lin_prev : P.s_prev)[tid])
                        : 1.0f;
    }
    __syncthreads();
    Real lam_r[MT], mu_r[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        lam_r[k] = lam_s[k];
        mu_r[k] = inv_price<Real>(lam_s[k]);
    }
    if (tid == 32) lr_s = lam_dot_R(P.lam, P.R, m);  // read after the grid stage's barriers
    double hsum = 0.0, uxsum = 0.0, lbsum = 0.0, racc = 0.0, rlin = 0.0;
    const long long stride = static_cast<long long>(gridDim.x) * kTile;
    const long long nround = (P.n + stride - 1) / stride;
    for (long long rr = 0; rr < nround; ++rr) {
        const long long i = rr * stride + static_cast<long long>(blockIdx.x) * kTile + tid;
        const bool valid = i < P.n;
        Real a[MT];
#pragma unroll
        for (int k = 0; k < MT; ++k) a[k] = (valid && k < m) ? static_cast<Real>(__ldg(&P.A[i * m + k])) : Real(0);
        JobSol<Real> s;
        s.cP = s.cQ = -1;
        s.xP = s.xQ = Real(0);
        int kind = RA_U_LINCAP;
        Real w = 1, p = 0;
        if (valid) {
            kind = P.kind[i];
            w = P.w[i];
            p = P.param[i];
            auto fetch = [&](int k, Real &av, Real &lv) {
                av = static_cast<Real>(__ldg(&P.A[i * m + k]));
                lv = lam_s[k];
            };
            solve_job<MT, CAP, false, Real>(a, lam_r, mu_r, 0, fetch, kind, w, p, s);
            hsum += static_cast<double>(s.h);
            uxsum += static_cast<double>(s.u);
            if (lag) {
                const float2 tp = lbt_prev[i];
                const uchar2 jp = lbj_prev[i];
                const float *sc = kind >= RA_U_LINCAP ? sl_s : s_s;
                Real tt = Real(0);
                if (jp.x != 255) tt += static_cast<Real>(sc[jp.x]) * static_cast<Real>(tp.x);
                if (jp.y != 255) tt += static_cast<Real>(sc[jp.y]) * static_cast<Real>(tp.y);
                lbsum += static_cast<double>(util<Real>(kind, w, p, tt));
            }
            if (REC) {
                lbt_out[i] = make_float2(static_cast<float>(s.tP), static_cast<float>(s.tQ));
                lbj_out[i] = make_uchar2(s.cP >= 0 ? s.cP : 255, s.cQ >= 0 ? s.cQ : 255);
            }
        }
        warp_rsum<MT, Real, double>(rows + warp * 32 * m, m, lane, false, 0, s, racc);
        if (!CAP) warp_rlin<Real, double>(valid && kind >= RA_U_LINCAP, lane, s, rlin);
    }
    reduce_and_finalize(hsum, uxsum, lbsum, racc, rlin, m, !CAP, true, P, red, &lr_s);
}

// ---------------------------------------------------------------------------- lower bound

// U(X~) = sum_i u_i(s_P t_P + s_Q t_Q), s the column scaling of an evaluation's
// r and r_lin (Section 5; see column_scales), from the compact per-job records.
__global__ void __launch_bounds__(kTile)
    lower_bound_kernel(const uint8_t *kind, const float *w, const float *param, const float2 *lbt,
                       const uchar2 *lbj, long long n, int m, const EvalOut *src, const double *R,
                       int cap, double *partials, unsigned *ticket, double *U_lb)
{
    __shared__ float s_s[RA_MAX_M];
    __shared__ float sl_s[RA_MAX_M];
    __shared__ double red[kWarps];
    __shared__ int is_last;
    const int tid = threadIdx.x;
    if (tid < RA_MAX_M) {
        float s = 1.0f, sl = 1.0f;
        if (tid < m) {
            double sd, sld;
            column_scales(R[tid], src->r[tid], src->r_lin[tid], cap, sd, sld);
            s = static_cast<float>(sd);
            sl = static_cast<float>(sld);
        }
        s_s[tid] = s;
        sl_s[tid] = sl;
    }
    __syncthreads();
    KahanF acc;
    for (long long i = static_cast<long long>(blockIdx.x) * kTile + tid; i < n;
         i += static_cast<long long>(gridDim.x) * kTile) {
        const float2 tp = lbt[i];
        const uchar2 jp = lbj[i];
        const int kd = kind[i];
        const float *sc = kd >= RA_U_LINCAP ? sl_s : s_s;
        float tt = 0.f;
        if (jp.x != 255) tt += sc[jp.x] * tp.x;
        if (jp.y != 255) tt += sc[jp.y] * tp.y;
        acc.add(util<float>(kd, w[i], param[i], tt));
    }
    const double accd = warp_sum_d(acc.value());
    if ((tid & 31) == 0) red[tid >> 5] = accd;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < kWarps; ++k) v += red[k];
        partials[blockIdx.x] = v;
        __threadfence();
        is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && tid == 0) {
        __threadfence();
        double v = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&partials[b]);
        *U_lb = isnan(src->sumh) ? src->sumh : v;   // the evaluation it scales was incomplete
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------- recovery

// Per-job allocation at lambda (Section 3, recovering an allocation), with
// the near-tie flag of the effective-price argmin.
template <int MT, bool CAP, typename Real>
__global__ void __launch_bounds__(kTile)
    recover_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                   long long n, int m, const double *lam, int32_t *jstar, int32_t *j12, float *x12,
                   float *tout, float *X, uint8_t *near_tie, unsigned long long *n_ties,
                   double *partials, unsigned *ticket, double *U)
{
    __shared__ Real lam_s[RA_MAX_M];
    __shared__ double red[kWarps];
    __shared__ int is_last;
    const int tid = threadIdx.x;
    if (tid < RA_MAX_M) lam_s[tid] = tid < m ? static_cast<Real>(lam[tid]) : Fn<Real>::inf();
    __syncthreads();
    Real lam_r[MT], mu_r[MT];
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        lam_r[k] = lam_s[k];
        mu_r[k] = inv_price<Real>(lam_s[k]);
    }
    double usum = 0.0;
    unsigned long long ties = 0;
    for (long long i = static_cast<long long>(blockIdx.x) * kTile + tid; i < n;
         i += static_cast<long long>(gridDim.x) * kTile) {
        Real a[MT];
#pragma unroll
        for (int k = 0; k < MT; ++k) a[k] = k < m ? static_cast<Real>(__ldg(&A[i * m + k])) : Real(0);
        const int kd = kind[i];
        const Real wi = w[i], pi = param[i];
        JobSol<Real> s;
        auto fetch = [&](int k, Real &av, Real &lv) {
            av = static_cast<Real>(__ldg(&A[i * m + k]));
            lv = lam_s[k];
        };
        solve_job<MT, CAP, true, Real>(a, lam_r, mu_r, 0, fetch, kd, wi, pi, s);
        usum += static_cast<double>(util<Real>(kd, wi, pi, s.t));
        const bool tie = s.best > Real(0) && s.second >= s.best * Real(1.0 / (1.0 + 1e-6));
        ties += tie ? 1ull : 0ull;
        if (near_tie) near_tie[i] = tie ? 1 : 0;
        if (jstar) jstar[i] = s.jstar;
        if (j12) {
            j12[2 * i] = s.cP >= 0 ? s.cP : s.cQ;
            j12[2 * i + 1] = s.cP >= 0 ? s.cQ : -1;
        }
        if (x12) {
            x12[2 * i] = static_cast<float>(s.cP >= 0 ? s.xP : s.xQ);
            x12[2 * i + 1] = static_cast<float>(s.cP >= 0 ? s.xQ : Real(0));
        }
        if (tout) tout[i] = static_cast<float>(s.t);
        if (X) {
            for (int j = 0; j < m; ++j) {
                float v = 0.f;
                if (j == s.cP) v = static_cast<float>(s.xP);
                if (j == s.cQ) v = static_cast<float>(s.xQ);
                X[i * m + j] = v;
            }
        }
    }
    if (n_ties) {
        for (int off = 16; off > 0; off >>= 1) ties += __shfl_xor_sync(kFull, ties, off);
        if ((tid & 31) == 0 && ties) atomicAdd(n_ties, ties);
    }
    usum = warp_sum_d(usum);
    if ((tid & 31) == 0) red[tid >> 5] = usum;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < kWarps; ++k) v += red[k];
        partials[blockIdx.x] = v;
        __threadfence();
        is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && tid == 0) {
        __threadfence();
        double v = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&partials[b]);
        if (U) *U = v;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------------------- records

__global__ void records_kernel(const float2 *lbt, const uchar2 *lbj, long long n, int32_t *j12,
                               float *t12)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const uchar2 j = lbj[i];
        const float2 t = lbt[i];
        j12[2 * i] = j.x == 255 ? -1 : j.x;
        j12[2 * i + 1] = j.y == 255 ? -1 : j.y;
        t12[2 * i] = t.x;
        t12[2 * i + 1] = t.y;
    }
}

// ---------------------------------------------------------------------------- dispatch

// Ring stages for a shared-memory budget per CTA: 106 KB lets two CTAs share
// an SM (the capped kernels, 128 registers), 70 KB three (the uncapped ones).
template <int MT>
int mt_stages(int m, size_t budget = 106 * 1024)
{
    const size_t sb = StageLayout<MT>::bytes(m);
    int s = static_cast<int>(budget / sb);
    if (s > kMaxStages) s = kMaxStages;
    if (s < 2) s = 2;
    return s;
}

template <int MT, bool CAP, bool LAG, bool REC>
cudaError_t launch_tma(const ra_problem *p, const DualParams &dp_in, cudaStream_t s)
{
    const long long num_full = p->n / kTile;
    int grid = p->grid_dual;
    if (num_full < grid) grid = static_cast<int>(num_full > 0 ? num_full : 1);
    DualParams dp = dp_in;
    dp.wait_ns = wait_limit_ns();
    dual_tma_kernel<MT, CAP, LAG, REC><<<grid, kTile, p->smem_dual, s>>>(dp, p->stages, num_full);
    return cudaGetLastError();
}

template <int MT, bool CAP, typename Real, bool LAG, bool REC>
cudaError_t launch_simple(const ra_problem *p, const DualParams &dp, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    const size_t smem = static_cast<size_t>(kTile) * p->m * sizeof(Real);
    dual_simple_kernel<MT, CAP, Real, LAG, REC><<<static_cast<int>(blocks), kTile, smem, s>>>(dp);
    return cudaGetLastError();
}

template <int MT, bool CAP>
cudaError_t launch_dual_mt(const ra_problem *p, const DualParams &dp, cudaStream_t s)
{
    const bool lag = dp.lbt_prev != nullptr;
    const bool rec = dp.lbt_out != nullptr;
    if (p->flags & RA_FP64_JOBMATH) {
        if (lag) return rec ? launch_simple<MT, CAP, double, true, true>(p, dp, s)
                            : launch_simple<MT, CAP, double, true, false>(p, dp, s);
        return rec ? launch_simple<MT, CAP, double, false, true>(p, dp, s)
                   : launch_simple<MT, CAP, double, false, false>(p, dp, s);
    }
    if (lag) return rec ? launch_tma<MT, CAP, true, true>(p, dp, s) : launch_tma<MT, CAP, true, false>(p, dp, s);
    return rec ? launch_tma<MT, CAP, false, true>(p, dp, s) : launch_tma<MT, CAP, false, false>(p, dp, s);
}

template <int MT, bool CAP>
cudaError_t set_attrs_mt()
{
    cudaError_t e;
#define RA_ATTR(L, R)                                                                              \
    e = cudaFuncSetAttribute(dual_tma_kernel<MT, CAP, L, R>,                                      \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemMax);            \
    if (e != cudaSuccess) return e;
    RA_ATTR(false, false)
    RA_ATTR(false, true)
    RA_ATTR(true, false)
    RA_ATTR(true, true)
#undef RA_ATTR
#define RA_ATTR(L, R)                                                                              \
    e = cudaFuncSetAttribute(dual_simple_kernel<MT, CAP, double, L, R>,                           \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTile * MT * 8);        \
    if (e != cudaSuccess) return e;                                                                \
    e = cudaFuncSetAttribute(dual_simple_kernel<MT, CAP, float, L, R>,                            \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTile * MT * 4);        \
    if (e != cudaSuccess) return e;
    RA_ATTR(false, false)
    RA_ATTR(false, true)
    RA_ATTR(true, false)
    RA_ATTR(true, true)
#undef RA_ATTR
    return cudaSuccess;
}

}  // namespace

cudaError_t configure_dual(ra_problem *p)
{
    const int m = p->m;
    p->mt = m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : 32;
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    // two / three CTAs per SM; a stage also holds the tile's 2.5 KB of records
    const size_t budget = cap ? 111 * 1024 : 70 * 1024;
    const size_t sb = ring_stage_bytes(m);  // layout does not depend on MT
    int stages = static_cast<int>(budget / sb);
    if (stages > kMaxStages) stages = kMaxStages;
    if (stages < 2) stages = 2;
    p->stages = stages;
    p->smem_dual = p->stages * sb + 128;
    if (p->smem_dual < kWarps * kPartW * sizeof(FF) + 128) p->smem_dual = kWarps * kPartW * sizeof(FF) + 128;
    cudaError_t e;
#define RA_IATTR(MT)                                                                               \
    if ((e = cudaFuncSetAttribute(init_tma_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  kRingSmemMax)) != cudaSuccess)                                     \
        return e;
    RA_IATTR(4)
    RA_IATTR(8)
    RA_IATTR(16)
    RA_IATTR(32)
#undef RA_IATTR
#define RA_GATTR(MT)                                                                               \
    if ((e = cudaFuncSetAttribute(dual_g2_kernel<MT, true>,                                       \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemMax)) !=     \
        cudaSuccess)                                                                               \
        return e;                                                                                  \
    if ((e = cudaFuncSetAttribute(dual_g2_kernel<MT, false>,                                      \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemMax)) !=     \
        cudaSuccess)                                                                               \
        return e;
    RA_GATTR(4)
    RA_GATTR(8)
    RA_GATTR(16)
    RA_GATTR(32)
#undef RA_GATTR
    if ((e = set_attrs_mt<4, true>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<8, true>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<16, true>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<32, true>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<4, false>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<8, false>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<16, false>()) != cudaSuccess) return e;
    if ((e = set_attrs_mt<32, false>()) != cudaSuccess) return e;
    int per_sm = 1;
    const void *fn = nullptr;
    switch (p->mt) {
    case 4: fn = cap ? reinterpret_cast<const void *>(dual_tma_kernel<4, true, true, true>)
                     : reinterpret_cast<const void *>(dual_tma_kernel<4, false, true, true>); break;
    case 8: fn = cap ? reinterpret_cast<const void *>(dual_tma_kernel<8, true, true, true>)
                     : reinterpret_cast<const void *>(dual_tma_kernel<8, false, true, true>); break;
    case 16: fn = cap ? reinterpret_cast<const void *>(dual_tma_kernel<16, true, true, true>)
                      : reinterpret_cast<const void *>(dual_tma_kernel<16, false, true, true>); break;
    default: fn = cap ? reinterpret_cast<const void *>(dual_tma_kernel<32, true, true, true>)
                      : reinterpret_cast<const void *>(dual_tma_kernel<32, false, true, true>); break;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTile, p->smem_dual);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    p->grid_dual = p->num_sms * per_sm;
    p->grid_aux = p->num_sms * 4;
    return cudaSuccess;
}

cudaError_t launch_dual(const ra_problem *p, const DualParams &dp, cudaStream_t s)
{
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    switch (p->mt) {
    case 4: return cap ? launch_dual_mt<4, true>(p, dp, s) : launch_dual_mt<4, false>(p, dp, s);
    case 8: return cap ? launch_dual_mt<8, true>(p, dp, s) : launch_dual_mt<8, false>(p, dp, s);
    case 16: return cap ? launch_dual_mt<16, true>(p, dp, s) : launch_dual_mt<16, false>(p, dp, s);
    default: return cap ? launch_dual_mt<32, true>(p, dp, s) : launch_dual_mt<32, false>(p, dp, s);
    }
}

cudaError_t launch_lower_bound(const ra_problem *p, const float2 *lbt, const uchar2 *lbj,
                               const EvalOut *src, double *U_lb, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    lower_bound_kernel<<<static_cast<int>(blocks), kTile, 0, s>>>(
        p->kind, p->w, p->param, lbt, lbj, p->n, p->m, src, p->R, !(p->flags & RA_NO_JOB_CAP),
        p->partials, p->ticket + 1, U_lb);
    return cudaGetLastError();
}

cudaError_t launch_records(const ra_problem *p, int32_t *j12, float *t12, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    records_kernel<<<static_cast<int>(blocks), kTile, 0, s>>>(p->lbt[0], p->lbj[0], p->n, j12, t12);
    return cudaGetLastError();
}

cudaError_t launch_dual_g2(const ra_problem *p, const double *lam_a, const double *lam_b,
                           double *g_out, cudaStream_t s)
{
    const long long num_full = p->n / kTile;
    int grid = p->grid_dual;
    if (num_full < grid) grid = static_cast<int>(num_full > 0 ? num_full : 1);
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
#define RA_G2(MT)                                                                                  \
    if (cap)                                                                                       \
        dual_g2_kernel<MT, true><<<grid, kTile, p->smem_dual, s>>>(                                \
            p->A, p->kind, p->w, p->param, p->R, p->n, p->m, lam_a, lam_b, p->stages, num_full,    \
            p->partials, p->ticket + 3, p->status, wait_limit_ns(), g_out);                        \
    else                                                                                           \
        dual_g2_kernel<MT, false><<<grid, kTile, p->smem_dual, s>>>(                               \
            p->A, p->kind, p->w, p->param, p->R, p->n, p->m, lam_a, lam_b, p->stages, num_full,    \
            p->partials, p->ticket + 3, p->status, wait_limit_ns(), g_out);
    switch (p->mt) {
    case 4: RA_G2(4) break;
    case 8: RA_G2(8) break;
    case 16: RA_G2(16) break;
    default: RA_G2(32) break;
    }
#undef RA_G2
    return cudaGetLastError();
}

cudaError_t launch_init(const ra_problem *p, double *lam1, cudaStream_t s)
{
    const long long num_full = p->n / kTile;
    int grid = p->grid_dual;
    if (num_full < grid) grid = static_cast<int>(num_full > 0 ? num_full : 1);
    const int cap = !(p->flags & RA_NO_JOB_CAP);
#define RA_INIT(MT)                                                                                \
    init_tma_kernel<MT><<<grid, kTile, p->smem_dual, s>>>(p->A, p->kind, p->w, p->param, p->R,      \
                                                          p->n, p->m, cap, p->stages, num_full,    \
                                                          p->partials, p->ticket + 2, p->status,   \
                                                          wait_limit_ns(), lam1)
    switch (p->mt) {
    case 4: RA_INIT(4); break;
    case 8: RA_INIT(8); break;
    case 16: RA_INIT(16); break;
    default: RA_INIT(32); break;
    }
#undef RA_INIT
    return cudaGetLastError();
}

template <int MT, bool CAP, typename Real>
static cudaError_t launch_recover_t(const ra_problem *p, int blocks, const double *lam,
                                    int32_t *jstar, int32_t *j12, float *x12, float *t, float *X,
                                    double *U, uint8_t *near_tie, unsigned long long *n_ties,
                                    cudaStream_t s)
{
    recover_kernel<MT, CAP, Real><<<blocks, kTile, 0, s>>>(p->A, p->kind, p->w, p->param, p->n, p->m,
                                                            lam, jstar, j12, x12, t, X, near_tie,
                                                            n_ties, p->partials, p->ticket + 3, U);
    return cudaGetLastError();
}

cudaError_t launch_recover(const ra_problem *p, const double *lam, int32_t *jstar, int32_t *j12,
                           float *x12, float *t, float *X, double *U, uint8_t *near_tie,
                           unsigned long long *n_ties, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    const int b = static_cast<int>(blocks);
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    const bool f64 = (p->flags & RA_FP64_JOBMATH) != 0;
#define RA_REC(MT)                                                                                 \
    if (f64) return cap ? launch_recover_t<MT, true, double>(p, b, lam, jstar, j12, x12, t, X, U, near_tie, n_ties, s) \
                        : launch_recover_t<MT, false, double>(p, b, lam, jstar, j12, x12, t, X, U, near_tie, n_ties, s); \
    return cap ? launch_recover_t<MT, true, float>(p, b, lam, jstar, j12, x12, t, X, U, near_tie, n_ties, s)          \
               : launch_recover_t<MT, false, float>(p, b, lam, jstar, j12, x12, t, X, U, near_tie, n_ties, s);
    switch (p->mt) {
    case 4: RA_REC(4)
    case 8: RA_REC(8)
    case 16: RA_REC(16)
    default: RA_REC(32)
    }
#undef RA_REC
}


int batch_stages(int mt, int cap)
{
    const size_t budget = cap ? 106 * 1024 : 70 * 1024;   // two / three CTAs per SM
    switch (mt) {
    case 4: return mt_stages<4>(4, budget);
    case 8: return mt_stages<8>(8, budget);
    case 16: return mt_stages<16>(16, budget);
    default: return mt_stages<32>(32, budget);
    }
}

size_t batch_smem(int mt, int cap) { return batch_stages(mt, cap) * StageLayout<4>::bytes(mt) + 128; }

cudaError_t batch_configure(int mt, int cap, int *blocks_per_sm)
{
    const void *fn = nullptr;
    switch (mt) {
    case 4: fn = cap ? reinterpret_cast<const void *>(batch_dual_kernel<4, true>)
                     : reinterpret_cast<const void *>(batch_dual_kernel<4, false>); break;
    case 8: fn = cap ? reinterpret_cast<const void *>(batch_dual_kernel<8, true>)
                     : reinterpret_cast<const void *>(batch_dual_kernel<8, false>); break;
    case 16: fn = cap ? reinterpret_cast<const void *>(batch_dual_kernel<16, true>)
                      : reinterpret_cast<const void *>(batch_dual_kernel<16, false>); break;
    default: fn = cap ? reinterpret_cast<const void *>(batch_dual_kernel<32, true>)
                      : reinterpret_cast<const void *>(batch_dual_kernel<32, false>); break;
    }
    cudaError_t e;
#define RA_BATTR(MT)                                                                               \
    if ((e = cudaFuncSetAttribute(batch_dual_kernel<MT, true>,                                    \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemMax)) !=     \
        cudaSuccess)                                                                               \
        return e;                                                                                  \
    if ((e = cudaFuncSetAttribute(batch_dual_kernel<MT, false>,                                   \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmemMax)) !=     \
        cudaSuccess)                                                                               \
        return e;
    RA_BATTR(4)
    RA_BATTR(8)
    RA_BATTR(16)
    RA_BATTR(32)
#undef RA_BATTR
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kTile, batch_smem(mt, cap));
}

cudaError_t launch_batch_dual(int mt, const BatchDualArgs &a_in, int grid, size_t smem, cudaStream_t s)
{
    BatchDualArgs a = a_in;
    a.wait_ns = wait_limit_ns();
#define RA_BD(MT)                                                                                  \
    if (a.cap) batch_dual_kernel<MT, true><<<grid, kTile, smem, s>>>(a);                          \
    else batch_dual_kernel<MT, false><<<grid, kTile, smem, s>>>(a);
    switch (mt) {
    case 4: RA_BD(4) break;
    case 8: RA_BD(8) break;
    case 16: RA_BD(16) break;
    default: RA_BD(32) break;
    }
#undef RA_BD
    return cudaGetLastError();
}

cudaError_t launch_batch_init(int mt, const BatchDualArgs &a, double *lam1, const long long *lam_off,
                              int grid, cudaStream_t s)
{
    switch (mt) {
    case 4: batch_init_kernel<4><<<grid, kTile, 0, s>>>(a, lam1, lam_off); break;
    case 8: batch_init_kernel<8><<<grid, kTile, 0, s>>>(a, lam1, lam_off); break;
    case 16: batch_init_kernel<16><<<grid, kTile, 0, s>>>(a, lam1, lam_off); break;
    default: batch_init_kernel<32><<<grid, kTile, 0, s>>>(a, lam1, lam_off); break;
    }
    return cudaGetLastError();
}

}  // namespace ra
