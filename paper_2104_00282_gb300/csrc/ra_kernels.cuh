// Device building blocks shared by the streaming kernels (ra_dual.cu) and
// the allocation-repair kernels (ra_repair.cu): PTX wrappers for the bulk-copy
// ring, utilities and their closed-form maximisers (Section 2.2, Eqs.
// e-opt-t-log / e-opt-t-target), the per-job subproblem of Algorithm 1, and
// the deterministic compensated / float-float reductions.  Everything has
// internal linkage: each translation unit gets its own copy.
#pragma once

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

// L2 policy for data read once per pass (the problem's rows, weights,
// parameters and kinds): evicted first, so that what is read again soon --
// the solver state, the lower-bound records -- stays in L2 across a pass
// that streams more than L2 holds.
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_load_stream(void *dst, const void *src, uint32_t bytes,
                                                 uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
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

// u(t), Section 2.2.  Power utilities: w t^p for 0 < p < 1, -w t^p for
// p < 0 (the alpha-fair utilities with alpha = 1 - p > 1); the latter is
// -inf at t = 0 like the logarithm.
template <typename Real>
__device__ __forceinline__ Real util(int kind, Real w, Real p, Real t)
{
    if (kind == RA_U_LOG) return w * Fn<Real>::log(t);
    if (kind == RA_U_POWER) {
        if (!(t > Real(0))) return p > Real(0) ? Real(0) : -Fn<Real>::inf();
        const Real v = w * Fn<Real>::exp2(p * Fn<Real>::log2(t));
        return p > Real(0) ? v : -v;
    }
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
    const float pw = w * __expf(p * L);          // +inf at t = 0 when p < 0
    const float up = p > 0.0f ? (t > 0.0f ? pw : 0.0f) : -pw;
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
        else t = Fn<Real>::exp2(Fn<Real>::log2(w * fabs(p) / alpha) / (Real(1) - p));
    } else {
        if (w <= alpha) return lo;
        if (alpha < Real(0)) return hi;
        t = p;
    }
    return fmin(fmax(t, lo), hi);
}

// FP32 variant of topt with the same selection structure: log w/alpha,
// power exp(log(w |p| / alpha) / (1 - p)) (u'(t) = w |p| t^(p-1) for either
// sign of p), both through the fast intrinsics.
template <>
__device__ __forceinline__ float topt<float>(int kind, float w, float p, float alpha, float lo,
                                             float hi)
{
    const float tl = __fdividef(w, alpha);
    const float tp = __expf(__fdividef(__logf(__fdividef(w * fabsf(p), alpha)), 1.0f - p));
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
    int segP, segQ;   // columns of the cost segment holding t (-1: the origin / none)
    Real alpha;       // its slope
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
    Real amax = Real(0);   // right end of the hull's domain (cap only)
#pragma unroll
    for (int k = 0; k < MT; ++k) {
        const Real v = a[k] * mu[k];
        if (v > bv[k & 3]) {
            bv[k & 3] = v;
            bk[k & 3] = k;
        }
        if (CAP) amax = a[k] > amax ? a[k] : amax;
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
        s.segP = s.segQ = -1;
        s.alpha = Real(0);
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
            if (aQ >= amax) {  // no vertex to the right: the scan would find none
                t = aQ;
                break;
            }
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
    s.segP = kP >= 0 ? colof<MT>(kP, rot) : -1;
    s.segQ = colof<MT>(kQ, rot);
    s.alpha = alpha;
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
    float amax = 0.f;                // right end of the hull's domain (cap only)
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
            if (CAP) amax = fmaxf(amax, fmaxf(fmaxf(av.x, av.y), fmaxf(av.z, av.w)));
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
                if (CAP) amax = fmaxf(amax, row[k]);
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
            if (aQ >= amax) {  // no vertex to the right: the scan would find none
                t = aQ;
                break;
            }
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
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(const KahanF &a) { return a.value(); }

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
    // the lane mask rotated with the chunk order, so that chunk c's four
    // bits sit at the constant positions 4c .. 4c + 3
    const unsigned lmr = LIN ? __funnelshift_r(lm, lm, 4 * rot) : 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int q = (c + rot) & 7;
        const float4 v = reinterpret_cast<const float4 *>(row)[q];
        cs[0] += v.x;
        cs[1] += v.y;
        cs[2] += v.z;
        cs[3] += v.w;
        if (LIN) {
            if (lmr & (1u << (4 * c))) cl[0] += v.x;
            if (lmr & (2u << (4 * c))) cl[1] += v.y;
            if (lmr & (4u << (4 * c))) cl[2] += v.z;
            if (lmr & (8u << (4 * c))) cl[3] += v.w;
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

}  // namespace
}  // namespace ra
