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
#include <type_traits>

#include "ra_kernels.cuh"

namespace ra {
namespace {

template <typename T>
__device__ void reduce_and_finalize(T hsum, T uxsum, T lbsum, T racc, T rlin, int m, bool lin,
                                    bool lane_owns_col, const DualParams &P, T (*red)[kPartW],
                                    const double *lr_s, bool own)
{
    // own: the third sum is the own bound's remainder s2neg (no lagged bound)
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
        P.out->Ulb_prev = own ? 0.0 : bad ? nan_d() : to_double(red[0][2]);
        P.out->s2neg = own && !bad ? to_double(red[0][2]) : nan_d();
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
// A stage of the batched pass: a tile of the width class (rows of mt columns)
// and room for its records.
__host__ __device__ inline size_t batch_stage_bytes(int mt) { return StageLayout<4>::bytes(mt) + kRecBytes; }

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
                            int *status, uint64_t wait_ns, Job &&job, Pre &&pre = Pre{},
                            long long tstride = 1)
{
    // tstride > 1: only full tiles 0, tstride, 2 tstride, ... (a strided
    // sample of the jobs; no ragged tail)
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
    const long long n_tiles = (num_full + tstride - 1) / tstride;
    const long long n_my = (n_tiles > blockIdx.x) ? (n_tiles - blockIdx.x + G - 1) / G : 0;
    auto issue = [&](long long it) {
        if (it >= n_my) return;
        const long long tile = (blockIdx.x + it * G) * tstride;
        const int st = static_cast<int>(it % stages);
        unsigned char *base = smem + st * st_bytes;
        const long long j0 = tile * kTile;
        mbar_arrive_expect_tx(&bars[st], static_cast<uint32_t>(core_bytes + (recs ? kRecBytes : 0)));
        const uint64_t pol = policy_evict_first();
        bulk_load_stream(base, A + j0 * m, static_cast<uint32_t>(a_bytes), &bars[st], pol);
        bulk_load_stream(base + a_bytes, W + j0, kTile * 4, &bars[st], pol);
        bulk_load_stream(base + a_bytes + kTile * 4, Par + j0, kTile * 4, &bars[st], pol);
        bulk_load_stream(base + a_bytes + kTile * 8, Kind + j0, kTile, &bars[st], pol);
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
        const long long i = (blockIdx.x + it * G) * tstride * kTile + tid;
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
    if (tstride == 1 && tail0 < n && blockIdx.x == static_cast<unsigned>(num_full % G)) {
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
__global__ void __launch_bounds__(kTile, (CAP && MT >= 16) ? 2 : 3)
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

    if ((P.skip != nullptr && *P.skip != 0) || (P.skip2 != nullptr && *P.skip2 != 0)) return;

    const int tid = threadIdx.x, lane = tid & 31;
    const int m = P.m;
    const bool grouped = (m == MT);
    const float2 *lbt_prev = P.lbt_prev;
    const uchar2 *lbj_prev = P.lbj_prev;
    float2 *lbt_out = P.lbt_out;
    uchar2 *lbj_out = P.lbj_out;
    const int q = P.pingpong != nullptr ? (*P.pingpong & 1) : 0;
    if (P.pingpong != nullptr) {
        lbt_prev = P.lbt_buf[q];
        lbj_prev = P.lbj_buf[q];
        lbt_out = P.lbt_buf[q ^ 1];
        lbj_out = P.lbj_buf[q ^ 1];
    }
    const bool lag = LAG && (P.lag_on == nullptr || *P.lag_on != 0);
    // records of this evaluation; the linear jobs' usage that scales them
    // (and, without the cap, the own bound's remainder sum) also without them
    const int rec_flag = P.rec_on == nullptr ? 1 : *P.rec_on;
    const bool rec_w = REC && (rec_flag & 1) != 0;
    const bool lin_w = REC && !CAP && rec_flag != 0;
    const bool own = lin_w && !LAG;
    if (P.pingpong != nullptr && blockIdx.x == 0 && tid == 0) P.out->rec_buf = rec_w ? (q ^ 1) : -1;
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
            // u(s t) >= u(t) + t u'(t) ln s fails only for p < 0 (Taylor remainder)
            if (!LAG && own && kind == RA_U_POWER && p < 0.f) lbsum.add(p * p * fabsf(s.u));
            if (rec_w) {
                lbt_out[i] = make_float2(s.tP, s.tQ);
                lbj_out[i] = make_uchar2(s.cP >= 0 ? s.cP : 255, s.cQ >= 0 ? s.cQ : 255);
            }
        }
        if (lin_w)
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
                        lin_w, grouped ? (lane / MT == 0) : true, P, ring_red(smem), &lr_s, own);
}

// Initial prices, Eq. e-initialization:
//   lambda^1 = (1/n) sum_i u_i'(a_i^T x0) a_i,  x0 = R / (kappa n),
// streamed through the same TMA ring: each job scales its own row in shared
// memory by d_i = u_i'(a_i^T x0) and the warp sums the rows column-wise.
template <int MT>
__global__ void __launch_bounds__(kTile, 2)
    init_tma_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                    const double *R, long long n, int m, int cap, int stages, long long num_full,
                    double *partials, unsigned *ticket, int *status, uint64_t wait_ns,
                    long long n_all, double *lam1, long long tstride)
{
    // n_all: jobs of the whole problem when these n are one shard of it (the
    // per-job budget R / n_all and the mean's divisor); n otherwise.
    // tstride > 1: the mean over every tstride-th full tile only
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ float x0_s[RA_MAX_M];
    const int tid = threadIdx.x, lane = tid & 31;
    const bool grouped = (m == MT);
    constexpr int C = MT / 4;
    const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
    if (tid == 0) {
        double kappa = 0.0;
        for (int j = 0; j < m; ++j) kappa += R[j] / static_cast<double>(n_all);
        const double div = (cap && kappa > 1.0) ? kappa : 1.0;
        for (int j = 0; j < RA_MAX_M; ++j)
            x0_s[j] = j < m ? static_cast<float>(R[j] / (static_cast<double>(n_all) * div)) : 0.0f;
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
            else if (kd == RA_U_POWER) d = wi * fabsf(pi) * exp2f((pi - 1.0f) * log2f(t));
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
                    wait_ns, job, NoPrologue{}, tstride);
    const FF z = red_zero<FF>();
    FF(*red)[kPartW] = ring_red(smem);
    if (grid_reduce(z, z, z, ff_of(racc), z, m, false, grouped ? (lane / MT == 0) : true, partials,
                    ticket, red)) {
        // a CTA whose wait gave up left its share out of the sums: no prices
        const bool bad = (ld_status(status) & kStatusTimeout) != 0;
        const double div = tstride > 1 ? static_cast<double>((num_full + tstride - 1) / tstride * kTile)
                                       : static_cast<double>(n_all);
        if (tid < m) lam1[tid] = bad ? nan_d() : to_double(red[0][4 + tid]) / div;
    }
}

// Scale of the starting prices along their ray (no per-job cap).  Scaling
// every price by s scales every job's cheapest effective price c_i by s
// (Section 4.1: the first cost segment leaves the origin towards the point of
// highest a_j / lambda_j, whatever the common scale), so
//     g(s lambda) = s lambda^T R + sum_i h_i(s c_i),
//     g'(s)       = lambda^T R - sum_i c_i t_i(s),
// and the minimiser along the ray is where the spending at the unscaled
// effective prices, sum_i c_i t_i(s), equals lambda^T R.  One pass sums that
// spending on the grid s_k = 2^(k - 8), k < kRayK, per job in closed form:
// c t = w / s for log utilities, c t_1 s^(-1/(1-p)) for power utilities (t_1
// the throughput at s = 1), c T while w > s c for linear utilities; the last
// CTA interpolates the crossing in log-log and rescales lambda in place.
constexpr int kRayK = 16;
template <int MT>
__global__ void __launch_bounds__(kTile, 2)
    ray_scale_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                     const double *R, long long n, int m, double *lam, int stages,
                     long long num_full, double *partials, unsigned *ticket, int *status,
                     uint64_t wait_ns, long long tstride)
{
    // tstride > 1: the spending of every tstride-th full tile, set against
    // the same share of lambda^T R
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ __align__(16) float mu_s[RA_MAX_M];
    __shared__ double lamd_s[RA_MAX_M], Rd_s[RA_MAX_M];
    __shared__ double lr_s;
    const int tid = threadIdx.x, lane = tid & 31;
    const bool grouped = (m == MT);
    constexpr int C = MT / 4;
    const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
    if (tid < RA_MAX_M) {
        lamd_s[tid] = tid < m ? lam[tid] : 0.0;
        Rd_s[tid] = tid < m ? R[tid] : 0.0;
        mu_s[tid] = inv_price<float>(tid < m ? static_cast<float>(lamd_s[tid]) : Fn<float>::inf());
    }
    __syncthreads();
    KahanF S[kRayK];
    auto job = [&](long long i, bool valid, const float *row, int kd, float wi, float pi,
                   float *warp_rows, const unsigned char *) {
        (void)i;
        (void)warp_rows;
        if (!valid) return;
        float vb = 0.f;   // max_j a_j / lambda_j = 1 / c
        if (grouped) {
#pragma unroll
            for (int c4 = 0; c4 < C; ++c4) {
                const int q = (c4 + rot) & (C - 1);
                const float4 av = reinterpret_cast<const float4 *>(row)[q];
                const float4 mv = reinterpret_cast<const float4 *>(mu_s)[q];
                vb = fmaxf(vb, fmaxf(fmaxf(av.x * mv.x, av.y * mv.y), fmaxf(av.z * mv.z, av.w * mv.w)));
            }
        } else {
            for (int k = 0; k < m; ++k) vb = fmaxf(vb, row[k] * mu_s[k]);
        }
        if (!(vb > 0.f)) return;
        const float c = 1.0f / vb;
        if (kd <= RA_U_POWER) {
            // spending at s_0 = 2^-8 and the factor between successive scales
            float base, ratio;
            if (kd == RA_U_LOG) {
                base = wi * 256.0f;
                ratio = 0.5f;
            } else {
                const float e = 1.0f / (1.0f - pi);
                base = fminf(__expf(__logf(c) + e * (__logf(wi * fabsf(pi) / c) + 8.0f * 0.69314718f)), 1e30f);
                ratio = exp2f(-e);
            }
#pragma unroll
            for (int k = 0; k < kRayK; ++k) {
                S[k].add(base);
                base *= ratio;
            }
        } else {
            const float spend = c * pi;
            float sk = 1.0f / 256.0f;
#pragma unroll
            for (int k = 0; k < kRayK; ++k) {
                S[k].add(wi > sk * c ? spend : 0.0f);
                sk *= 2.0f;
            }
        }
    };
    unsigned char *smem = align128<MT>(smem_dyn);
    stream_jobs<MT>(A, w, param, kind, nullptr, nullptr, n, m, stages, num_full, smem, bars, status,
                    wait_ns, job, [&] {
                        if (tid == 32) lr_s = lam_dot_R(lamd_s, Rd_s, m);
                    }, tstride);
    // lane k of every warp takes the warp's total of S_k
    FF mine = red_zero<FF>();
#pragma unroll
    for (int k = 0; k < kRayK; ++k) {
        const FF v = warp_sum(ff_of(S[k]));
        if (lane == k) mine = v;
    }
    const FF z = red_zero<FF>();
    FF(*red)[kPartW] = ring_red(smem);
    if (grid_reduce(z, z, z, mine, z, kRayK, false, true, partials, ticket, red) && tid == 0) {
        if (ld_status(status) & kStatusTimeout) return;   // incomplete sums: keep the prices
        const double T = tstride > 1
                             ? lr_s * static_cast<double>((num_full + tstride - 1) / tstride * kTile) /
                                   static_cast<double>(n)
                             : lr_s;
        double x = kRayK - 1;   // log2(s) + 8 of the crossing
        if (!(to_double(red[0][4]) > T)) {
            x = 0.0;
        } else {
            for (int k = 1; k < kRayK; ++k) {
                const double a = to_double(red[0][4 + k - 1]), b = to_double(red[0][4 + k]);
                if (b <= T) {
                    x = (b > 0.0 && isfinite(a)) ? (k - 1) + (log2(a) - log2(T)) / (log2(a) - log2(b))
                                                 : static_cast<double>(k);
                    break;
                }
            }
        }
        const double sc = exp2(x - 8.0);
        for (int j = 0; j < m; ++j) lam[j] *= sc;
    }
}

// Dual values g(lambda_a) and g(lambda_b) in one pass over the data (the
// two start points a warm start chooses between): each job is solved at both
// price vectors from the same staged row.  g_out[0], g_out[1] receive
// lambda^T R + sum_i h_i for each.  With `out` set the pass is also the
// solver's first evaluation at lambda_a: U(X), r and r_lin of a's
// allocation are reduced as in dual_tma_kernel, the EvalOut is filled and
// a's per-job records go to rec_t / rec_j (reported as buffer 1, the one a
// solve's first evaluation writes).
template <int MT, bool CAP>
__global__ void __launch_bounds__(kTile, CAP ? 2 : 3)
    dual_g2_kernel(const float *A, const uint8_t *kind, const float *w, const float *param,
                   const double *R, long long n, int m, const double *lam_a, const double *lam_b,
                   int stages, long long num_full, double *partials, unsigned *ticket, int *status,
                   uint64_t wait_ns, double *g_out, float2 *rec_t, uchar2 *rec_j, EvalOut *out)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bars[kMaxStages];
    __shared__ __align__(16) float la_s[RA_MAX_M], ma_s[RA_MAX_M], lb_s[RA_MAX_M], mb_s[RA_MAX_M];
    __shared__ double lr_s[2];
    __shared__ double lad_s[RA_MAX_M], lbd_s[RA_MAX_M], Rd_s[RA_MAX_M];
    const int tid = threadIdx.x, lane = tid & 31;
    const bool grouped = (m == MT);
    const bool full = out != nullptr;   // the same for the whole grid
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
    KahanF ha, hb, ux, racc, rlin;
    auto job = [&](long long i, bool valid, const float *row, int kd, float wi, float pi,
                   float *warp_rows, const unsigned char *) {
        JobSol<float> sa, sb;
        sa.cP = sa.cQ = -1;
        sa.xP = sa.xQ = 0.f;
        if (valid) {
            solve_job_sm<MT, CAP>(row, ma_s, la_s, m, grouped, rot, kd, wi, pi, sa);
            solve_job_sm<MT, CAP>(row, mb_s, lb_s, m, grouped, rot, kd, wi, pi, sb);
            ha.add(sa.h);
            hb.add(sb.h);
            if (full) {
                ux.add(sa.u);
                rec_t[i] = make_float2(sa.tP, sa.tQ);
                rec_j[i] = make_uchar2(sa.cP >= 0 ? sa.cP : 255, sa.cQ >= 0 ? sa.cQ : 255);
            }
        }
        if (full) {   // every thread: warp collectives
            if (!CAP)
                warp_rsum_lin<MT, KahanF>(warp_rows, m, lane, grouped, rot, sa,
                                          valid && kd >= RA_U_LINCAP, racc, rlin);
            else
                warp_rsum<MT, float, KahanF>(warp_rows, m, lane, grouped, rot, sa, racc);
        }
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
    if (!full) {
        if (grid_reduce(ff_of(ha), ff_of(hb), z, z, z, 0, false, true, partials, ticket, red) &&
            tid == 0) {
            const bool bad = (ld_status(status) & kStatusTimeout) != 0;
            g_out[0] = bad ? nan_d() : lr_s[0] + to_double(red[0][0]);
            g_out[1] = bad ? nan_d() : lr_s[1] + to_double(red[0][1]);
        }
        return;
    }
    const bool lin = !CAP;
    if (!grid_reduce(ff_of(ha), ff_of(ux), ff_of(hb), ff_of(racc), ff_of(rlin), m, lin,
                     grouped ? (lane / MT == 0) : true, partials, ticket, red))
        return;
    const bool bad = (ld_status(status) & kStatusTimeout) != 0;
    if (tid < m) {
        const double r = bad ? nan_d() : to_double(red[0][4 + tid]);
        out->r[tid] = r;
        out->q[tid] = R[tid] - r;
        out->r_lin[tid] = bad ? nan_d() : lin ? to_double(red[0][4 + m + tid]) : 0.0;
    }
    if (tid == 0) {
        const double sumh = bad ? nan_d() : to_double(red[0][0]);
        out->sumh = sumh;
        out->g = lr_s[0] + sumh;
        out->Ux = bad ? nan_d() : to_double(red[0][1]);
        out->Ulb_prev = 0.0;
        out->s2neg = nan_d();   // no own bound for this pass
        out->rec_buf = 1;
        g_out[0] = out->g;
        g_out[1] = bad ? nan_d() : lr_s[1] + to_double(red[0][2]);
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
        unsigned char *base = smem + st * batch_stage_bytes(MT);
        // the previous evaluation's records of the tile come with it when the
        // problem's lagged bound is on (the same flag the consumers read)
        const int pq = B.chunk_prob[prod.c];
        const bool recs = B.lag_on[pq] != 0;
        const int ppq = B.pingpong[pq] & 1;
        mbar_arrive_expect_tx(&bars[st], static_cast<uint32_t>(st_bytes + (recs ? kRecBytes : 0)));
        const uint64_t pol = policy_evict_first();
        bulk_load_stream(base, P.A + j0 * m, static_cast<uint32_t>(a_bytes), &bars[st], pol);
        bulk_load_stream(base + a_bytes, P.w + j0, kTile * 4, &bars[st], pol);
        bulk_load_stream(base + a_bytes + kTile * 4, P.param + j0, kTile * 4, &bars[st], pol);
        bulk_load_stream(base + a_bytes + kTile * 8, P.kind + j0, kTile, &bars[st], pol);
        if (recs) {
            unsigned char *rb = base + StageLayout<MT>::bytes(MT);
            bulk_load(rb, P.lbt[ppq] + j0, kTile * sizeof(float2), &bars[st]);
            bulk_load(rb + kTile * sizeof(float2), P.lbj[ppq] + j0, kTile * sizeof(uchar2), &bars[st]);
        }
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
        const unsigned char *rec_s = nullptr;   // the tile's staged records (full tiles, lag on)
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
            unsigned char *base = smem + st * batch_stage_bytes(MT);
            const size_t a_bytes = static_cast<size_t>(kTile) * m * 4;
            float *a_s = reinterpret_cast<float *>(base);
            row = a_s + tid * m;
            warp_rows = a_s + warp * 32 * m;
            kind = base[a_bytes + kTile * 8 + tid];
            w = reinterpret_cast<const float *>(base + a_bytes)[tid];
            pr = reinterpret_cast<const float *>(base + a_bytes + kTile * 4)[tid];
            if (lag) rec_s = base + StageLayout<MT>::bytes(MT);
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
            if (rec_s != nullptr) {
                tp = reinterpret_cast<const float2 *>(rec_s)[tid];
                jp = reinterpret_cast<const uchar2 *>(rec_s + kTile * sizeof(float2))[tid];
            } else {
                tp = lbt_prev[i];
                jp = lbj_prev[i];
            }
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

// Batched Eq. e-initialization (once per batch solve): each tile's rows are
// copied into shared memory with coalesced 16-byte loads (a thread's own row
// read from global memory would touch a different 128-byte line per lane),
// then read back per thread in rotated 16-byte chunks as in the streaming
// kernels; one FP64 partial per chunk, per-problem ticket and fixed-order
// final sum.
template <int MT>
__global__ void __launch_bounds__(kTile) batch_init_kernel(BatchDualArgs B, double *lam1,
                                                           const long long *lam_off)
{
    __shared__ float x0_s[RA_MAX_M];
    __shared__ FF red[kWarps][kPartW];
    __shared__ int is_last;
    __shared__ __align__(16) float rows[kTile * MT];   // 16-byte chunks are read and written
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
        const bool grouped = (m == MT);
        constexpr int C = MT / 4;
        const int rot = grouped ? ((tid / (32 / MT)) & (C - 1)) : 0;
        for (int k = 0; k < B.chunk_ntiles[c]; ++k) {
            const long long i0 = static_cast<long long>(B.chunk_tile0[c] + k) * kTile;
            const long long i = i0 + tid;
            const bool valid = i < P.n;
            const long long left = P.n - i0;
            const int cnt = static_cast<int>((left < kTile ? left : kTile) * m);
            const float *src = P.A + i0 * m;   // 16-byte aligned: i0 is a multiple of 256
            __syncthreads();   // the previous tile's rows are consumed
            if ((cnt & 3) == 0) {
                for (int e = tid; e < (cnt >> 2); e += kTile)
                    reinterpret_cast<float4 *>(rows)[e] = __ldg(reinterpret_cast<const float4 *>(src) + e);
            } else {
                for (int e = tid; e < cnt; e += kTile) rows[e] = __ldg(src + e);
            }
            __syncthreads();
            // slot k of a holds column colof(k, rot) (rotated 16-byte chunks)
            float a[MT];
            load_row<MT>(a, rows + tid * m, nullptr, i, valid, m, grouped, rot);
            if (!valid) {
#pragma unroll
                for (int k = 0; k < MT; ++k) a[k] = 0.0f;
            }
            float tc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < MT; ++k) tc[k & 3] = fmaf(a[k], x0_s[colof<MT>(k, rot)], tc[k & 3]);
            const float t = (tc[0] + tc[1]) + (tc[2] + tc[3]);
            float d = 0.0f;
            if (valid) {
                const int kd = P.kind[i];
                const float wi = P.w[i], pi = P.param[i];
                if (kd == RA_U_LOG) d = wi / t;
                else if (kd == RA_U_POWER) d = wi * fabsf(pi) * exp2f((pi - 1.0f) * log2f(t));
                else d = t < pi ? wi : 0.0f;
            }
            float *own = rows + tid * m;
            if (grouped) {
#pragma unroll
                for (int cc = 0; cc < C; ++cc)
                    reinterpret_cast<float4 *>(own)[(cc + rot) & (C - 1)] =
                        make_float4(d * a[4 * cc], d * a[4 * cc + 1], d * a[4 * cc + 2], d * a[4 * cc + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < MT; ++j)
                    if (j < m) own[j] = d * a[j];
            }
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

// Per-job throughput records in the per-job precision.
template <typename Real> struct RecOf;
template <> struct RecOf<float> {
    using type = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct RecOf<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

// One thread per job with direct global loads; used for FP64 per-job
// arithmetic (the precision study) and as the generic path.
template <int MT, bool CAP, typename Real, bool LAG, bool REC>
__global__ void __launch_bounds__(kTile)
    dual_simple_kernel(DualParams P)
{
    extern __shared__ __align__(16) unsigned char smem_simple[];
    __shared__ Real lam_s[RA_MAX_M];
    __shared__ Real s_s[RA_MAX_M];
    __shared__ Real sl_s[RA_MAX_M];
    __shared__ double red[kWarps][kPartW];
    __shared__ double lr_s;
    Real *rows = reinterpret_cast<Real *>(smem_simple);  // kTile x m

    if ((P.skip != nullptr && *P.skip != 0) || (P.skip2 != nullptr && *P.skip2 != 0)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = P.m;
    // records in the per-job precision: FP64 job math keeps FP64 throughputs
    // (its buffers are 16 bytes per job), so its lagged bound is FP64 too
    using Rec = typename RecOf<Real>::type;
    const Rec *lbt_prev = reinterpret_cast<const Rec *>(P.lbt_prev);
    const uchar2 *lbj_prev = P.lbj_prev;
    Rec *lbt_out = reinterpret_cast<Rec *>(P.lbt_out);
    uchar2 *lbj_out = P.lbj_out;
    const int q = P.pingpong != nullptr ? (*P.pingpong & 1) : 0;
    if (P.pingpong != nullptr) {
        lbt_prev = reinterpret_cast<const Rec *>(P.lbt_buf[q]);
        lbj_prev = P.lbj_buf[q];
        lbt_out = reinterpret_cast<Rec *>(P.lbt_buf[q ^ 1]);
        lbj_out = P.lbj_buf[q ^ 1];
    }
    const bool lag = LAG && (P.lag_on == nullptr || *P.lag_on != 0);
    const int rec_flag = P.rec_on == nullptr ? 1 : *P.rec_on;
    const bool rec = REC && (rec_flag & 1) != 0;
    const bool own = REC && !CAP && !LAG && rec_flag != 0;
    if (P.pingpong != nullptr && blockIdx.x == 0 && tid == 0) P.out->rec_buf = rec ? (q ^ 1) : -1;
    if (tid < RA_MAX_M) {
        lam_s[tid] = tid < m ? static_cast<Real>(P.lam[tid]) : Fn<Real>::inf();
        s_s[tid] = (lag && tid < m) ? static_cast<Real>(P.s_prev[tid]) : Real(1);
        sl_s[tid] = (lag && tid < m)
                        ? static_cast<Real>((P.s_lin_prev ? P.s_lin_prev : P.s_prev)[tid])
                        : Real(1);
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
                const Rec tp = lbt_prev[i];
                const uchar2 jp = lbj_prev[i];
                const Real *sc = kind >= RA_U_LINCAP ? sl_s : s_s;
                Real tt = Real(0);
                if (jp.x != 255) tt += sc[jp.x] * static_cast<Real>(tp.x);
                if (jp.y != 255) tt += sc[jp.y] * static_cast<Real>(tp.y);
                lbsum += static_cast<double>(util<Real>(kind, w, p, tt));
            }
            if (own && kind == RA_U_POWER && p < Real(0))
                lbsum += static_cast<double>(p * p * fabs(s.u));
            if (rec) {
                lbt_out[i] = RecOf<Real>::make(s.tP, s.tQ);
                lbj_out[i] = make_uchar2(s.cP >= 0 ? s.cP : 255, s.cQ >= 0 ? s.cQ : 255);
            }
        }
        warp_rsum<MT, Real, double>(rows + warp * 32 * m, m, lane, false, 0, s, racc);
        if (!CAP) warp_rlin<Real, double>(valid && kind >= RA_U_LINCAP, lane, s, rlin);
    }
    reduce_and_finalize(hsum, uxsum, lbsum, racc, rlin, m, !CAP, true, P, red, &lr_s, own);
}

// ---------------------------------------------------------------------------- lower bound

// U(X~) = sum_i u_i(s_P t_P + s_Q t_Q), s the column scaling of an evaluation's
// r and r_lin (Section 5; see column_scales), from the compact per-job records.
template <typename Real>
__device__ __forceinline__ void lower_bound_body(const uint8_t *kind, const float *w,
                                                 const float *param, const void *lbt_v,
                                                 const uchar2 *lbj, long long n, int m,
                                                 const EvalOut *src, const double *R, int cap,
                                                 double *partials, unsigned *ticket, double *U_lb)
{
    using Rec = typename RecOf<Real>::type;
    const Rec *lbt = static_cast<const Rec *>(lbt_v);
    __shared__ Real s_s[RA_MAX_M];
    __shared__ Real sl_s[RA_MAX_M];
    __shared__ double red[kWarps];
    __shared__ int is_last;
    const int tid = threadIdx.x;
    if (tid < RA_MAX_M) {
        Real s = Real(1), sl = Real(1);
        if (tid < m) {
            double sd, sld;
            column_scales(R[tid], src->r[tid], src->r_lin[tid], cap, sd, sld);
            s = static_cast<Real>(sd);
            sl = static_cast<Real>(sld);
        }
        s_s[tid] = s;
        sl_s[tid] = sl;
    }
    __syncthreads();
    typename std::conditional<sizeof(Real) == 8, double, KahanF>::type acc{};
    auto add_job = [&](int kd, float wi, float pi, uchar2 jp, Real tP, Real tQ) {
        const Real *sc = kd >= RA_U_LINCAP ? sl_s : s_s;
        Real tt = Real(0);
        if (jp.x != 255) tt += sc[jp.x] * tP;
        if (jp.y != 255) tt += sc[jp.y] * tQ;
        acc_add(acc, util<Real>(kd, static_cast<Real>(wi), static_cast<Real>(pi), tt));
    };
    const long long nthr = static_cast<long long>(gridDim.x) * kTile;
    const long long gtid = static_cast<long long>(blockIdx.x) * kTile + tid;
    if constexpr (sizeof(Real) == 4) {
        // FP32 records: a thread takes four consecutive jobs at a time with
        // 16-, 8- and 4-byte loads (records, their columns, kinds, weights,
        // parameters: 76 bytes), two such groups in flight; all five arrays
        // are at least 16-byte aligned
        const long long ng = n >> 2;
        const float4 *t4 = reinterpret_cast<const float4 *>(lbt);
        const uint2 *j4 = reinterpret_cast<const uint2 *>(lbj);
        const uint32_t *k4 = reinterpret_cast<const uint32_t *>(kind);
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        const float4 *p4 = reinterpret_cast<const float4 *>(param);
        constexpr int kG = 2;
        for (long long g0 = gtid; g0 < ng; g0 += kG * nthr) {
            float4 ta[kG], tb[kG], wv[kG], pv[kG];
            uint2 jj[kG];
            uint32_t kk[kG];
#pragma unroll
            for (int u = 0; u < kG; ++u) {
                const long long gi = g0 + u * nthr;
                if (gi < ng) {
                    ta[u] = t4[2 * gi];
                    tb[u] = t4[2 * gi + 1];
                    jj[u] = j4[gi];
                    kk[u] = k4[gi];
                    wv[u] = w4[gi];
                    pv[u] = p4[gi];
                }
            }
#pragma unroll
            for (int u = 0; u < kG; ++u) {
                if (g0 + u * nthr >= ng) continue;
                const uchar2 c0 = make_uchar2(jj[u].x & 255u, (jj[u].x >> 8) & 255u);
                const uchar2 c1 = make_uchar2((jj[u].x >> 16) & 255u, jj[u].x >> 24);
                const uchar2 c2 = make_uchar2(jj[u].y & 255u, (jj[u].y >> 8) & 255u);
                const uchar2 c3 = make_uchar2((jj[u].y >> 16) & 255u, jj[u].y >> 24);
                add_job(kk[u] & 255u, wv[u].x, pv[u].x, c0, ta[u].x, ta[u].y);
                add_job((kk[u] >> 8) & 255u, wv[u].y, pv[u].y, c1, ta[u].z, ta[u].w);
                add_job((kk[u] >> 16) & 255u, wv[u].z, pv[u].z, c2, tb[u].x, tb[u].y);
                add_job(kk[u] >> 24, wv[u].w, pv[u].w, c3, tb[u].z, tb[u].w);
            }
        }
        // the last n mod 4 jobs
        const long long i = (ng << 2) + gtid;
        if (i < n) add_job(kind[i], w[i], param[i], lbj[i], lbt[i].x, lbt[i].y);
    } else {
        // FP64 records: one job per thread and trip, kU trips in flight
        constexpr int kU = 4;
        for (long long i0 = gtid; i0 < n; i0 += kU * nthr) {
            Rec tp[kU];
            uchar2 jp[kU];
            int kd[kU];
            float wv[kU], pv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const long long i = i0 + u * nthr;
                const bool in = i < n;
                tp[u] = in ? lbt[i] : Rec{};
                jp[u] = in ? lbj[i] : make_uchar2(255, 255);
                kd[u] = in ? static_cast<int>(kind[i]) : -1;
                wv[u] = in ? w[i] : 0.f;
                pv[u] = in ? param[i] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (kd[u] >= 0) add_job(kd[u], wv[u], pv[u], jp[u], tp[u].x, tp[u].y);
        }
    }
    const double accd = warp_sum_d(acc_value(acc));
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
    if (!is_last) return;
    // grid stage, all threads of the last CTA: thread t adds partials t,
    // t + 256, ... in order, then the warps' butterflies and warp order --
    // a fixed order, so the bound is deterministic
    __threadfence();
    double v = 0.0;
    for (unsigned b = tid; b < gridDim.x; b += kTile) v += __ldcg(&partials[b]);
    v = warp_sum_d(v);
    __syncthreads();   // red[] is reused
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += red[k];
        *U_lb = isnan(src->sumh) ? src->sumh : t;   // the evaluation it scales was incomplete
        *ticket = 0u;
    }
}

template <typename Real>
__global__ void __launch_bounds__(kTile)
    lower_bound_kernel(const uint8_t *kind, const float *w, const float *param, const void *lbt_v,
                       const uchar2 *lbj, long long n, int m, const EvalOut *src, const double *R,
                       int cap, double *partials, unsigned *ticket, double *U_lb)
{
    lower_bound_body<Real>(kind, w, param, lbt_v, lbj, n, m, src, R, cap, partials, ticket, U_lb);
}

// The solver's lower-bound pass: the records the evaluation `src` wrote (the
// buffer it names in src->rec_buf; nothing when it wrote none) into slot
// U_slot[src->rec_buf].  It runs beside the price update of the same
// evaluation, which reads the other slot (the previous evaluation's bound).
template <typename Real>
__global__ void __launch_bounds__(kTile)
    lagged_bound_kernel(const uint8_t *kind, const float *w, const float *param,
                        const void *lbt0, const void *lbt1, const uchar2 *lbj0, const uchar2 *lbj1,
                        long long n, int m, const EvalOut *src, const double *R, int cap,
                        double *partials, unsigned *ticket, double *U_slot, const int32_t *skip)
{
    if (skip != nullptr && *skip != 0) return;
    const int b = src->rec_buf;
    if (b < 0) return;
    lower_bound_body<Real>(kind, w, param, b ? lbt1 : lbt0, b ? lbj1 : lbj0, n, m, src, R, cap,
                           partials, ticket, U_slot + b);
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

template <typename Rec>
__global__ void records_kernel(const Rec *lbt, const uchar2 *lbj, long long n, int32_t *j12,
                               float *t12)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const uchar2 j = lbj[i];
        const Rec t = lbt[i];
        j12[2 * i] = j.x == 255 ? -1 : j.x;
        j12[2 * i + 1] = j.y == 255 ? -1 : j.y;
        t12[2 * i] = static_cast<float>(t.x);
        t12[2 * i + 1] = static_cast<float>(t.y);
    }
}

// ---------------------------------------------------------------------------- dispatch

// Ring stages for a shared-memory budget per CTA: 106 KB lets two CTAs share
// an SM (the capped kernels, 128 registers), 70 KB three (the uncapped ones).

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
    // three CTAs per SM (two for the capped walk from 16 columns, whose
    // registers would spill at three); a stage also holds the tile's 2.5 KB
    // of records
    const size_t budget = (cap && p->mt >= 16) ? 111 * 1024 : 70 * 1024;
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
#define RA_RATTR(MT)                                                                               \
    if ((e = cudaFuncSetAttribute(ray_scale_kernel<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  kRingSmemMax)) != cudaSuccess)                                     \
        return e;
    RA_RATTR(4)
    RA_RATTR(8)
    RA_RATTR(16)
    RA_RATTR(32)
#undef RA_RATTR
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
    // the initial-price and ray-scaling passes hold more registers per thread
    // (fewer CTAs fit an SM); their persistent grids must fit in one wave
    const void *fi = nullptr, *fr = nullptr;
    switch (p->mt) {
    case 4: fi = reinterpret_cast<const void *>(init_tma_kernel<4>);
            fr = reinterpret_cast<const void *>(ray_scale_kernel<4>); break;
    case 8: fi = reinterpret_cast<const void *>(init_tma_kernel<8>);
            fr = reinterpret_cast<const void *>(ray_scale_kernel<8>); break;
    case 16: fi = reinterpret_cast<const void *>(init_tma_kernel<16>);
             fr = reinterpret_cast<const void *>(ray_scale_kernel<16>); break;
    default: fi = reinterpret_cast<const void *>(init_tma_kernel<32>);
             fr = reinterpret_cast<const void *>(ray_scale_kernel<32>); break;
    }
    int per_i = 1, per_r = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_i, fi, kTile, p->smem_dual)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_r, fr, kTile, p->smem_dual)) != cudaSuccess)
        return e;
    p->grid_init = p->num_sms * (per_i < 1 ? 1 : per_i);
    p->grid_ray = p->num_sms * (per_r < 1 ? 1 : per_r);
    if (p->grid_init > p->grid_dual) p->grid_init = p->grid_dual;
    if (p->grid_ray > p->grid_dual) p->grid_ray = p->grid_dual;
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

// g(lambda) with FP64 per-job arithmetic whatever the problem's flags (no
// records, no lagged bound): the exact check of a gap that FP32 arithmetic
// can only estimate.
cudaError_t launch_dual_exact(const ra_problem *p, const double *lam, EvalOut *out, cudaStream_t s)
{
    DualParams dp{};
    dp.A = p->A;
    dp.kind = p->kind;
    dp.w = p->w;
    dp.param = p->param;
    dp.R = p->R;
    dp.n = p->n;
    dp.m = p->m;
    dp.lam = lam;
    dp.partials = p->partials;
    dp.ticket = p->ticket + 7;
    dp.status = p->status;
    dp.out = out;
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
    switch (p->mt) {
    case 4: return cap ? launch_simple<4, true, double, false, false>(p, dp, s) : launch_simple<4, false, double, false, false>(p, dp, s);
    case 8: return cap ? launch_simple<8, true, double, false, false>(p, dp, s) : launch_simple<8, false, double, false, false>(p, dp, s);
    case 16: return cap ? launch_simple<16, true, double, false, false>(p, dp, s) : launch_simple<16, false, double, false, false>(p, dp, s);
    default: return cap ? launch_simple<32, true, double, false, false>(p, dp, s) : launch_simple<32, false, double, false, false>(p, dp, s);
    }
}

cudaError_t launch_lower_bound(const ra_problem *p, const float2 *lbt, const uchar2 *lbj,
                               const EvalOut *src, double *U_lb, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    if (p->flags & RA_FP64_JOBMATH)
        lower_bound_kernel<double><<<static_cast<int>(blocks), kTile, 0, s>>>(
            p->kind, p->w, p->param, lbt, lbj, p->n, p->m, src, p->R, !(p->flags & RA_NO_JOB_CAP),
            p->partials, p->ticket + 1, U_lb);
    else
        lower_bound_kernel<float><<<static_cast<int>(blocks), kTile, 0, s>>>(
            p->kind, p->w, p->param, lbt, lbj, p->n, p->m, src, p->R, !(p->flags & RA_NO_JOB_CAP),
            p->partials, p->ticket + 1, U_lb);
    return cudaGetLastError();
}

cudaError_t launch_lagged_bound(const ra_problem *p, const int32_t *skip, cudaStream_t s)
{
    // two CTAs per SM: the solver step (one CTA, ~110 registers a thread)
    // launched beside this pass must still find room on an SM
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > 2LL * p->num_sms) blocks = 2LL * p->num_sms;
    const int cap = !(p->flags & RA_NO_JOB_CAP);
    if (p->flags & RA_FP64_JOBMATH)
        lagged_bound_kernel<double><<<static_cast<int>(blocks), kTile, 0, s>>>(
            p->kind, p->w, p->param, p->lbt[0], p->lbt[1], p->lbj[0], p->lbj[1], p->n, p->m, p->ev,
            p->R, cap, p->partials, p->ticket + 1, p->lb_slot, skip);
    else
        lagged_bound_kernel<float><<<static_cast<int>(blocks), kTile, 0, s>>>(
            p->kind, p->w, p->param, p->lbt[0], p->lbt[1], p->lbj[0], p->lbj[1], p->n, p->m, p->ev,
            p->R, cap, p->partials, p->ticket + 1, p->lb_slot, skip);
    return cudaGetLastError();
}

cudaError_t launch_records(const ra_problem *p, int32_t *j12, float *t12, cudaStream_t s)
{
    long long blocks = (p->n + kTile - 1) / kTile;
    if (blocks > p->grid_aux) blocks = p->grid_aux;
    if (p->flags & RA_FP64_JOBMATH)
        records_kernel<<<static_cast<int>(blocks), kTile, 0, s>>>(
            reinterpret_cast<const double2 *>(p->lbt[0]), p->lbj[0], p->n, j12, t12);
    else
        records_kernel<<<static_cast<int>(blocks), kTile, 0, s>>>(p->lbt[0], p->lbj[0], p->n, j12, t12);
    return cudaGetLastError();
}

cudaError_t launch_dual_g2(const ra_problem *p, const double *lam_a, const double *lam_b,
                           double *g_out, bool first_eval, cudaStream_t s)
{
    float2 *rt = first_eval ? p->lbt[1] : nullptr;
    uchar2 *rj = first_eval ? p->lbj[1] : nullptr;
    EvalOut *ev = first_eval ? p->ev : nullptr;
    const long long num_full = p->n / kTile;
    int grid = p->grid_dual;
    if (num_full < grid) grid = static_cast<int>(num_full > 0 ? num_full : 1);
    const bool cap = !(p->flags & RA_NO_JOB_CAP);
#define RA_G2(MT)                                                                                  \
    if (cap)                                                                                       \
        dual_g2_kernel<MT, true><<<grid, kTile, p->smem_dual, s>>>(                                \
            p->A, p->kind, p->w, p->param, p->R, p->n, p->m, lam_a, lam_b, p->stages, num_full,    \
            p->partials, p->ticket + 3, p->status, wait_limit_ns(), g_out, rt, rj, ev);            \
    else                                                                                           \
        dual_g2_kernel<MT, false><<<grid, kTile, p->smem_dual, s>>>(                               \
            p->A, p->kind, p->w, p->param, p->R, p->n, p->m, lam_a, lam_b, p->stages, num_full,    \
            p->partials, p->ticket + 3, p->status, wait_limit_ns(), g_out, rt, rj, ev);
    switch (p->mt) {
    case 4: RA_G2(4) break;
    case 8: RA_G2(8) break;
    case 16: RA_G2(16) break;
    default: RA_G2(32) break;
    }
#undef RA_G2
    return cudaGetLastError();
}

cudaError_t launch_init(const ra_problem *p, double *lam1, cudaStream_t s, long long n_all,
                        long long tstride)
{
    if (n_all <= 0) n_all = p->n;
    const long long num_full = p->n / kTile;
    if (tstride < 1 || num_full < tstride) tstride = 1;
    int grid = p->grid_init;
    const long long tiles = (num_full + tstride - 1) / tstride;
    if (tiles < grid) grid = static_cast<int>(tiles > 0 ? tiles : 1);
    const int cap = !(p->flags & RA_NO_JOB_CAP);
#define RA_INIT(MT)                                                                                \
    init_tma_kernel<MT><<<grid, kTile, p->smem_dual, s>>>(p->A, p->kind, p->w, p->param, p->R,      \
                                                          p->n, p->m, cap, p->stages, num_full,    \
                                                          p->partials, p->ticket + 2, p->status,   \
                                                          wait_limit_ns(), n_all, lam1, tstride)
    switch (p->mt) {
    case 4: RA_INIT(4); break;
    case 8: RA_INIT(8); break;
    case 16: RA_INIT(16); break;
    default: RA_INIT(32); break;
    }
#undef RA_INIT
    return cudaGetLastError();
}

cudaError_t launch_ray_scale(const ra_problem *p, double *lam, cudaStream_t s, long long tstride)
{
    const long long num_full = p->n / kTile;
    if (tstride < 1 || num_full < tstride) tstride = 1;
    int grid = p->grid_ray;
    const long long tiles = (num_full + tstride - 1) / tstride;
    if (tiles < grid) grid = static_cast<int>(tiles > 0 ? tiles : 1);
#define RA_RAY(MT)                                                                                 \
    ray_scale_kernel<MT><<<grid, kTile, p->smem_dual, s>>>(p->A, p->kind, p->w, p->param, p->R,     \
                                                           p->n, p->m, lam, p->stages, num_full,   \
                                                           p->partials, p->ticket + 6, p->status,  \
                                                           wait_limit_ns(), tstride)
    switch (p->mt) {
    case 4: RA_RAY(4); break;
    case 8: RA_RAY(8); break;
    case 16: RA_RAY(16); break;
    default: RA_RAY(32); break;
    }
#undef RA_RAY
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
    int s = static_cast<int>(budget / batch_stage_bytes(mt));
    if (s > kMaxStages) s = kMaxStages;
    if (s < 2) s = 2;
    return s;
}

size_t batch_smem(int mt, int cap) { return batch_stages(mt, cap) * batch_stage_bytes(mt) + 128; }

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
