// Learned warm start: per-resource summary statistics of a problem, the shared
// per-resource MLP 26 -> 256 -> 256 -> 1 (GELU) that maps them to log prices,
// its training step (mean squared error on log lambda*, back-propagation,
// Adam), and the start-price choice between the network's prices and the
// paper's Eq. e-initialization by the smaller dual value g.
//
// All arithmetic is FP32 except the reductions of the statistics (FP64) and
// the dual evaluations (the library's dual pass).  Every sum runs in a fixed
// order, so results are bitwise reproducible.

#include <cmath>
#include <cstring>

#include "ra_internal.cuh"

namespace ra {
namespace {

constexpr int kFeatRes = RA_MLP_STATS;     // statistics per resource
constexpr int kFeatIn = RA_MLP_IN;         // network input per resource
constexpr int kHid = RA_MLP_HIDDEN;
constexpr int kQuant = 8;
constexpr int kSampleMax = 16384;
constexpr int oW1 = 0;
constexpr int ob1 = oW1 + kFeatIn * kHid;
constexpr int oW2 = ob1 + kHid;
constexpr int ob2 = oW2 + kHid * kHid;
constexpr int oW3 = ob2 + kHid;
constexpr int ob3 = oW3 + kHid;
static_assert(ob3 + 1 == RA_MLP_PARAMS, "parameter layout");

// ---------------------------------------------------------------------------- statistics

// Rows of the sample: all rows when n <= 16384, else i_k = floor(k n / 16384).
__device__ __forceinline__ long long sample_row(long long k, long long n, int S)
{
    return k * n / S;
}

// Order-preserving map of a float to an unsigned key (NaN excluded).
__device__ __forceinline__ unsigned fkey(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float fkey_inv(unsigned k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Statistics of problem blockIdx.y: the 8 quantiles of A[:, j] over the
// sample (order statistics of rank floor((2l+1) S / 16), selected exactly by
// a radix select over the float's order-preserving key, 8 bits a pass:
// integer bin counts, so the selection does not depend on thread timing) and
// log(R_j / n) of every resource j, and the fractions of log, power and linear
// utilities and the mean of log w over the sample (every resource's row).
// Work split: with nq = kQuant a CTA selects all 8 quantiles of resource
// blockIdx.x (CTA m: the shared statistics); with nq = 1 (a single problem,
// whose 8 selections would otherwise run on m SMs only) CTA 8 j + l selects
// quantile l of resource j and CTA 8 m the shared statistics.
__global__ void __launch_bounds__(1024) stats_kernel(const FeatProblem *probs, FeatProblem one,
                                                     float *stats, int nq)
{
    extern __shared__ unsigned key[];   // kSampleMax keys
    __shared__ double red[32][3];
    __shared__ unsigned hist[kQuant][256];
    __shared__ unsigned pref[kQuant];   // key bits fixed so far
    __shared__ unsigned rank[kQuant];   // rank within the keys matching pref
    const FeatProblem P = probs ? probs[blockIdx.y] : one;
    const int per = kQuant / nq;        // CTAs per resource
    const int j = blockIdx.x / per;
    const int l0 = (blockIdx.x % per) * nq;   // first quantile of this CTA
    if (j > P.m || (j == P.m && l0 != 0)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long n = P.n;
    const int S = n < kSampleMax ? static_cast<int>(n) : kSampleMax;
    if (j == P.m) {
        // the statistics every resource shares (utility mix, mean log w), once
        // per problem: integer counts and compensated FP32 sums (the FP64
        // pipe is slow on this GPU), FP64 across warps in a fixed order
        int cl = 0, cp = 0;
        float sw = 0.f, cw = 0.f;
        for (int k = tid; k < S; k += blockDim.x) {
            const long long row = sample_row(k, n, S);
            const int kd = P.kind[row];
            cl += kd == RA_U_LOG;
            cp += kd == RA_U_POWER;
            const float y = logf(fmaxf(P.w[row], 1e-30f)) - cw;
            const float t = sw + y;
            cw = (t - sw) - y;
            sw = t;
        }
        cl = __reduce_add_sync(0xffffffffu, cl);
        cp = __reduce_add_sync(0xffffffffu, cp);
        double swd = static_cast<double>(sw) - static_cast<double>(cw);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) swd += __shfl_xor_sync(0xffffffffu, swd, off);
        if (lane == 0) {
            red[warp][0] = cl;
            red[warp][1] = cp;
            red[warp][2] = swd;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0, c = 0.0;
            const int nw = (blockDim.x + 31) / 32;
            for (int w2 = 0; w2 < nw; ++w2) {
                a += red[w2][0];
                b += red[w2][1];
                c += red[w2][2];
            }
            for (int jj = 0; jj < P.m; ++jj) {
                float *o2 = stats + (P.row0 + jj) * kFeatRes;
                o2[9] = static_cast<float>(a / S);
                o2[10] = static_cast<float>(b / S);
                o2[11] = static_cast<float>((S - a - b) / S);
                o2[12] = static_cast<float>(c / S);
            }
        }
        return;
    }
    {
        // the sampled rows are scattered over A: eight loads in flight per
        // thread before their keys are stored
        constexpr int kB = 8;
        int k = tid;
        for (; k + (kB - 1) * static_cast<int>(blockDim.x) < S; k += kB * blockDim.x) {
            float v[kB];
#pragma unroll
            for (int b = 0; b < kB; ++b) v[b] = P.A[sample_row(k + b * blockDim.x, n, S) * P.m + j];
#pragma unroll
            for (int b = 0; b < kB; ++b) key[k + b * blockDim.x] = fkey(v[b]);
        }
        for (; k < S; k += blockDim.x) key[k] = fkey(P.A[sample_row(k, n, S) * P.m + j]);
    }
    if (tid < nq) {
        pref[tid] = 0u;
        rank[tid] = static_cast<unsigned>(((2 * (l0 + tid) + 1) * S) / 16);
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int e = tid; e < kQuant * 256; e += blockDim.x) (&hist[0][0])[e] = 0u;
        __syncthreads();
        // first pass: warp-aggregated counts, the lanes holding the same bin
        // add once (a column's values share few exponents, so per-key atomics
        // would pile onto a handful of bins)
        const int kend = (S + 31) & ~31;
        for (int k = tid; k < kend; k += blockDim.x) {
            const bool in = k < S;
            const unsigned kv = in ? key[k] : 0u;
            const unsigned bin = (kv >> shift) & 255u;
            if (pass == 0) {   // the same histogram serves every rank
                const unsigned grp = __match_any_sync(0xffffffffu, in ? bin : 0xffffffffu);
                if (in && (__ffs(grp) - 1) == lane) atomicAdd(&hist[0][bin], __popc(grp));
            } else {   // few keys still match a rank's prefix: plain atomics
                for (int l = 0; l < nq; ++l)
                    if (in && ((kv ^ pref[l]) >> (shift + 8)) == 0u) atomicAdd(&hist[l][bin], 1u);
            }
        }
        __syncthreads();
        if (warp < nq) {   // warp l finds the bin holding its rank
            const unsigned *h = hist[pass == 0 ? 0 : warp];
            unsigned c[8], tot = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = h[lane * 8 + q];
                tot += c[q];
            }
            unsigned incl = tot;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const unsigned excl = incl - tot;
            const unsigned r = rank[warp];
            const bool mine = r >= excl && r < incl;
            const unsigned owner = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                unsigned before = excl;
                int q = 0;
                while (q < 7 && r >= before + c[q]) before += c[q++];
                pref[warp] |= static_cast<unsigned>(lane * 8 + q) << shift;
                rank[warp] = r - before;
            }
            (void)owner;
        }
        __syncthreads();
    }
    float *out = stats + (P.row0 + j) * kFeatRes;
    if (tid < nq) out[l0 + tid] = logf(fmaxf(fkey_inv(pref[tid]), 1e-30f));
    if (tid == kQuant && l0 == 0)
        out[8] = static_cast<float>(log(fmax(P.R[j] / static_cast<double>(n), 1e-30)));
}

// Network input of every resource of problem blockIdx.x: its statistics,
// then their mean over the problem's resources (FP64, resource order).
__global__ void features_kernel(const FeatProblem *probs, FeatProblem one, const float *stats,
                                float *feats)
{
    const FeatProblem P = probs ? probs[blockIdx.x] : one;
    __shared__ float mean[kFeatRes];
    if (threadIdx.x < kFeatRes) {
        double s = 0.0;
        for (int j = 0; j < P.m; ++j) s += stats[(P.row0 + j) * kFeatRes + threadIdx.x];
        mean[threadIdx.x] = static_cast<float>(s / P.m);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < P.m * kFeatIn; idx += blockDim.x) {
        const int j = idx / kFeatIn, c = idx % kFeatIn;
        feats[(P.row0 + j) * kFeatIn + c] = c < kFeatRes ? stats[(P.row0 + j) * kFeatRes + c]
                                                         : mean[c - kFeatRes];
    }
}

// ---------------------------------------------------------------------------- MLP

__device__ __forceinline__ float gelu(float z)
{
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
           z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

enum { kEpiStore = 0, kEpiBiasGelu = 1, kEpiGeluGrad = 2 };

// C (M x N) = op(A) (M x K) * op(B) (K x N) in FP32, A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn]; 64 x 64 tiles, 16-deep k slices staged in shared
// memory, 4 x 4 outputs per thread, k summed in order (deterministic).
// Epilogues: store; z = acc + bias -> Z, GELU(z) -> H; acc * GELU'(Z) -> C.
template <int EPI>
__global__ void __launch_bounds__(256)
    gemm_kernel(int M, int N, int K, const float *A, long long sam, long long sak, const float *B,
                long long sbk, long long sbn, float *C, long long ldc, const float *bias, float *Z,
                float *H)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn) acc[i][jn] = 0.0f;
    const bool a_mfast = sam == 1;  // consecutive threads walk the unit stride
    const bool b_kfast = sbk == 1;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 1024; e += 256) {
            const int mm = a_mfast ? (e & 63) : (e >> 4);
            const int kk = a_mfast ? (e >> 6) : (e & 15);
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[gm * sam + gk * sak] : 0.0f;
        }
        for (int e = tid; e < 1024; e += 256) {
            const int nn = b_kfast ? (e >> 4) : (e & 63);
            const int kk = b_kfast ? (e & 15) : (e >> 6);
            const int gk = k0 + kk, gn = n0 + nn;
            Bs[kk][nn] = (gk < K && gn < N) ? B[gk * sbk + gn * sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int jn = 0; jn < 4; ++jn) b[jn] = Bs[kk][tx + 16 * jn];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) acc[i][jn] = fmaf(a[i], b[jn], acc[i][jn]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int jn = 0; jn < 4; ++jn) {
            const int gn = n0 + tx + 16 * jn;
            if (gn >= N) continue;
            const long long o = gm * ldc + gn;
            if (EPI == kEpiStore) {
                C[o] = acc[i][jn];
            } else if (EPI == kEpiBiasGelu) {
                const float z = acc[i][jn] + bias[gn];
                Z[o] = z;
                H[o] = gelu(z);
            } else {
                C[o] = acc[i][jn] * gelu_grad(Z[o]);
            }
        }
    }
}

// Few-row layer (inference on one problem's resources): CTA r computes row r,
// thread c output column c, z = sum_k x_rk W_kc in order k = 0..K-1 with the
// same fused multiply-adds as gemm_kernel, so both give identical bits; then
// z + bias -> Z and GELU -> H.  Needs N == blockDim.x.
__global__ void __launch_bounds__(256)
    rows_bias_gelu_kernel(int K, int N, const float *X, const float *W, const float *bias, float *Z,
                          float *H)
{
    extern __shared__ float xr[];
    const int r = blockIdx.x, c = threadIdx.x;
    for (int k = c; k < K; k += blockDim.x) xr[k] = X[static_cast<long long>(r) * K + k];
    __syncthreads();
    float acc = 0.0f;
    for (int k = 0; k < K; ++k) acc = fmaf(xr[k], W[static_cast<long long>(k) * N + c], acc);
    const float z = acc + bias[c];
    Z[static_cast<long long>(r) * N + c] = z;
    H[static_cast<long long>(r) * N + c] = gelu(z);
}

// Inference on one problem's resources (few rows), the whole network in one
// launch: CTA r computes row r.  Its latency is the chain of dependent L2
// loads of W2 (256 per output unit), so each hidden unit of the second layer
// is split over four threads (quarter g sums k in [64g, 64g + 64) in order)
// and the quarters are added in order g = 0..3; layer 1 and the head as in
// the training path.  The result differs from the training path's forward
// only by that summation order (a few FP32 ulps).
constexpr int kInferSplit = 4;

// The network on one input row xr (shared memory, kFeatIn floats), all
// kHid * kInferSplit threads of the CTA taking part; thread 0 gets y.
__device__ __forceinline__ float mlp_row(const float *xr, const float *theta, float *h1, float *h2,
                                         float (*part)[kHid])
{
    const int t = threadIdx.x;
    const int c = t % kHid, g = t / kHid;
    if (g == 0) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < kFeatIn; ++k) acc = fmaf(xr[k], theta[oW1 + k * kHid + c], acc);
        h1[c] = gelu(acc + theta[ob1 + c]);
    }
    __syncthreads();
    constexpr int KQ = kHid / kInferSplit;
    float acc = 0.0f;
#pragma unroll 16
    for (int k = g * KQ; k < (g + 1) * KQ; ++k) acc = fmaf(h1[k], theta[oW2 + k * kHid + c], acc);
    part[g][c] = acc;
    __syncthreads();
    if (g == 0) {
        float z = part[0][c];
#pragma unroll
        for (int q = 1; q < kInferSplit; ++q) z += part[q][c];
        h2[c] = gelu(z + theta[ob2 + c]);
    }
    __syncthreads();
    float s2 = 0.0f;
    if (t < 32) {
#pragma unroll
        for (int k = 0; k < kHid / 32; ++k) s2 = fmaf(h2[t + 32 * k], theta[oW3 + t + 32 * k], s2);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    return s2 + theta[ob3];
}

__global__ void __launch_bounds__(kHid * kInferSplit) infer_rows_kernel(const float *X, const float *theta, float *y)
{
    __shared__ float xr[kFeatIn];
    __shared__ float h1[kHid];
    __shared__ float h2[kHid];
    __shared__ float part[kInferSplit][kHid];
    const int r = blockIdx.x, t = threadIdx.x;
    if (t < kFeatIn) xr[t] = X[static_cast<long long>(r) * kFeatIn + t];
    __syncthreads();
    const float v = mlp_row(xr, theta, h1, h2, part);
    if (t == 0) y[r] = v;
}

// The warm start's whole network step for one problem's m resources, CTA r
// for resource r: its input row (its 13 statistics, then their mean over the
// resources, summed in FP64 in resource order as features_kernel does), the
// network, and the start price max(exp(y) - RA_MLP_PRICE_OFFSET, 0) -- the
// work of features_kernel, infer_rows_kernel and exp_prices_kernel in one
// launch.
__global__ void __launch_bounds__(kHid * kInferSplit)
    warm_infer_kernel(const float *stats, int m, const float *theta, float *feats, float *y,
                      double *lam)
{
    __shared__ float xr[kFeatIn];
    __shared__ float h1[kHid];
    __shared__ float h2[kHid];
    __shared__ float part[kInferSplit][kHid];
    const int r = blockIdx.x, t = threadIdx.x;
    if (t < kFeatRes) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += stats[j * kFeatRes + t];
        xr[kFeatRes + t] = static_cast<float>(s / m);
        xr[t] = stats[r * kFeatRes + t];
    }
    __syncthreads();
    if (t < kFeatIn) feats[r * kFeatIn + t] = xr[t];
    const float v = mlp_row(xr, theta, h1, h2, part);
    if (t == 0) {
        y[r] = v;
        lam[r] = fmax(exp(static_cast<double>(v)) - RA_MLP_PRICE_OFFSET, 0.0);
    }
}

// y_r = h2_r . W3 + b3, one warp per row, lanes in a fixed butterfly.
__global__ void head_kernel(int rows, const float *h2, const float *theta, float *y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const float *h = h2 + static_cast<long long>(warp) * kHid;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kHid / 32; ++k) s = fmaf(h[lane + 32 * k], theta[oW3 + lane + 32 * k], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) y[warp] = s + theta[ob3];
}

// Mean squared error and dL/dy = 2 (y - t) / rows; dL/db3 = sum dL/dy.  One
// CTA, FP64 partial sums in thread order.
__global__ void __launch_bounds__(1024)
    loss_kernel(int rows, const float *y, const float *target, float *dy, float *grad, float *loss)
{
    __shared__ double s1[1024], s2[1024];
    const int tid = threadIdx.x;
    double a = 0.0, b = 0.0;
    const float inv = 2.0f / static_cast<float>(rows);
    for (int r = tid; r < rows; r += blockDim.x) {
        const float e = y[r] - target[r];
        const float d = inv * e;
        dy[r] = d;
        a += static_cast<double>(e) * e;
        b += d;
    }
    s1[tid] = a;
    s2[tid] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (tid < h) {
            s1[tid] += s1[tid + h];
            s2[tid] += s2[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        grad[ob3] = static_cast<float>(s2[0]);
        if (loss) *loss = static_cast<float>(s1[0] / rows);
    }
}

// out[c] = sum_r X[r, c] (* wv[r] when wv is given): 32 columns x 8 row
// groups per CTA, row group g takes rows g, g+8, ...; groups added in order.
__global__ void colsum_kernel(int rows, int cols, const float *X, const float *wv, float *out)
{
    __shared__ float part[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x, g = threadIdx.y;
    float s = 0.0f;
    if (c < cols)
        for (int r = g; r < rows; r += 8) {
            const float v = X[static_cast<long long>(r) * cols + c];
            s = wv ? fmaf(v, wv[r], s) : s + v;
        }
    part[g][threadIdx.x] = s;
    __syncthreads();
    if (g == 0 && c < cols) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
        out[c] = t;
    }
}

// dz2[r, k] = dy[r] W3[k] GELU'(z2[r, k])
__global__ void head_back_kernel(int rows, const float *dy, const float *theta, const float *z2,
                                 float *dz2)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<long long>(rows) * kHid) return;
    const int r = static_cast<int>(i / kHid), k = static_cast<int>(i % kHid);
    dz2[i] = dy[r] * theta[oW3 + k] * gelu_grad(z2[i]);
}

// Adam (Kingma and Ba 2015, Algorithm 1); c1 = 1/(1 - b1^t), c2 = 1/(1 - b2^t).
__global__ void adam_kernel(int np, float *theta, const float *grad, float *m1, float *m2, float lr,
                            float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.0f - b1) * g;
    const float v = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    theta[i] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
}

__global__ void exp_prices_kernel(int m, const float *y, double *lam)
{
    const int j = threadIdx.x;
    if (j < m) lam[j] = fmax(exp(static_cast<double>(y[j])) - RA_MLP_PRICE_OFFSET, 0.0);
}

// Start prices: the network's when their dual value is finite and not larger
// than that of the cold start (the fallback keeps Eq. e-initialization).
__global__ void choose_kernel(int m, const double *lam_w, const double *lam_c, const double *g2,
                              double *lam0, int32_t *used)
{
    const bool warm = isfinite(g2[0]) && !(g2[0] > g2[1]);
    const int j = threadIdx.x;
    if (j < m) lam0[j] = warm ? lam_w[j] : lam_c[j];
    if (j == 0) *used = warm ? 1 : 0;
}

template <int EPI>
cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float *A, long long sam, long long sak,
                 const float *B, long long sbk, long long sbn, float *C, long long ldc,
                 const float *bias = nullptr, float *Z = nullptr, float *H = nullptr)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<EPI><<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, Z, H);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_features(const FeatProblem *probs, const FeatProblem &one, int P, int m_max,
                            float *stats, float *feats, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSampleMax * 4);
    if (e != cudaSuccess) return e;
    // one problem: a CTA per resource and quantile (8 m + 1 CTAs instead of m + 1)
    const int nq = P == 1 ? 1 : kQuant;
    stats_kernel<<<dim3((m_max + 1) * (kQuant / nq), P), 1024, kSampleMax * 4, s>>>(probs, one, stats, nq);
    features_kernel<<<P, 256, 0, s>>>(probs, one, stats, feats);
    return cudaGetLastError();
}

cudaError_t mlp_reserve(ra_mlp *net, int rows)
{
    if (rows <= net->cap_rows) return cudaSuccess;
    cudaFree(net->act);
    net->act = nullptr;
    net->cap_rows = 0;
    const size_t per = static_cast<size_t>(rows);
    // z1 h1 z2 h2 dz2 dz1 (rows x 256 each), y dy (rows each)
    cudaError_t e = cudaMalloc(&net->act, sizeof(float) * per * (6 * kHid + 2));
    if (e != cudaSuccess) return e;
    net->cap_rows = rows;
    return cudaSuccess;
}

static void mlp_buffers(ra_mlp *net, int rows, float **z1, float **h1, float **z2, float **h2,
                        float **dz2, float **dz1, float **y, float **dy)
{
    const size_t L = static_cast<size_t>(net->cap_rows) * kHid;
    *z1 = net->act;
    *h1 = *z1 + L;
    *z2 = *h1 + L;
    *h2 = *z2 + L;
    *dz2 = *h2 + L;
    *dz1 = *dz2 + L;
    *y = *dz1 + L;
    *dy = *y + net->cap_rows;
    (void)rows;
}

cudaError_t mlp_forward(ra_mlp *net, const float *X, int rows, float *y_out, cudaStream_t s)
{
    cudaError_t e = mlp_reserve(net, rows);
    if (e != cudaSuccess) return e;
    float *z1, *h1, *z2, *h2, *dz2, *dz1, *y, *dy;
    mlp_buffers(net, rows, &z1, &h1, &z2, &h2, &dz2, &dz1, &y, &dy);
    const float *th = net->theta;
    if (rows <= 64 && y_out) {   // inference on one problem's resources
        infer_rows_kernel<<<rows, kHid * kInferSplit, 0, s>>>(X, th, y_out);
        return cudaGetLastError();
    }
    if (rows <= 64) {   // one problem's resources: one CTA per row
        rows_bias_gelu_kernel<<<rows, kHid, kFeatIn * 4, s>>>(kFeatIn, kHid, X, th + oW1, th + ob1, z1, h1);
        rows_bias_gelu_kernel<<<rows, kHid, kHid * 4, s>>>(kHid, kHid, h1, th + oW2, th + ob2, z2, h2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        if ((e = gemm<kEpiBiasGelu>(s, rows, kHid, kFeatIn, X, kFeatIn, 1, th + oW1, kHid, 1, nullptr,
                                    kHid, th + ob1, z1, h1)) != cudaSuccess)
            return e;
        if ((e = gemm<kEpiBiasGelu>(s, rows, kHid, kHid, h1, kHid, 1, th + oW2, kHid, 1, nullptr, kHid,
                                    th + ob2, z2, h2)) != cudaSuccess)
            return e;
    }
    head_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(rows, h2, th, y_out ? y_out : y);
    return cudaGetLastError();
}

cudaError_t mlp_train_step(ra_mlp *net, const float *X, const float *target, int rows, float lr,
                           float *loss, cudaStream_t s)
{
    cudaError_t e = mlp_forward(net, X, rows, nullptr, s);
    if (e != cudaSuccess) return e;
    float *z1, *h1, *z2, *h2, *dz2, *dz1, *y, *dy;
    mlp_buffers(net, rows, &z1, &h1, &z2, &h2, &dz2, &dz1, &y, &dy);
    float *g = net->grad;
    const float *th = net->theta;
    loss_kernel<<<1, 1024, 0, s>>>(rows, y, target, dy, g, loss);
    colsum_kernel<<<kHid / 32, dim3(32, 8), 0, s>>>(rows, kHid, h2, dy, g + oW3);           // dW3
    const long long tot = static_cast<long long>(rows) * kHid;
    head_back_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, s>>>(rows, dy, th, z2, dz2);
    if ((e = gemm<kEpiStore>(s, kHid, kHid, rows, h1, 1, kHid, dz2, kHid, 1, g + oW2, kHid)) !=
        cudaSuccess)                                                                           // dW2 = h1^T dz2
        return e;
    colsum_kernel<<<kHid / 32, dim3(32, 8), 0, s>>>(rows, kHid, dz2, nullptr, g + ob2);     // db2
    if ((e = gemm<kEpiGeluGrad>(s, rows, kHid, kHid, dz2, kHid, 1, th + oW2, 1, kHid, dz1, kHid,
                                nullptr, z1)) != cudaSuccess)                                   // dz1 = (dz2 W2^T) * GELU'(z1)
        return e;
    if ((e = gemm<kEpiStore>(s, kFeatIn, kHid, rows, X, 1, kFeatIn, dz1, kHid, 1, g + oW1, kHid)) !=
        cudaSuccess)                                                                           // dW1 = X^T dz1
        return e;
    colsum_kernel<<<kHid / 32, dim3(32, 8), 0, s>>>(rows, kHid, dz1, nullptr, g + ob1);     // db1
    net->t += 1;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, net->t));
    const double c2 = 1.0 / (1.0 - std::pow(0.999, net->t));
    adam_kernel<<<(RA_MLP_PARAMS + 255) / 256, 256, 0, s>>>(RA_MLP_PARAMS, net->theta, g, net->m1,
                                                            net->m2, lr, static_cast<float>(c1),
                                                            static_cast<float>(c2));
    return cudaGetLastError();
}

cudaError_t launch_warm_network(const FeatProblem &one, int m, float *stats, const ra_mlp *net,
                                float *feats, float *y, double *lam, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSampleMax * 4);
    if (e != cudaSuccess) return e;
    stats_kernel<<<dim3((m + 1) * kQuant, 1), 1024, kSampleMax * 4, s>>>(nullptr, one, stats, 1);
    warm_infer_kernel<<<m, kHid * kInferSplit, 0, s>>>(stats + static_cast<long long>(one.row0) * kFeatRes,
                                                       m, net->theta, feats, y, lam);
    return cudaGetLastError();
}

cudaError_t launch_exp_prices(int m, const float *y, double *lam, cudaStream_t s)
{
    exp_prices_kernel<<<1, 32, 0, s>>>(m, y, lam);
    return cudaGetLastError();
}

cudaError_t launch_choose(int m, const double *lam_w, const double *lam_c, const double *g2,
                          double *lam0, int32_t *used, cudaStream_t s)
{
    choose_kernel<<<1, 32, 0, s>>>(m, lam_w, lam_c, g2, lam0, used);
    return cudaGetLastError();
}

}  // namespace ra
