// ra_eval_dual_static: the dual evaluation of ra_eval_dual without any device
// allocation, for callers that may not allocate (serving loops with a
// no-allocation rule, hosts whose framework owns all device memory).  Its
// scratch (per-CTA partial sums, the last-CTA ticket, the status word and
// the result slots) lives in one file-scope static device array that every
// GPU loading this library holds until the process exits.  The call is
// asynchronous: a bounded wait that gave up shows as NaN in g and q.

#include <cstring>
#include <mutex>

#include "ra_internal.cuh"

namespace {

// Partial sums for at most kStaticMaxCtas CTAs, plus the result slots.
constexpr int kStaticMaxCtas = 1024;
constexpr size_t kPartialBytes = sizeof(double) * ra::kPartW * kStaticMaxCtas;
constexpr size_t kOutOffset = kPartialBytes;
constexpr size_t kTicketOffset = kOutOffset + ((sizeof(ra::EvalOut) + 255) / 256) * 256;
constexpr size_t kStatusOffset = kTicketOffset + 256;
constexpr size_t kScratchBytes = kStatusOffset + 256;  // about 546 KB

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Launch configuration per (device, m, cap mode), computed on the first call
// (configure_dual also sets the kernels' attributes on that device).
struct LaunchConfig {
    bool valid;
    int num_sms, mt, stages, grid_dual, grid_aux;
    size_t smem_dual;
};
LaunchConfig g_config[kMaxDevices][RA_MAX_M][2] = {};

// Device address of the scratch array on `dev` (the current device), looked
// up once per device: in host code the symbol names a host-side stand-in, so
// the kernel must be given the address the runtime reports.
ra_status scratch_on(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return ra::fail(RA_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || ptr == nullptr)
            return ra::fail(RA_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[dev]);
    return RA_OK;
}

}  // namespace

extern "C" ra_status ra_eval_dual_static(int64_t n, int32_t m, const float *A, const uint8_t *kind,
                                         const float *w, const float *param, const double *R,
                                         const double *lambda, uint32_t flags, void *stream,
                                         double *g, double *q)
{
    if (n < 1) return ra::fail(RA_EINVAL, "n = %lld must be >= 1", (long long)n);
    if (m < 1 || m > RA_MAX_M) return ra::fail(RA_EINVAL, "m = %d must lie in [1, %d]", m, RA_MAX_M);
    if (!A || !kind || !w || !param || !R || !lambda || !g || !q)
        return ra::fail(RA_EINVAL, "a pointer argument is NULL");
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(kind) |
         reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(param)) & 15u)
        return ra::fail(RA_EINVAL, "A, kind, w and param must be 16-byte aligned");
    if (flags & ~RA_NO_JOB_CAP)
        return ra::fail(RA_EINVAL, "only RA_NO_JOB_CAP may be set (flags 0x%x)", flags);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ra::fail(RA_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    ra_status st = scratch_on(dev, &scratch);
    if (st != RA_OK) return st;

    // launch configuration exactly as ra_problem_create computes it (no workspace)
    ra_problem p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.m = m;
    p.flags = flags;
    p.A = A;
    p.kind = kind;
    p.w = w;
    p.param = param;
    p.R = R;
    p.stream = static_cast<cudaStream_t>(stream);
    p.device = dev;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        LaunchConfig &c = g_config[dev][m - 1][(flags & RA_NO_JOB_CAP) ? 1 : 0];
        if (!c.valid) {
            e = cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = ra::configure_dual(&p);
            if (e != cudaSuccess)
                return ra::fail(RA_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
            c = LaunchConfig{true, p.num_sms, p.mt, p.stages, p.grid_dual, p.grid_aux, p.smem_dual};
        }
        p.num_sms = c.num_sms;
        p.mt = c.mt;
        p.stages = c.stages;
        p.grid_dual = c.grid_dual;
        p.grid_aux = c.grid_aux;
        p.smem_dual = c.smem_dual;
    }
    if (p.grid_dual > kStaticMaxCtas)
        return ra::fail(RA_EINVAL,
                        "this GPU runs %d CTAs per evaluation; the static scratch holds partial sums "
                        "for at most %d",
                        p.grid_dual, kStaticMaxCtas);

    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + kTicketOffset);
    int *status = reinterpret_cast<int *>(scratch + kStatusOffset);
    ra::EvalOut *out = reinterpret_cast<ra::EvalOut *>(scratch + kOutOffset);
    // the array keeps the previous call's contents: the ticket and the status
    // word must start at zero
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), p.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), p.stream);
    if (e != cudaSuccess) return ra::fail(RA_ECUDA, "scratch reset: %s", cudaGetErrorString(e));

    ra::DualParams dp{};
    dp.A = A;
    dp.kind = kind;
    dp.w = w;
    dp.param = param;
    dp.R = R;
    dp.n = n;
    dp.m = m;
    dp.lam = lambda;
    dp.partials = reinterpret_cast<double *>(scratch);
    dp.ticket = ticket;
    dp.status = status;
    dp.out = out;
    e = ra::launch_dual(&p, dp, p.stream);
    if (e != cudaSuccess) return ra::fail(RA_ECUDA, "dual launch: %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(g, &out->g, sizeof(double), cudaMemcpyDeviceToDevice, p.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q, out->q, sizeof(double) * m, cudaMemcpyDeviceToDevice, p.stream);
    if (e != cudaSuccess) return ra::fail(RA_ECUDA, "copy results: %s", cudaGetErrorString(e));
    return RA_OK;
}
