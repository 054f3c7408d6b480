// noalloc.cu -- hmc_cg_solve_noalloc: the FP64 CG solve for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: hosts whose device memory is
// handed out by a framework's own pool or by a fixed-budget real-time
// allocator, and plugins loaded into a process that forbids its extensions
// from growing the device heap.  They cannot create an hmc_ctx, whose
// workspaces are cudaMalloc'ed.  This entry point runs the same persistent
// FP64 CG kernel as hmc_cg_solve(prec = HMC_PREC_FP64), but its scratch (the
// exp(i phi) table, the CG vectors r, p, q, the team partial sums, the
// barrier and status words) lives in one file-scope __device__ array that
// every GPU loading the library holds until exit.  The call waits for its
// own result (it copies the statistics to the host and synchronises the
// stream), so it refuses to run on a stream that is being captured into a
// CUDA graph.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "ctx.h"
#include "launch.h"

namespace hmc {
namespace {

// Largest space-time volume N = V * Nt the static scratch holds.
constexpr int kNoAllocMaxN = 32768;
constexpr size_t kVecBytes = sizeof(double2) * (size_t)kNoAllocMaxN;
constexpr size_t kPartialBytes = sizeof(double) * kPartialDoubles;
// layout: cis | r | p | q | partials | scalars[16] | bar[2] | status
constexpr size_t kOffR = kVecBytes;
constexpr size_t kOffP = 2 * kVecBytes;
constexpr size_t kOffQ = 3 * kVecBytes;
constexpr size_t kOffPartials = 4 * kVecBytes;
constexpr size_t kOffScalars = kOffPartials + kPartialBytes;
constexpr size_t kOffBar = kOffScalars + 16 * sizeof(double);
constexpr size_t kOffStatus = kOffBar + 256;
constexpr size_t kScratchBytes = kOffStatus + 256;  // about 2.1 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct DeviceScratch {
    CUcontext ctx;      // context the address was looked up in
    void* addr;         // device address of the array in that context
    int num_sms;
};
DeviceScratch g_scratch[kMaxDevices];

// The current context of the calling thread (driver entry point, so the
// library needs no link against the driver library).
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext*);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    });
    CUcontext c = nullptr;
    if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

// Set-up once per device (and again if that device's context was replaced,
// e.g. after cudaDeviceReset), with the device current: the host-side name
// of the array is only a stand-in, so look up its device address.
int scratch_for_current_device(void** addr, int* num_sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HMC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HMC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceScratch& d = g_scratch[dev];
    const CUcontext ctx = current_context();
    if (!d.addr || !ctx || d.ctx != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return HMC_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return HMC_ERR_CUDA;
        d.num_sms = sms;
        d.addr = p;
        d.ctx = current_context();
    }
    *addr = d.addr;
    *num_sms = d.num_sms;
    return HMC_OK;
}

}  // namespace
}  // namespace hmc

extern "C" int hmc_cg_solve_noalloc(const double* E, int L, int Nt, const double* phi,
                                    const void* chi, void* x, double tol, int max_iter,
                                    hmc_cg_stats* stats, void* stream) {
    using namespace hmc;
    if (!E || !phi || !chi || !x || chi == x || !stats) return HMC_ERR_BAD_ARG;
    if (L < 1 || Nt < 1 || !(tol > 0.0) || max_iter < 1) return HMC_ERR_BAD_ARG;
    std::memset(stats, 0, sizeof(*stats));
    cudaStream_t s = (cudaStream_t)stream;
    // a stream under graph capture: refuse before anything is enqueued (the
    // call synchronises and reads its result on the host), so the caller's
    // capture stays valid
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return HMC_ERR_UNSUPPORTED;
    }
    if (cap != cudaStreamCaptureStatusNone) return HMC_ERR_UNSUPPORTED;
    const long long V = 2LL * L * L;
    if (V * Nt > kNoAllocMaxN) return HMC_ERR_UNSUPPORTED;
    void* base = nullptr;
    int num_sms = 0;
    int st = scratch_for_current_device(&base, &num_sms);
    if (st != HMC_OK) return st;
    unsigned char* b = static_cast<unsigned char*>(base);
    ChainView v;
    std::memset(&v, 0, sizeof(v));
    v.L = L;
    v.V = (int)V;
    v.Nt = Nt;
    v.N = (int)(V * Nt);
    v.E = E;
    v.cis = reinterpret_cast<double2*>(b);
    v.r = reinterpret_cast<double2*>(b + kOffR);
    v.p = reinterpret_cast<double2*>(b + kOffP);
    v.q = reinterpret_cast<double2*>(b + kOffQ);
    v.partials = reinterpret_cast<double*>(b + kOffPartials);
    v.scalars = reinterpret_cast<double*>(b + kOffScalars);
    v.bar = reinterpret_cast<unsigned*>(b + kOffBar);
    v.status = reinterpret_cast<int*>(b + kOffStatus);
    // the barrier must start at zero, the status word and the outputs clear
    if (cudaMemsetAsync(b + kOffScalars, 0, kScratchBytes - kOffScalars, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    st = launch_cg_f64(v, num_sms, phi, (const double2*)chi, (double2*)x, tol, max_iter, s);
    if (st != HMC_OK) return st;
    double out[3];
    int dev_status = 0;
    if (cudaMemcpyAsync(out, v.scalars, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&dev_status, v.status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HMC_ERR_CUDA;
    if (dev_status != 0) {
        stats->status = dev_status;
        return dev_status;
    }
    stats->iterations = (int)out[0];
    stats->true_residual = out[1];
    stats->status = (int)out[2];
    return stats->status;
}
