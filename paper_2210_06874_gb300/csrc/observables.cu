// observables.cu -- the zero-momentum single-particle correlator on
// sublattice A from one M^{-1} source (the correlator whose decay in
// Euclidean time gives the single-particle gap Delta of the paper's §2).
//
// Source b: V_A^{-1/2} on the A sites (indices 0..V/2-1, sublattice-major)
// of slice 0, zero elsewhere.  g = M^{-1} b = M^dag (M M^dag)^{-1} b (CG in
// the requested precision, then the FP64 M^dag).  C(t) = V_A^{-1/2} sum over
// the A sites x of g_t(x), one FP64 block reduction per slice in a fixed
// order (deterministic).
#include <cmath>
#include <cstring>

#include "../../include/hmc.h"
#include "ctx.h"

namespace hmc {
namespace obs {

__global__ void k_source(double2* b, int V, int Nt) {
    const int VA = V / 2;
    const double a = 1.0 / sqrt((double)VA);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)V * Nt;
         e += (long long)gridDim.x * blockDim.x)
        b[e] = make_double2(e < VA ? a : 0.0, 0.0);
}

// One block per slice t: C[t] = V_A^{-1/2} sum_{x < V_A} g[t][x].
__global__ void k_sum_a(const double2* g, double2* C, int V) {
    __shared__ double2 s[256];
    const int t = blockIdx.x, VA = V / 2;
    double2 acc = make_double2(0.0, 0.0);
    for (int x = threadIdx.x; x < VA; x += blockDim.x) {
        const double2 v = g[(size_t)t * V + x];
        acc.x += v.x;
        acc.y += v.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s[threadIdx.x].x += s[threadIdx.x + o].x;
            s[threadIdx.x].y += s[threadIdx.x + o].y;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double a = 1.0 / sqrt((double)VA);
        C[t] = make_double2(s[0].x * a, s[0].y * a);
    }
}

}  // namespace obs
}  // namespace hmc

extern "C" int hmc_correlator_k0(hmc_ctx* c, const double* phi, double tol, int max_iter,
                                 int precision, void* C, hmc_cg_stats* stats, void* stream) {
    if (!c || !phi || !C || !stats) return HMC_ERR_BAD_ARG;
    if (precision != HMC_PREC_FP64 && precision != HMC_PREC_MIXED) return HMC_ERR_BAD_ARG;
    const hmc::ChainView& v = c->view;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)v.N * sizeof(double2);
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, 3 * n, s) != cudaSuccess) return HMC_ERR_CUDA;
    double2* b = (double2*)buf;
    double2* y = (double2*)((char*)buf + n);
    double2* g = (double2*)((char*)buf + 2 * n);
    hmc::obs::k_source<<<256, 256, 0, s>>>(b, v.V, v.Nt);
    int st = cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
    if (st == HMC_OK) st = hmc_cg_solve(c, phi, b, y, tol, max_iter, precision, stats, stream);
    if (st == HMC_OK) st = hmc_apply_Mdag(c, phi, y, g, HMC_PREC_FP64, stream);
    if (st == HMC_OK) {
        hmc::obs::k_sum_a<<<v.Nt, 256, 0, s>>>(g, (double2*)C, v.V);
        if (cudaGetLastError() != cudaSuccess) st = HMC_ERR_CUDA;
    }
    cudaFreeAsync(buf, s);
    return st;
}
