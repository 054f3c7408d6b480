// observables.cu -- observables from M^{-1} sources (the paper's §2 names
// the single-particle gap Delta and the staggered magnetisation m_s as the
// order parameters of the transition).
//
// (1) The zero-momentum single-particle correlator on sublattice A from one
// M^{-1} source (the correlator whose decay in Euclidean time gives Delta).
//
// Source b: V_A^{-1/2} on the A sites (indices 0..V/2-1, sublattice-major)
// of slice 0, zero elsewhere.  g = M^{-1} b = M^dag (M M^dag)^{-1} b (CG in
// the requested precision, then the FP64 M^dag).  C(t) = V_A^{-1/2} sum over
// the A sites x of g_t(x), one FP64 block reduction per slice in a fixed
// order (deterministic).
#include <cmath>
#include <cstring>

#include "../../include/hmc.h"
#include "common.cuh"
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

// (2) Staggered spin traces.  With eps_x = +1 on sublattice A (x < V/2) and
// -1 on B, and G = M^{-1}: T_s = tr(eps G), T_u = tr(G), T_ss =
// tr(eps G eps G), estimated per Z2 noise vector eta (Philox stream 4,
// eta(e) = 1 - 2 (word0 & 1), counter (e, 4, sample, chain)) by
//     v = M^{-1} eta,  w = M^{-1} (eps v),
//     (eta^T eps v, eta^T v, eta^T eps w)        (eta is real).
// Each M^{-1} is M^dag (M M^dag)^{-1} (CG, then the FP64 M^dag).  Wick's
// theorem for the particles and (at mu = 0) for the holes, whose propagator
// is conj(G), gives the staggered space-time susceptibility of the field,
//     chi_s = (Re T_u - Re T_ss) / (2 N),  N = V Nt.
// All sums are FP64 in a fixed order: per-block tree sums over a grid that
// depends on N only, then one block sums the partials.

constexpr int kDotBlocks = 256;   // partial-sum blocks of one sample's dot products

__global__ void k_z2(double2* eta, int N, uint64_t seed, uint64_t sample, uint32_t chain) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        const uint4 r = philox_draw(seed, kStreamZ2, sample, chain, (uint32_t)e);
        eta[e] = make_double2((r.x & 1u) ? -1.0 : 1.0, 0.0);
    }
}

__global__ void k_eps(const double2* v, double2* ev, int V, int N) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        const double2 a = v[e];
        const double sg = (e % V) < V / 2 ? 1.0 : -1.0;
        ev[e] = make_double2(sg * a.x, sg * a.y);
    }
}

// Tree sum of six doubles over the 256 threads of a block (fixed order).
__device__ void block_sum6(double (*s)[256], double* acc) {
    for (int j = 0; j < 6; ++j) s[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int j = 0; j < 6; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + o];
        __syncthreads();
    }
}

// Partials of (eta eps v, eta v, eta eps w) as 6 doubles per block.
__global__ void __launch_bounds__(256) k_dots(const double2* eta, const double2* v,
                                              const double2* w, int V, int N, double* part) {
    __shared__ double s[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        const double n = eta[e].x;
        const double ne = (e % V) < V / 2 ? n : -n;
        const double2 a = v[e], b = w[e];
        acc[0] += ne * a.x;
        acc[1] += ne * a.y;
        acc[2] += n * a.x;
        acc[3] += n * a.y;
        acc[4] += ne * b.x;
        acc[5] += ne * b.y;
    }
    block_sum6(s, acc);
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// One block: sums the kDotBlocks partials into sample row out[0..2].
__global__ void __launch_bounds__(256) k_dots_final(const double* part, double2* out) {
    __shared__ double s[6][256];
    double acc[6];
    for (int j = 0; j < 6; ++j) acc[j] = part[threadIdx.x * 6 + j];
    block_sum6(s, acc);
    if (threadIdx.x < 3)
        out[threadIdx.x] = make_double2(s[2 * threadIdx.x][0], s[2 * threadIdx.x + 1][0]);
}

// One block: means over the samples (fixed order) and chi_s.
__global__ void __launch_bounds__(256) k_trace_mean(const double2* samples, int n, int N,
                                                    double2* mean) {
    __shared__ double s[6][256];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        for (int j = 0; j < 3; ++j) {
            acc[2 * j] += samples[3 * k + j].x;
            acc[2 * j + 1] += samples[3 * k + j].y;
        }
    block_sum6(s, acc);
    if (threadIdx.x == 0) {
        double m[6];
        for (int j = 0; j < 6; ++j) m[j] = s[j][0] / n;
        for (int j = 0; j < 3; ++j) mean[j] = make_double2(m[2 * j], m[2 * j + 1]);
        mean[3] = make_double2((m[2] - m[4]) / (2.0 * N), 0.0);
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

extern "C" int hmc_spin_traces(hmc_ctx* c, const double* phi, int n_noise, uint64_t seed,
                               uint32_t chain, double tol, int max_iter, int precision,
                               void* samples, void* mean, hmc_cg_stats* stats, void* stream) {
    if (!c || !phi || !mean || !stats) return HMC_ERR_BAD_ARG;
    if (precision != HMC_PREC_FP64 && precision != HMC_PREC_MIXED) return HMC_ERR_BAD_ARG;
    if (n_noise < 1 || n_noise > (1 << 20)) return HMC_ERR_BAD_ARG;
    if (c->params.mu != 0.0) return HMC_ERR_UNSUPPORTED;
    const hmc::ChainView& v = c->view;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)v.N * sizeof(double2);
    const size_t nsamp = (size_t)n_noise * 3 * sizeof(double2);
    const size_t npart = (size_t)hmc::obs::kDotBlocks * 6 * sizeof(double);
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, 5 * n + nsamp + npart, s) != cudaSuccess) return HMC_ERR_CUDA;
    double2* eta = (double2*)buf;
    double2* y = (double2*)((char*)buf + n);
    double2* vv = (double2*)((char*)buf + 2 * n);
    double2* ev = (double2*)((char*)buf + 3 * n);
    double2* w = (double2*)((char*)buf + 4 * n);
    double2* samp = (double2*)((char*)buf + 5 * n);
    double* part = (double*)((char*)buf + 5 * n + nsamp);
    const int grid = (int)((v.N + 255) / 256 < 1184 ? (v.N + 255) / 256 : 1184);
    hmc_cg_stats one;
    *stats = hmc_cg_stats{0, 0, 0.0, HMC_OK, 0};
    int st = HMC_OK;
    for (int k = 0; k < n_noise && st == HMC_OK; ++k) {
        hmc::obs::k_z2<<<grid, 256, 0, s>>>(eta, v.N, seed, (uint64_t)k, chain);
        if (cudaGetLastError() != cudaSuccess) st = HMC_ERR_CUDA;
        // v = M^{-1} eta, then w = M^{-1} (eps v)
        for (int half = 0; half < 2 && st == HMC_OK; ++half) {
            const double2* src = half == 0 ? eta : ev;
            double2* dst = half == 0 ? vv : w;
            st = hmc_cg_solve(c, phi, src, y, tol, max_iter, precision, &one, stream);
            stats->iterations += one.iterations;
            stats->reliable_updates += one.reliable_updates;
            stats->fp64_iterations += one.fp64_iterations;
            if (one.true_residual > stats->true_residual) stats->true_residual = one.true_residual;
            if (st == HMC_OK) st = hmc_apply_Mdag(c, phi, y, dst, HMC_PREC_FP64, stream);
            if (st == HMC_OK && half == 0) {
                hmc::obs::k_eps<<<grid, 256, 0, s>>>(vv, ev, v.V, v.N);
                if (cudaGetLastError() != cudaSuccess) st = HMC_ERR_CUDA;
            }
        }
        if (st == HMC_OK) {
            hmc::obs::k_dots<<<hmc::obs::kDotBlocks, 256, 0, s>>>(eta, vv, w, v.V, v.N, part);
            hmc::obs::k_dots_final<<<1, 256, 0, s>>>(part, samp + 3 * (size_t)k);
            if (cudaGetLastError() != cudaSuccess) st = HMC_ERR_CUDA;
        }
    }
    if (st == HMC_OK) {
        hmc::obs::k_trace_mean<<<1, 256, 0, s>>>(samp, n_noise, v.N, (double2*)mean);
        if (cudaGetLastError() != cudaSuccess) st = HMC_ERR_CUDA;
    }
    if (st == HMC_OK && samples &&
        cudaMemcpyAsync(samples, samp, nsamp, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        st = HMC_ERR_CUDA;
    stats->status = st;
    cudaFreeAsync(buf, s);
    if (st == HMC_OK && cudaStreamSynchronize(s) != cudaSuccess) st = HMC_ERR_CUDA;
    return st;
}
