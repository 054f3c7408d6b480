// api.cu -- the C ABI declared in include/hmc.h: context management,
// host-side construction of the lattice and of E = exp(delta*kappa*h), the
// generator kernel, and the entry points that dispatch to the FP64 and the
// mixed-precision paths.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "launch.h"
#include "tc_path.h"

namespace hmc {

// ------------------------------------------------------------------ lattice
// Honeycomb bonds (§1, Fig. 1): the A site of cell (m1,m2) bonds to the B
// sites of cells (m1,m2), (m1-1,m2), (m1,m2-1), indices mod L; multiplicity
// is kept (L = 1 gives three bonds between the same pair).
static int site(int s, int m1, int m2, int L) {
    m1 = ((m1 % L) + L) % L;
    m2 = ((m2 % L) + L) % L;
    return s * L * L + m1 * L + m2;
}

static void hop_apply(int L, const std::vector<double>& v, std::vector<double>& out) {
    std::fill(out.begin(), out.end(), 0.0);
    for (int m1 = 0; m1 < L; ++m1)
        for (int m2 = 0; m2 < L; ++m2) {
            const int a = site(0, m1, m2, L);
            const int nb[3] = {site(1, m1, m2, L), site(1, m1 - 1, m2, L), site(1, m1, m2 - 1, L)};
            for (int b : nb) {
                out[a] += v[b];
                out[b] += v[a];
            }
        }
}

// E = exp(dk * h).  h commutes with lattice translations, so
// E[(s,m),(s',m')] depends on (s, s', m - m') only: two columns suffice.
// Each column is the Taylor series sum_n (dk h)^n e_y / n! of the sparse h,
// summed until the term is below 1e-18 of the sum (for dk > 0 every term is
// non-negative, so there is no cancellation).  The matrix is symmetrised.
static void build_transfer_matrix(int L, double dk, std::vector<double>& E) {
    const int V = 2 * L * L;
    std::vector<double> col[2];
    std::vector<double> term(V), next(V);
    for (int sp = 0; sp < 2; ++sp) {
        col[sp].assign(V, 0.0);
        std::fill(term.begin(), term.end(), 0.0);
        term[site(sp, 0, 0, L)] = 1.0;
        col[sp] = term;
        for (int n = 1; n < 400; ++n) {
            hop_apply(L, term, next);
            double tmax = 0.0, smax = 0.0;
            for (int i = 0; i < V; ++i) {
                term[i] = next[i] * (dk / n);
                col[sp][i] += term[i];
                tmax = std::fmax(tmax, std::fabs(term[i]));
                smax = std::fmax(smax, std::fabs(col[sp][i]));
            }
            if (n > 2 && tmax <= 1e-18 * smax) break;
        }
    }
    E.assign((size_t)V * V, 0.0);
    for (int sp = 0; sp < 2; ++sp)
        for (int q1 = 0; q1 < L; ++q1)
            for (int q2 = 0; q2 < L; ++q2) {
                const int y = site(sp, q1, q2, L);
                for (int s = 0; s < 2; ++s)
                    for (int m1 = 0; m1 < L; ++m1)
                        for (int m2 = 0; m2 < L; ++m2) {
                            const int x = site(s, m1, m2, L);
                            E[(size_t)x * V + y] = col[sp][site(s, m1 - q1, m2 - q2, L)];
                        }
            }
    for (int x = 0; x < V; ++x)
        for (int y = x + 1; y < V; ++y) {
            const double a = 0.5 * (E[(size_t)x * V + y] + E[(size_t)y * V + x]);
            E[(size_t)x * V + y] = a;
            E[(size_t)y * V + x] = a;
        }
}

// ------------------------------------------------------------------ rng
__global__ void k_rng_draw(uint64_t seed, uint32_t stream_id, uint64_t traj, uint32_t chain,
                           int64_t n, uint32_t* raw, double* z0, double* z1) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox_draw(seed, stream_id, traj, chain, (uint32_t)e);
        if (raw) {
            raw[4 * e + 0] = r.x;
            raw[4 * e + 1] = r.y;
            raw[4 * e + 2] = r.z;
            raw[4 * e + 3] = r.w;
        }
        if (z0 || z1) {
            const double2 z = normal_pair(r);
            if (z0) z0[e] = z.x;
            if (z1) z1[e] = z.y;
        }
    }
}

int launch_rng_draw(uint64_t seed, uint32_t stream_id, uint64_t traj, uint32_t chain, int64_t n,
                    uint32_t* raw, double* z0, double* z1, cudaStream_t s) {
    if (n <= 0) return HMC_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_rng_draw<<<(int)blocks, 256, 0, s>>>(seed, stream_id, traj, chain, n, raw, z0, z1);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

}  // namespace hmc

using namespace hmc;

// ------------------------------------------------------------------ helpers
static void* ctx_alloc(hmc_ctx* c, size_t bytes, bool* ok) {
    if (!*ok) return nullptr;
    void* p = nullptr;
    if (c->n_allocs >= (int)(sizeof(c->allocs) / sizeof(c->allocs[0])) ||
        cudaMalloc(&p, bytes == 0 ? 16 : bytes) != cudaSuccess) {
        *ok = false;
        return nullptr;
    }
    c->allocs[c->n_allocs++] = p;
    cudaMemset(p, 0, bytes == 0 ? 16 : bytes);
    return p;
}

static int valid_params(const hmc_params* p) {
    if (!p) return 0;
    if (p->L < 1 || p->Nt < 1) return 0;
    if (!(p->U > 0.0) || !(p->beta > 0.0) || !std::isfinite(p->kappa)) return 0;
    if (p->n_md < 1 || !(p->traj_length > 0.0)) return 0;
    if (!(p->cg_tol > 0.0) || p->cg_max_iter < 1) return 0;
    if (p->precision != HMC_PREC_FP64 && p->precision != HMC_PREC_MIXED) return 0;
    if (p->ru_delta < 0.0 || p->ru_delta >= 1.0) return 0;
    if (p->team_ctas < 0 || p->team_ctas > 1024) return 0;
    if (p->inner_ctas < 0 || p->inner_ctas > 1024) return 0;
    if (p->operand_mode < 0 || p->operand_mode > 5) return 0;
    if (p->cluster_mode < 0 || p->cluster_mode > 2) return 0;
    if (p->integrator < 0 || p->integrator > 1) return 0;
    if (p->ru_every < 0) return 0;
    if (p->hb_inner < 0 || p->hb_inner > 64) return 0;
    if (p->hb_inner > 0 && (!(p->hb_gamma >= 0.0 && p->hb_gamma < 1.0) || p->integrator != 0))
        return 0;
    // |delta mu| <= 5: the scaled E keeps its FP16 split in range
    if (!std::isfinite(p->mu) || std::fabs(p->mu * p->beta / p->Nt) > 5.0) return 0;
    if (p->operand_mode == 4 || p->operand_mode == 5) {
        if (p->tile_slices < 0 || p->tile_slices > 64) return 0;
    } else if (p->tile_slices != 0 && p->tile_slices != 8 && p->tile_slices != 16 &&
               p->tile_slices != 32) {
        return 0;
    }
    // indices of [Nt][V] vectors are 32-bit in the kernels
    const long long N = 2LL * p->L * p->L * (long long)p->Nt;
    if (N > (1LL << 30)) return 0;
    return 1;
}

static int finish_status(hmc_ctx* c, cudaStream_t s, int* dev_status) {
    int st = 0;
    if (cudaMemcpyAsync(&st, c->view.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HMC_ERR_CUDA;
    *dev_status = st;
    return HMC_OK;
}

extern "C" {

const char* hmc_version(void) { return "hmc-gb300 0.1 (sm_103a)"; }

int hmc_ctx_create(const hmc_params* p, hmc_ctx** out) {
    if (!out || !valid_params(p)) return HMC_ERR_BAD_ARG;
    *out = nullptr;
    hmc_ctx* c = new hmc_ctx();
    std::memset(c, 0, sizeof(*c));
    c->params = *p;
    // default reliable-update threshold: a residual drop of 20 between FP64
    // updates.  The best value depends on the chain (measured: 0.01 saves
    // FP64 work on one CTA at L = 12, while at L = 24, beta = 12 the FP32
    // iteration stalls without frequent updates); the autotuner times it.
    if (c->params.ru_delta == 0.0) c->params.ru_delta = 0.05;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        delete c;
        return HMC_ERR_CUDA;
    }
    ChainView& v = c->view;
    v.L = p->L;
    v.V = 2 * p->L * p->L;
    v.Nt = p->Nt;
    v.N = v.V * v.Nt;
    v.delta = p->beta / p->Nt;
    v.kappa = p->kappa;
    v.U = p->U;
    std::vector<double> E;
    build_transfer_matrix(p->L, v.delta * p->kappa, E);
    if (p->mu != 0.0) {
        // chemical potential of the particles: H of §1 carries + mu sum_x rho_x,
        // rho_x = p^dag p - h^dag h, so the particle transfer matrix is
        // exp(delta (kappa h - mu)) = e^{-delta mu} exp(delta kappa h)
        const double f = std::exp(-v.delta * p->mu);
        for (double& e : E) e *= f;
    }
    bool ok = true;
    const size_t N = (size_t)v.N;
    double* dE = (double*)ctx_alloc(c, E.size() * sizeof(double), &ok);
    v.cis = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.x = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.r = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.p = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.q = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.chi = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.rho = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    v.xh = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    if (p->hb_inner > 0) {
        v.chi2 = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
        v.phi2 = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
        v.x2 = (double2*)ctx_alloc(c, N * sizeof(double2), &ok);
    }
    v.pi = (double*)ctx_alloc(c, N * sizeof(double), &ok);
    v.phi_old = (double*)ctx_alloc(c, N * sizeof(double), &ok);
    v.bar = (unsigned*)ctx_alloc(c, 8 * sizeof(unsigned), &ok);
    v.status = (int*)ctx_alloc(c, kStatusBlockBytes, &ok);
    v.partials = (double*)ctx_alloc(c, sizeof(double) * kPartialDoubles, &ok);
    v.scalars = (double*)ctx_alloc(c, sizeof(double) * kNumScalars, &ok);
    if (ok && cudaMemcpy(dE, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice) !=
                  cudaSuccess)
        ok = false;
    v.E = dE;
    if (ok && tc_ctx_init(c) != HMC_OK) ok = false;
    if (ok && cudaMallocHost((void**)&c->scalars_host, sizeof(double) * kNumScalars) != cudaSuccess)
        ok = false;
    if (ok && cudaDeviceSynchronize() != cudaSuccess) ok = false;
    if (!ok) {
        hmc_ctx_destroy(c);
        return HMC_ERR_CUDA;
    }
    *out = c;
    return HMC_OK;
}

int hmc_ctx_destroy(hmc_ctx* c) {
    if (!c) return HMC_OK;
    cudaDeviceSynchronize();
    tc_ctx_free(c);
    for (int i = 0; i < c->n_allocs; ++i) cudaFree(c->allocs[i]);
    if (c->scalars_host) cudaFreeHost(c->scalars_host);
    delete c;
    return HMC_OK;
}

int hmc_get_transfer_matrix(hmc_ctx* c, double* E_host, size_t n_elems) {
    if (!c || !E_host) return HMC_ERR_BAD_ARG;
    const size_t need = (size_t)c->view.V * c->view.V;
    if (n_elems < need) return HMC_ERR_BAD_ARG;
    return cudaMemcpy(E_host, c->view.E, need * sizeof(double), cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? HMC_OK
               : HMC_ERR_CUDA;
}

static int apply_common(hmc_ctx* c, const double* phi, const void* in, void* out, int prec,
                        void* stream, bool dag) {
    if (!c || !phi || !in || !out || in == out) return HMC_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == HMC_PREC_FP64) {
        int st = launch_cis_f64(c->view, phi, s);
        if (st != HMC_OK) return st;
        return launch_apply_f64(c->view, dag, (const double2*)in, (double2*)out, s);
    }
    if (prec == HMC_PREC_MIXED) return tc_apply(c, phi, (const float2*)in, (float2*)out, dag, s);
    return HMC_ERR_BAD_ARG;
}

int hmc_apply_M(hmc_ctx* c, const double* phi, const void* in, void* out, int prec,
                void* stream) {
    return apply_common(c, phi, in, out, prec, stream, false);
}

int hmc_apply_Mdag(hmc_ctx* c, const double* phi, const void* in, void* out, int prec,
                   void* stream) {
    return apply_common(c, phi, in, out, prec, stream, true);
}

int hmc_cg_solve(hmc_ctx* c, const double* phi, const void* chi, void* x, double tol,
                 int max_iter, int prec, hmc_cg_stats* stats, void* stream) {
    if (!c || !phi || !chi || !x || chi == x || !stats) return HMC_ERR_BAD_ARG;
    if (!(tol > 0.0) || max_iter < 1) return HMC_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(stats, 0, sizeof(*stats));
    if (cudaMemsetAsync(c->view.status, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(c->view.bar, 0, 8 * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(c->view.scalars, 0, sizeof(double) * kNumScalars, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    int st;
    if (prec == HMC_PREC_FP64)
        st = launch_cg_f64(c->view, c->num_sms, phi, (const double2*)chi, (double2*)x, tol,
                           max_iter, s);
    else if (prec == HMC_PREC_MIXED)
        st = tc_cg(c, phi, (const double2*)chi, (double2*)x, tol, max_iter, s);
    else
        return HMC_ERR_BAD_ARG;
    if (st != HMC_OK) return st;
    if (cudaMemcpyAsync(c->scalars_host, c->view.scalars, sizeof(double) * kNumScalars,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    int dev = 0;
    if ((st = finish_status(c, s, &dev)) != HMC_OK) return st;
    if (dev != 0) {
        stats->status = dev;
        return dev;
    }
    stats->iterations = (int)c->scalars_host[0];
    stats->true_residual = c->scalars_host[1];
    stats->status = (int)c->scalars_host[2];
    stats->reliable_updates = (int)c->scalars_host[3];
    stats->fp64_iterations = (int)c->scalars_host[4];
    return stats->status;
}

int hmc_force(hmc_ctx* c, const double* phi, const void* x, double* F, void* stream) {
    if (!c || !phi || !x || !F) return HMC_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = launch_cis_f64(c->view, phi, s);
    if (st != HMC_OK) return st;
    return launch_force_f64(c->view, phi, (const double2*)x, F, s);
}

int hmc_action(hmc_ctx* c, const double* phi, const void* chi, const void* x, double* S_host,
               void* stream) {
    if (!c || !phi || !chi || !x || !S_host) return HMC_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int st = launch_action(c->view, phi, (const double2*)chi, (const double2*)x, c->view.scalars, s);
    if (st != HMC_OK) return st;
    if (cudaMemcpyAsync(c->scalars_host, c->view.scalars, sizeof(double), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HMC_ERR_CUDA;
    *S_host = c->scalars_host[0];
    return std::isfinite(*S_host) ? HMC_OK : HMC_ERR_NONFINITE;
}

int hmc_trajectory(hmc_ctx* c, double* phi, uint64_t seed, uint64_t traj_index, uint32_t chain,
                   hmc_traj_out* out, void* stream) {
    if (!c || !phi || !out) return HMC_ERR_BAD_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(out, 0, sizeof(*out));
    if (cudaMemsetAsync(c->view.status, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(c->view.bar, 0, 8 * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(c->view.scalars, 0, sizeof(double) * kNumScalars, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    TrajArgs a;
    a.phi = phi;
    a.seed = seed;
    a.traj = traj_index;
    a.chain = chain;
    a.n_md = c->params.n_md;
    a.eps = c->params.traj_length / c->params.n_md;
    a.tol = c->params.cg_tol;
    a.max_iter = c->params.cg_max_iter;
    a.ru_delta = c->params.ru_delta;
    a.integrator = c->params.integrator;
    a.hb_gamma = c->params.hb_gamma;
    a.hb_inner = c->params.hb_inner;
    // mass preconditioning: FP64, or the mixed path on split-K tiles (whose
    // epilogues carry the heavy operator's hop factor)
    if (a.hb_inner > 0 && c->params.precision != HMC_PREC_FP64 && c->params.operand_mode != 5)
        return HMC_ERR_UNSUPPORTED;
    int st;
    if (c->params.precision == HMC_PREC_FP64)
        st = launch_trajectory_f64(c->view, c->num_sms, a, s);
    else
        st = tc_trajectory(c, a, s);
    if (st != HMC_OK) return st;
    if (cudaMemcpyAsync(c->scalars_host, c->view.scalars, sizeof(double) * kNumScalars,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HMC_ERR_CUDA;
    int dev = 0;
    if ((st = finish_status(c, s, &dev)) != HMC_OK) return st;
    const double* v = c->scalars_host;
    out->dH = v[kTrajDH];
    out->H0 = v[kTrajH0];
    out->H1 = v[kTrajH1];
    out->u = v[kTrajU];
    out->accept = (int)v[kTrajAccept];
    out->cg_iterations = (int)v[kTrajIters];
    out->cg_solves = (int)v[kTrajSolves];
    out->reliable_updates = (int)v[kTrajRU];
    out->max_true_residual = v[kTrajMaxRes];
    out->fp64_iterations = (int)v[kTrajFp64Iters];
    out->cg_iterations_outer = (int)v[kTrajItersOuter];
    out->cg_solves_outer = (int)v[kTrajSolvesOuter];
    out->status = dev != 0 ? dev : (int)v[kTrajStatus];
    return out->status;
}

int hmc_ctx_set_wait_limit(hmc_ctx* c, double seconds) {
    if (!c || !(seconds >= 0.0) || seconds > 3600.0) return HMC_ERR_BAD_ARG;
    const uint64_t ns = (uint64_t)(seconds * 1e9);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(c->view.status + 2, &ns, sizeof(ns), cudaMemcpyHostToDevice) != cudaSuccess)
        return HMC_ERR_CUDA;
    return HMC_OK;
}

int hmc_debug_team_padding(hmc_ctx* c, int extra_ctas) {
    if (!c || extra_ctas < 0 || extra_ctas > kMaxTeam) return HMC_ERR_BAD_ARG;
    c->view.team_pad = extra_ctas;
    return HMC_OK;
}

int hmc_rng_draw(uint64_t seed, uint32_t stream_id, uint64_t traj, uint32_t chain, int64_t n,
                 uint32_t* raw, double* z0, double* z1, void* stream) {
    if (n < 0 || n > (1LL << 32)) return HMC_ERR_BAD_ARG;
    return launch_rng_draw(seed, stream_id, traj, chain, n, raw, z0, z1, (cudaStream_t)stream);
}

}  // extern "C"
