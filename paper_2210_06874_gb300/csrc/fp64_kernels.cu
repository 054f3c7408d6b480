// fp64_kernels.cu -- kernels of the FP64 path and their launchers.
//
//  k_cis        exp(i phi) table (one pass over phi)
//  k_apply      one application of M or M^dag (one tile per CTA)
//  k_force      F = phi/(delta U) + 2 Im(x conj(M^dag x))
//  k_cg         persistent CG solve of (M M^dag) x = chi
//  k_trajectory persistent HMC trajectory: heat bath, leapfrog, Metropolis
#include "fp64_path.cuh"
#include "launch.h"

namespace hmc {
namespace f64 {

__global__ void k_cis(const double* __restrict__ phi, double2* __restrict__ cis, int N) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        double s, co;
        sincos(phi[e], &s, &co);
        cis[e] = make_double2(co, s);
    }
}

template <bool DAG>
__global__ void __launch_bounds__(NTHR) k_apply(ChainView c, const double2* in, double2* out) {
    __shared__ Smem sm;
    EpiArgs ea = {};
    apply_tile<DAG, EPI_STORE>(c, blockIdx.x, in, out, ea, sm);
}

__global__ void __launch_bounds__(NTHR) k_force(ChainView c, const double* phi,
                                                const double2* x, double* F) {
    __shared__ Smem sm;
    EpiArgs ea = {};
    ea.phi = phi;
    ea.F = F;
    ea.inv_dU = 1.0 / (c.delta * c.U);
    apply_tile<true, EPI_FORCE>(c, blockIdx.x, x, nullptr, ea, sm);
}

__device__ __forceinline__ Team make_team(const ChainView& c) {
    Team tm;
    tm.rank = blockIdx.x;
    tm.size = gridDim.x + c.team_pad;
    tm.bar = c.bar;
    tm.status = c.status;
    tm.partials = c.partials;
    tm.cs = nullptr;
    return tm;
}

__device__ __forceinline__ void fill_cis(const ChainView& c, const Team& tm, const double* phi) {
    HMC_TEAM_ELEMS(e, c, tm) {
        double s, co;
        sincos(phi[e], &s, &co);
        c.cis[e] = make_double2(co, s);
    }
}

// Action Eq. (2.1) without the momenta: per-CTA partials of
// sum(phi^2) / (2 delta U) + Re(chi^dag x), then a one-CTA fixed-order sum.
__global__ void k_action_partials(const double* __restrict__ phi, const double2* __restrict__ chi,
                                  const double2* __restrict__ x, int N, double half_inv_dU,
                                  double* __restrict__ partials) {
    double v[1] = {0.0};
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
        const double ph = phi[e];
        const double2 a = chi[e], b = x[e];
        v[0] += half_inv_dU * ph * ph + a.x * b.x + a.y * b.y;
    }
    block_reduce<1>(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out) {
    double v[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) v[0] += partials[j];
    block_reduce<1>(v);
    if (threadIdx.x == 0) *out = v[0];
}

// scalars: [0] iterations [1] true residual [2] status
__global__ void __launch_bounds__(NTHR) k_cg(ChainView c, const double* phi, const double2* chi,
                                             double2* x, double tol, int max_iter) {
    __shared__ Smem sm;
    Team tm = make_team(c);
    fill_cis(c, tm, phi);
    if (!team_barrier(tm)) return;
    CgResult res;
    if (!cg_solve(c, tm, chi, x, tol, max_iter, res, sm)) return;
    if (tm.rank == 0 && threadIdx.x == 0) {
        c.scalars[0] = res.iterations;
        c.scalars[1] = res.true_res;
        c.scalars[2] = res.status;
    }
}

// scalars: see TrajSlot in launch.h
__global__ void __launch_bounds__(NTHR) k_trajectory(ChainView c, TrajArgs a) {
    __shared__ Smem sm;
    Team tm = make_team(c);
    double* phi = a.phi;
    const double inv_dU = 1.0 / (c.delta * c.U);
    const double rsqrt2 = 0.70710678118654752440;
    // 1. heat bath: momenta, pseudofermion noise, start energy
    double h0[3] = {0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 zp = normal_pair(philox_draw(a.seed, kStreamMomentum, a.traj, a.chain, e));
        const double2 zr = normal_pair(philox_draw(a.seed, kStreamNoise, a.traj, a.chain, e));
        const double ph = phi[e];
        c.pi[e] = zp.x;
        const double2 rho = make_double2(zr.x * rsqrt2, zr.y * rsqrt2);
        c.rho[e] = rho;
        c.phi_old[e] = ph;
        double s, co;
        sincos(ph, &s, &co);
        c.cis[e] = make_double2(co, s);
        h0[0] += ph * ph;
        h0[1] += rho.x * rho.x + rho.y * rho.y;
        h0[2] += zp.x * zp.x;
    }
    if (!team_sum<3>(tm, h0)) return;
    // chi^dag (M M^dag)^{-1} chi = rho^dag rho at the start field
    const double H0 = 0.5 * h0[0] * inv_dU + h0[1] + 0.5 * h0[2];
    // 2. chi = M rho
    EpiArgs ea = {};
    apply_team<false, EPI_STORE>(c, tm, c.rho, c.chi, ea, sm);
    if (!team_barrier(tm)) return;
    // 3. leapfrog
    int iters = 0, solves = 0, status = HMC_OK;
    double max_res = 0.0;
    ea.phi = phi;
    ea.pi = c.pi;
    ea.inv_dU = inv_dU;
    const double ed = a.eps * c.delta;
    const double edrift = md_drift(a) * ed;
    const int n_stages = md_stages(a);
    for (int step = 0; step <= n_stages; ++step) {
        if (step > 0) {
            HMC_TEAM_ELEMS(e, c, tm) {
                const double ph = fma(edrift, c.pi[e], phi[e]);
                phi[e] = ph;
                double s, co;
                sincos(ph, &s, &co);
                c.cis[e] = make_double2(co, s);
            }
            if (!team_barrier(tm)) return;
        }
        CgResult res;
        if (!cg_solve(c, tm, c.chi, c.x, a.tol, a.max_iter, res, sm)) return;
        iters += res.iterations;
        ++solves;
        max_res = fmax(max_res, res.true_res);
        if (res.status != HMC_OK && status == HMC_OK) status = res.status;
        ea.kick = md_kick(a, step) * ed;
        apply_team<true, EPI_FORCE>(c, tm, c.x, nullptr, ea, sm);
        if (!team_barrier(tm)) return;
    }
    // 4. end energy and Metropolis
    double h1[3] = {0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double ph = phi[e], pv = c.pi[e];
        const double2 ch = c.chi[e], xv = c.x[e];
        h1[0] += ph * ph;
        h1[1] += ch.x * xv.x + ch.y * xv.y;
        h1[2] += pv * pv;
    }
    if (!team_sum<3>(tm, h1)) return;
    const double H1 = 0.5 * h1[0] * inv_dU + h1[1] + 0.5 * h1[2];
    const double dH = H1 - H0;
    const double u = uniform_pair(philox_draw(a.seed, kStreamMetropolis, a.traj, a.chain, 0)).x;
    const bool accept = u < exp(-dH);
    if (!accept) {
        HMC_TEAM_ELEMS(e, c, tm) phi[e] = c.phi_old[e];
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
        c.scalars[kTrajDH] = dH;
        c.scalars[kTrajH0] = H0;
        c.scalars[kTrajH1] = H1;
        c.scalars[kTrajU] = u;
        c.scalars[kTrajAccept] = accept ? 1.0 : 0.0;
        c.scalars[kTrajIters] = iters;
        c.scalars[kTrajSolves] = solves;
        c.scalars[kTrajRU] = 0;
        c.scalars[kTrajMaxRes] = max_res;
        c.scalars[kTrajStatus] = status;
    }
}

// One HMC trajectory with mass preconditioning (Hasenbusch 2001) and the
// two-level nested leapfrog (Sexton and Weingarten 1992), all in FP64.
// Heavy operator M_g = 1 - g S E D (the contraction scaled by g); two
// pseudofermions chi_1 = M_g rho_1 (rho_1 from stream 3) and
// chi_2 = M_g^{-1} M rho_2 = M_g^dag (M_g M_g^dag)^{-1} M rho_2 (rho_2 from
// the plain noise stream), H = S_B + chi_1^dag (M_g M_g^dag)^{-1} chi_1
// + phi_2^dag (M M^dag)^{-1} phi_2 + pi^2/2 with phi_2 = M_g chi_2.
// Outer level (n_md steps of eps): the ratio force
//     F_2 = 2 Im(x_2 conj(M^dag x_2)) - 2 Im(conj(M_g^dag x_2 - x_2) chi_2);
// inner level (hb_inner steps of eps / hb_inner inside each outer step):
//     F_B + F_1 = phi / (delta U) + 2 Im(x_1 conj(M_g^dag x_1)).
// Consecutive inner kicks are merged.  Every solve starts from zero.
// Scalars as k_trajectory, plus the outer level's CG iterations and solves.
__global__ void __launch_bounds__(NTHR) k_trajectory_hb(ChainView c, TrajArgs a) {
    __shared__ Smem sm;
    Team tm = make_team(c);
    double* phi = a.phi;
    const double inv_dU = 1.0 / (c.delta * c.U);
    const double rsqrt2 = 0.70710678118654752440;
    const double gm1 = a.hb_gamma - 1.0;
    // 1. heat bath: momenta, the two noise vectors, start energy
    double h0[3] = {0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 zp = normal_pair(philox_draw(a.seed, kStreamMomentum, a.traj, a.chain, e));
        const double2 z2 = normal_pair(philox_draw(a.seed, kStreamNoise, a.traj, a.chain, e));
        const double2 z1 = normal_pair(philox_draw(a.seed, kStreamHeavy, a.traj, a.chain, e));
        const double ph = phi[e];
        c.pi[e] = zp.x;
        const double2 r1 = make_double2(z1.x * rsqrt2, z1.y * rsqrt2);
        const double2 r2 = make_double2(z2.x * rsqrt2, z2.y * rsqrt2);
        c.rho[e] = r1;
        c.xh[e] = r2;
        c.phi_old[e] = ph;
        double s, co;
        sincos(ph, &s, &co);
        c.cis[e] = make_double2(co, s);
        h0[0] += ph * ph;
        h0[1] += r1.x * r1.x + r1.y * r1.y + r2.x * r2.x + r2.y * r2.y;
        h0[2] += zp.x * zp.x;
    }
    if (!team_sum<3>(tm, h0)) return;
    // S_1 = rho_1^dag rho_1 and S_2 = rho_2^dag rho_2 at the start field
    const double H0 = 0.5 * h0[0] * inv_dU + h0[1] + 0.5 * h0[2];
    // 2. chi_1 = M_g rho_1; chi_2 = M_g^dag (M_g M_g^dag)^{-1} M rho_2
    EpiArgs eg = {};
    eg.hop_m1 = gm1;
    EpiArgs e1 = {};
    apply_team<false, EPI_STORE>(c, tm, c.rho, c.chi, eg, sm);
    apply_team<false, EPI_STORE>(c, tm, c.xh, c.phi2, e1, sm);
    if (!team_barrier(tm)) return;
    int iters_in = 0, iters_out = 0, solves_in = 0, solves_out = 0, status = HMC_OK;
    double max_res = 0.0;
    CgResult res;
    if (!cg_solve(c, tm, c.phi2, c.x2, a.tol, a.max_iter, res, sm, false, gm1)) return;
    iters_in += res.iterations;
    ++solves_in;
    max_res = fmax(max_res, res.true_res);
    if (res.status != HMC_OK) status = res.status;
    apply_team<true, EPI_STORE>(c, tm, c.x2, c.chi2, eg, sm);
    if (!team_barrier(tm)) return;
    // 3. nested leapfrog
    const double ed = a.eps * c.delta;
    const double h = 1.0 / a.hb_inner;
    auto drift = [&](double cf) {
        HMC_TEAM_ELEMS(e, c, tm) {
            const double ph = fma(cf * ed, c.pi[e], phi[e]);
            phi[e] = ph;
            double s, co;
            sincos(ph, &s, &co);
            c.cis[e] = make_double2(co, s);
        }
        return team_barrier(tm);
    };
    auto kick_inner = [&](double cf) {
        CgResult r;
        if (!cg_solve(c, tm, c.chi, c.x, a.tol, a.max_iter, r, sm, false, gm1)) return false;
        iters_in += r.iterations;
        ++solves_in;
        max_res = fmax(max_res, r.true_res);
        if (r.status != HMC_OK && status == HMC_OK) status = r.status;
        EpiArgs ef = {};
        ef.hop_m1 = gm1;
        ef.phi = phi;
        ef.pi = c.pi;
        ef.inv_dU = inv_dU;
        ef.kick = cf * ed;
        apply_team<true, EPI_FORCE>(c, tm, c.x, nullptr, ef, sm);
        return team_barrier(tm);
    };
    auto kick_outer = [&](double cf) {
        apply_team<false, EPI_STORE>(c, tm, c.chi2, c.phi2, eg, sm);   // phi_2 = M_g chi_2
        if (!team_barrier(tm)) return false;
        CgResult r;
        if (!cg_solve(c, tm, c.phi2, c.x2, a.tol, a.max_iter, r, sm)) return false;
        iters_out += r.iterations;
        ++solves_out;
        max_res = fmax(max_res, r.true_res);
        if (r.status != HMC_OK && status == HMC_OK) status = r.status;
        EpiArgs ef = {};
        ef.phi = phi;
        ef.pi = c.pi;
        ef.inv_dU = 0.0;              // the bosonic force sits on the inner level
        ef.kick = cf * ed;
        apply_team<true, EPI_FORCE>(c, tm, c.x2, nullptr, ef, sm);
        if (!team_barrier(tm)) return false;
        ef.hop_m1 = gm1;
        ef.chi = c.chi2;
        apply_team<true, EPI_RATIO>(c, tm, c.x2, nullptr, ef, sm);
        return team_barrier(tm);
    };
    if (!kick_outer(0.5)) return;
    for (int k = 0; k < a.n_md; ++k) {
        for (int m = 0; m < a.hb_inner; ++m) {
            if (!kick_inner(m == 0 ? 0.5 * h : h)) return;
            if (!drift(h)) return;
        }
        if (!kick_inner(0.5 * h)) return;
        if (!kick_outer(k + 1 < a.n_md ? 1.0 : 0.5)) return;
    }
    // 4. end energy (the last kick of each level was at the final field) and
    // Metropolis
    double h1[4] = {0.0, 0.0, 0.0, 0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double ph = phi[e], pv = c.pi[e];
        const double2 c1 = c.chi[e], x1 = c.x[e], p2 = c.phi2[e], x2 = c.x2[e];
        h1[0] += ph * ph;
        h1[1] += c1.x * x1.x + c1.y * x1.y;
        h1[2] += p2.x * x2.x + p2.y * x2.y;
        h1[3] += pv * pv;
    }
    if (!team_sum<4>(tm, h1)) return;
    const double H1 = 0.5 * h1[0] * inv_dU + h1[1] + h1[2] + 0.5 * h1[3];
    const double dH = H1 - H0;
    const double u = uniform_pair(philox_draw(a.seed, kStreamMetropolis, a.traj, a.chain, 0)).x;
    const bool accept = u < exp(-dH);
    if (!accept) {
        HMC_TEAM_ELEMS(e, c, tm) phi[e] = c.phi_old[e];
    }
    if (tm.rank == 0 && threadIdx.x == 0) {
        c.scalars[kTrajDH] = dH;
        c.scalars[kTrajH0] = H0;
        c.scalars[kTrajH1] = H1;
        c.scalars[kTrajU] = u;
        c.scalars[kTrajAccept] = accept ? 1.0 : 0.0;
        c.scalars[kTrajIters] = iters_in + iters_out;
        c.scalars[kTrajSolves] = solves_in + solves_out;
        c.scalars[kTrajRU] = 0;
        c.scalars[kTrajMaxRes] = max_res;
        c.scalars[kTrajStatus] = status;
        c.scalars[kTrajItersOuter] = iters_out;
        c.scalars[kTrajSolvesOuter] = solves_out;
    }
}

}  // namespace f64

// ------------------------------------------------------------ launchers
static int persistent_grid(const void* kernel, int threads, int num_sms, int want) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess ||
        occ < 1)
        return -1;
    int g = num_sms * occ;
    if (g > kMaxTeam) g = kMaxTeam;
    if (want < g) g = want;
    return g < 1 ? 1 : g;
}

static cudaError_t launch_coop(const void* kernel, int grid, int threads, void** args,
                               cudaStream_t s) {
    return cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(threads), args, 0, s);
}

int launch_cis_f64(const ChainView& c, const double* phi, cudaStream_t s) {
    int blocks = (c.N + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    f64::k_cis<<<blocks, 256, 0, s>>>(phi, c.cis, c.N);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int launch_apply_f64(const ChainView& c, bool dag, const double2* in, double2* out,
                     cudaStream_t s) {
    const int nt = ((c.V + f64::TI - 1) / f64::TI) * ((c.Nt + f64::TT - 1) / f64::TT);
    if (dag)
        f64::k_apply<true><<<nt, f64::NTHR, 0, s>>>(c, in, out);
    else
        f64::k_apply<false><<<nt, f64::NTHR, 0, s>>>(c, in, out);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int launch_force_f64(const ChainView& c, const double* phi, const double2* x, double* F,
                     cudaStream_t s) {
    const int nt = ((c.V + f64::TI - 1) / f64::TI) * ((c.Nt + f64::TT - 1) / f64::TT);
    f64::k_force<<<nt, f64::NTHR, 0, s>>>(c, phi, x, F);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int launch_action(const ChainView& c, const double* phi, const double2* chi, const double2* x,
                  double* out, cudaStream_t s) {
    int blocks = (c.N + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    f64::k_action_partials<<<blocks, 256, 0, s>>>(phi, chi, x, c.N, 0.5 / (c.delta * c.U),
                                                 c.partials);
    f64::k_sum_partials<<<1, 256, 0, s>>>(c.partials, blocks, out);
    return cudaGetLastError() == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

int launch_cg_f64(const ChainView& c, int num_sms, const double* phi, const double2* chi,
                  double2* x, double tol, int max_iter, cudaStream_t s) {
    const int nt = ((c.V + f64::TI - 1) / f64::TI) * ((c.Nt + f64::TT - 1) / f64::TT);
    const int grid = persistent_grid((const void*)f64::k_cg, f64::NTHR, num_sms, nt);
    if (grid < 1) return HMC_ERR_CUDA;
    ChainView cv = c;
    void* args[] = {&cv, &phi, &chi, &x, &tol, &max_iter};
    return launch_coop((const void*)f64::k_cg, grid, f64::NTHR, args, s) == cudaSuccess
               ? HMC_OK
               : HMC_ERR_CUDA;
}

int launch_trajectory_f64(const ChainView& c, int num_sms, const TrajArgs& a, cudaStream_t s) {
    const int nt = ((c.V + f64::TI - 1) / f64::TI) * ((c.Nt + f64::TT - 1) / f64::TT);
    const void* fn = a.hb_inner > 0 ? (const void*)f64::k_trajectory_hb
                                    : (const void*)f64::k_trajectory;
    if (a.hb_inner > 0 && (!c.chi2 || !c.phi2 || !c.x2)) return HMC_ERR_BAD_ARG;
    const int grid = persistent_grid(fn, f64::NTHR, num_sms, nt);
    if (grid < 1) return HMC_ERR_CUDA;
    ChainView cv = c;
    TrajArgs av = a;
    void* args[] = {&cv, &av};
    return launch_coop(fn, grid, f64::NTHR, args, s) == cudaSuccess ? HMC_OK : HMC_ERR_CUDA;
}

}  // namespace hmc
