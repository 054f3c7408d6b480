// fp64_path.cuh -- FP64 fermion-matrix application on CUDA cores and the
// solver / force / trajectory steps built on it (device functions).
//
// Operator (exponential-hopping form of the fermion matrix, Eq. (2.2)):
//   (M psi)_t     = psi_t - s_t     E (e^{i phi_{t-1}} psi_{t-1})
//   (M^dag psi)_t = psi_t - s_{t+1} e^{-i phi_t} (E psi_{t+1}),   s_0 = -1.
// The contraction E * u over all slices is a real V x V times complex
// V x Nt product; an output tile is TI sites x TT slices, K runs over all
// sites in chunks of KC.  E is symmetric, so the chunk E[i0.., k0..] is read
// as rows k of E (coalesced) and stored k-major in shared memory.
#pragma once

#include "common.cuh"
#include "ctx.h"

namespace hmc {
namespace f64 {

constexpr int TI = 32;     // sites per tile (= lanes of a warp)
constexpr int TT = 8;      // slices per tile (= warps of the CTA)
constexpr int KC = 32;     // K chunk
constexpr int NTHR = TI * TT;
static_assert(NTHR == KC * TT && (KC * TI) % NTHR == 0, "FP64 tile: chunk loads per thread");

struct Smem {
    double Et[KC][TI];     // Et[kk][ii] = E[k0+kk][i0+ii] = E[i0+ii][k0+kk]
    double2 U[TT][KC];     // source vectors of the tile's slices
};

// Epilogue modes of a tile.
enum Epi : int {
    EPI_STORE = 0,       // out = M(in) (or M^dag); optional partial |out|^2
    EPI_CG_UPDATE = 1,   // M q -> Ap; x += alpha p; r -= alpha Ap; partial |r|^2
    EPI_RESIDUAL = 2,    // r = chi - M(in); partial |r|^2
    EPI_FORCE = 3,       // M^dag x -> y; F = phi/(dU) + 2 Im(x conj y);
                         //   store F if F != null; pi -= kick * F if pi != null
    EPI_RATIO = 4,       // M_g^dag x -> y; pi -= kick * (-2 Im(conj(y - x) chi)):
                         //   the M_g part of the ratio force of mass preconditioning
};

struct EpiArgs {
    double alpha;
    double2* x;
    double2* r;
    const double2* p;
    const double2* chi;
    const double* phi;
    double* F;
    double* pi;
    double kick;
    double inv_dU;   // 1 / (delta U)
    double hop_m1;   // hop - 1: the contraction is scaled by hop (M_g of mass
                     // preconditioning uses hop = g; 0 here is the plain M)
};

__device__ __forceinline__ int num_tiles(const ChainView& c) {
    return ((c.V + TI - 1) / TI) * ((c.Nt + TT - 1) / TT);
}

// One output tile.  `in` is the vector M (DAG=false) or M^dag (DAG=true)
// acts on.  Returns this thread's contribution to the tile's reduction.
template <bool DAG, int EPI>
__device__ double apply_tile(const ChainView& c, int tile, const double2* __restrict__ in,
                             double2* __restrict__ out, const EpiArgs& ea, Smem& sm) {
    const int V = c.V, Nt = c.Nt;
    const int nti = (V + TI - 1) / TI;
    const int i0 = (tile % nti) * TI, t0 = (tile / nti) * TT;
    const int ii = threadIdx.x & (TI - 1), tt = threadIdx.x / TI;
    const double* __restrict__ E = c.E;
    const double2* __restrict__ cis = c.cis;
    // Chunk k0's E block and source values are loaded into registers while
    // the previous chunk is contracted from shared memory (one buffer: the
    // registers are the second stage), so the L2 latency of a chunk hides
    // behind the FP64 arithmetic of the one before.  The summation order is
    // that of a plain loop over k.
    constexpr int kEPer = KC * TI / NTHR;   // E elements per thread and chunk
    const int ukk = threadIdx.x % KC, us = threadIdx.x / KC;
    double ev[kEPer];
    double2 uv;
    auto fetch = [&](int k0) {
#pragma unroll
        for (int j = 0; j < kEPer; ++j) {
            const int e = threadIdx.x + j * NTHR;
            const int kk = e / TI, cc = e % TI;
            const int k = k0 + kk, i = i0 + cc;
            ev[j] = (k < V && i < V) ? E[(size_t)k * V + i] : 0.0;
        }
        const int k = k0 + ukk, tq = t0 + us;
        uv = make_double2(0.0, 0.0);
        if (k < V && tq < Nt) {
            if (DAG) {
                const int ts = (tq + 1 == Nt) ? 0 : tq + 1;
                uv = in[(size_t)ts * V + k];
            } else {
                const int ts = (tq == 0) ? Nt - 1 : tq - 1;
                uv = cmul(cis[(size_t)ts * V + k], in[(size_t)ts * V + k]);
            }
        }
    };
    double ar = 0.0, ai = 0.0;
    fetch(0);
    for (int k0 = 0; k0 < V; k0 += KC) {
#pragma unroll
        for (int j = 0; j < kEPer; ++j) {
            const int e = threadIdx.x + j * NTHR;
            sm.Et[e / TI][e % TI] = ev[j];
        }
        sm.U[us][ukk] = uv;
        __syncthreads();
        if (k0 + KC < V) fetch(k0 + KC);
#pragma unroll 8
        for (int kk = 0; kk < KC; ++kk) {
            const double e = sm.Et[kk][ii];
            const double2 u = sm.U[tt][kk];
            ar = fma(e, u.x, ar);
            ai = fma(e, u.y, ai);
        }
        __syncthreads();
    }
    const int i = i0 + ii, t = t0 + tt;
    if (i >= V || t >= Nt) return 0.0;
    const size_t o = (size_t)t * V + i;
    const double hop = 1.0 + ea.hop_m1;
    double2 w = make_double2(ar * hop, ai * hop);
    double sgn;
    if (DAG) {
        sgn = (t == Nt - 1) ? -1.0 : 1.0;
        w = cmulc(cis[o], w);
    } else {
        sgn = (t == 0) ? -1.0 : 1.0;
    }
    const double2 src = in[o];
    const double2 res = make_double2(src.x - sgn * w.x, src.y - sgn * w.y);
    if (EPI == EPI_STORE) {
        out[o] = res;
        return res.x * res.x + res.y * res.y;
    } else if (EPI == EPI_CG_UPDATE) {
        const double2 pv = ea.p[o];
        double2 xv = ea.x[o], rv = ea.r[o];
        xv.x = fma(ea.alpha, pv.x, xv.x);
        xv.y = fma(ea.alpha, pv.y, xv.y);
        rv.x = fma(-ea.alpha, res.x, rv.x);
        rv.y = fma(-ea.alpha, res.y, rv.y);
        ea.x[o] = xv;
        ea.r[o] = rv;
        return rv.x * rv.x + rv.y * rv.y;
    } else if (EPI == EPI_RESIDUAL) {
        const double2 ch = ea.chi[o];
        const double2 rv = make_double2(ch.x - res.x, ch.y - res.y);
        ea.r[o] = rv;
        return rv.x * rv.x + rv.y * rv.y;
    } else if (EPI == EPI_FORCE) {  // in = x, res = y = M^dag x
        const double ph = ea.phi[o];
        // Im(x conj(y)) = x.y*y.x - x.x*y.y
        const double f = ph * ea.inv_dU + 2.0 * (src.y * res.x - src.x * res.y);
        if (ea.F) ea.F[o] = f;
        if (ea.pi) ea.pi[o] -= ea.kick * f;
        return f * f;
    } else {  // EPI_RATIO: in = x, res = y = M_g^dag x, d = y - x
        const double2 ch = ea.chi[o];
        const double dx = res.x - src.x, dy = res.y - src.y;
        // Im(conj(d) chi) = d.x*chi.y - d.y*chi.x
        const double f = -2.0 * (dx * ch.y - dy * ch.x);
        ea.pi[o] -= ea.kick * f;
        return f * f;
    }
}

// All tiles of one application, spread over the team.
template <bool DAG, int EPI>
__device__ __forceinline__ double apply_team(const ChainView& c, const Team& tm,
                                             const double2* in, double2* out,
                                             const EpiArgs& ea, Smem& sm) {
    double acc = 0.0;
    const int nt = num_tiles(c);
    for (int tile = tm.rank; tile < nt; tile += tm.size)
        acc += apply_tile<DAG, EPI>(c, tile, in, out, ea, sm);
    return acc;
}

#define HMC_TEAM_ELEMS(e, c, tm) \
    for (int e = (tm).rank * blockDim.x + threadIdx.x; e < (c).N; e += (tm).size * blockDim.x)

struct CgResult {
    int iterations;
    double true_res;   // |chi - M M^dag x| / |chi|
    int status;
};

// Conjugate gradient on M M^dag (FP64; with hop_m1 != 0 on M_g M_g^dag, the
// contraction scaled by 1 + hop_m1), CG vectors in the chain workspace
// (r, p, q), from x = 0 or (warm) from the x given, whose residual
// chi - M M^dag x then starts the iteration.  cis must hold exp(i phi).
// Ends with the FP64 true residual, which leaves chi - M M^dag x in r and
// M^dag x in q.
__device__ inline bool cg_solve(const ChainView& c, Team& tm, const double2* chi, double2* x,
                         double tol, int max_iter, CgResult& res, Smem& sm,
                         bool warm = false, double hop_m1 = 0.0) {
    double2 *r = c.r, *p = c.p, *q = c.q;
    double v1[1] = {0.0};
    HMC_TEAM_ELEMS(e, c, tm) {
        const double2 ch = chi[e];
        if (!warm) {
            x[e] = make_double2(0.0, 0.0);
            r[e] = ch;
            p[e] = ch;
        }
        v1[0] += ch.x * ch.x + ch.y * ch.y;
    }
    if (!team_sum<1>(tm, v1)) return false;
    const double chi2 = v1[0];
    double rr = chi2;
    res.iterations = 0;
    res.status = HMC_OK;
    res.true_res = 0.0;
    if (!(chi2 > 0.0)) {
        if (!finite_d(chi2)) res.status = HMC_ERR_NONFINITE;
        return true;
    }
    const double stop = tol * tol * chi2;
    EpiArgs ea = {};
    ea.x = x;
    ea.r = r;
    ea.p = p;
    ea.hop_m1 = hop_m1;
    if (warm) {
        // r = chi - M (M^dag x), p = r
        apply_team<true, EPI_STORE>(c, tm, x, q, ea, sm);
        if (!team_barrier(tm)) return false;
        ea.chi = chi;
        double vr[1] = {apply_team<false, EPI_RESIDUAL>(c, tm, q, nullptr, ea, sm)};
        if (!team_sum<1>(tm, vr)) return false;
        rr = vr[0];
        HMC_TEAM_ELEMS(e, c, tm) p[e] = r[e];
        if (!team_barrier(tm)) return false;
        if (!finite_d(rr)) res.status = HMC_ERR_NONFINITE;
    }
    int it = 0;
    bool conv = res.status == HMC_OK && rr <= stop;
    while (!conv && res.status == HMC_OK && it < max_iter) {
        double vq[1] = {apply_team<true, EPI_STORE>(c, tm, p, q, ea, sm)};  // q = M^dag p
        if (!team_sum<1>(tm, vq)) return false;
        const double qq = vq[0];
        if (!finite_d(qq) || !(qq > 0.0)) { res.status = HMC_ERR_NONFINITE; break; }
        ea.alpha = rr / qq;
        double vr[1] = {apply_team<false, EPI_CG_UPDATE>(c, tm, q, nullptr, ea, sm)};
        if (!team_sum<1>(tm, vr)) return false;
        const double rr_new = vr[0];
        ++it;
        if (!finite_d(rr_new)) { res.status = HMC_ERR_NONFINITE; break; }
        if (rr_new <= stop) { conv = true; break; }
        const double beta = rr_new / rr;
        rr = rr_new;
        HMC_TEAM_ELEMS(e, c, tm) {
            const double2 rv = r[e], pv = p[e];
            p[e] = make_double2(fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y));
        }
        if (!team_barrier(tm)) return false;
    }
    res.iterations = it;
    if (res.status == HMC_OK && !conv) res.status = HMC_ERR_CG_NOT_CONVERGED;
    // FP64 true residual r = chi - M (M^dag x)
    if (!team_barrier(tm)) return false;
    apply_team<true, EPI_STORE>(c, tm, x, q, ea, sm);
    if (!team_barrier(tm)) return false;
    ea.chi = chi;
    double vt[1] = {apply_team<false, EPI_RESIDUAL>(c, tm, q, nullptr, ea, sm)};
    if (!team_sum<1>(tm, vt)) return false;
    res.true_res = sqrt(vt[0] / chi2);
    if (!finite_d(res.true_res)) res.status = HMC_ERR_NONFINITE;
    return true;
}

}  // namespace f64
}  // namespace hmc
