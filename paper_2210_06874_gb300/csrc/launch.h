// launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ctx.h"

namespace hmc {

struct TrajArgs {
    double* phi;        // device field, in/out
    uint64_t seed;
    uint64_t traj;
    uint32_t chain;
    double eps;         // tau / n_md
    int n_md;
    double tol;
    int max_iter;
    double ru_delta;    // mixed path: reliable-update trigger
    int integrator;     // 0 leapfrog, 1 second-order minimum-norm (Omelyan)
    double hb_gamma;    // mass preconditioning: hop factor g of M_g (hb_inner > 0)
    int hb_inner;       // inner leapfrog steps per outer step (0: off)
};

// Molecular-dynamics schedule of a symmetric second-order integrator: kick
// md_kick(0) eps, then for m = 1 .. md_stages: drift md_drift eps, kick
// md_kick(m) eps (one force evaluation per kick).
//   leapfrog:  n_md stages, drift 1, kicks 1/2, 1, ..., 1, 1/2
//   minimum-norm (Omelyan, Mryglod, Folk 2003): 2 n_md stages, drift 1/2,
//   kicks lam, 1-2lam, 2lam, 1-2lam, ..., 2lam, 1-2lam, lam with
//   lam = 0.1931833275037836 (the minimum of the norm of its error terms)
constexpr double kOmelyanLambda = 0.1931833275037836;
__host__ __device__ inline int md_stages(const TrajArgs& a) {
    return a.integrator == 1 ? 2 * a.n_md : a.n_md;
}
__host__ __device__ inline double md_drift(const TrajArgs& a) {
    return a.integrator == 1 ? 0.5 : 1.0;
}
__host__ __device__ inline double md_kick(const TrajArgs& a, int m) {
    const int M = md_stages(a);
    if (a.integrator == 1) {
        if (m == 0 || m == M) return kOmelyanLambda;
        return (m & 1) ? 1.0 - 2.0 * kOmelyanLambda : 2.0 * kOmelyanLambda;
    }
    return (m == 0 || m == M) ? 0.5 : 1.0;
}

// Slots of ChainView::scalars written by the trajectory kernels.
enum TrajSlot : int {
    kTrajDH = 0, kTrajH0, kTrajH1, kTrajU, kTrajAccept, kTrajIters, kTrajSolves,
    kTrajRU, kTrajMaxRes, kTrajStatus, kTrajFp64Iters, kTrajItersOuter,
    // 12 and 13 keep the mixed CG's segment state
    kTrajSolvesOuter = 14, kNumScalars = 16
};

int launch_cis_f64(const ChainView& c, const double* phi, cudaStream_t s);
int launch_apply_f64(const ChainView& c, bool dag, const double2* in, double2* out,
                     cudaStream_t s);
int launch_force_f64(const ChainView& c, const double* phi, const double2* x, double* F,
                     cudaStream_t s);
int launch_action(const ChainView& c, const double* phi, const double2* chi, const double2* x,
                  double* out, cudaStream_t s);
int launch_cg_f64(const ChainView& c, int num_sms, const double* phi, const double2* chi,
                  double2* x, double tol, int max_iter, cudaStream_t s);
int launch_trajectory_f64(const ChainView& c, int num_sms, const TrajArgs& a, cudaStream_t s);

int launch_rng_draw(uint64_t seed, uint32_t stream_id, uint64_t traj, uint32_t chain,
                    int64_t n, uint32_t* raw, double* z0, double* z1, cudaStream_t s);

}  // namespace hmc
