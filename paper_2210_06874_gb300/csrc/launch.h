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
};

// Slots of ChainView::scalars written by the trajectory kernels.
enum TrajSlot : int {
    kTrajDH = 0, kTrajH0, kTrajH1, kTrajU, kTrajAccept, kTrajIters, kTrajSolves,
    kTrajRU, kTrajMaxRes, kTrajStatus, kNumScalars = 16
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
