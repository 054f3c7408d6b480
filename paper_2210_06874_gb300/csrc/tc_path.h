// tc_path.h -- entry points of the mixed-precision (tensor-core) path (internal).
#pragma once

#include <cuda_runtime.h>

#include "ctx.h"
#include "launch.h"

namespace hmc {

int tc_ctx_init(hmc_ctx* c);   // FP16 split of E, FP32 workspaces
void tc_ctx_free(hmc_ctx* c);
int tc_apply(hmc_ctx* c, const double* phi, const float2* in, float2* out, bool dag,
             cudaStream_t s);
int tc_cg(hmc_ctx* c, const double* phi, const double2* chi, double2* x, double tol,
          int max_iter, cudaStream_t s);
int tc_trajectory(hmc_ctx* c, const TrajArgs& a, cudaStream_t s);

}  // namespace hmc
