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

struct TcBatch;
int tc_batch_create(const hmc_params* p, int n, TcBatch** out);
void tc_batch_destroy(TcBatch* b);
void tc_batch_offsets(const TcBatch* b, long long* off);
int tc_batch_size(const TcBatch* b);
int tc_batch_trajectory(TcBatch* b, double* phi, uint64_t seed, uint64_t traj,
                        hmc_traj_out* out, cudaStream_t caller);

}  // namespace hmc
