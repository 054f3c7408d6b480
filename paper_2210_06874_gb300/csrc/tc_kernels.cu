// tc_kernels.cu -- mixed-precision path (placeholder until the tensor-core
// contraction lands).
#include "tc_path.h"

namespace hmc {

int tc_ctx_init(hmc_ctx*) { return HMC_OK; }
void tc_ctx_free(hmc_ctx*) {}
int tc_apply(hmc_ctx*, const double*, const float2*, float2*, bool, cudaStream_t) {
    return HMC_ERR_UNSUPPORTED;
}
int tc_cg(hmc_ctx*, const double*, const double2*, double2*, double, int, cudaStream_t) {
    return HMC_ERR_UNSUPPORTED;
}
int tc_trajectory(hmc_ctx*, const TrajArgs&, cudaStream_t) { return HMC_ERR_UNSUPPORTED; }

}  // namespace hmc
