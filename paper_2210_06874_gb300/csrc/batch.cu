// batch.cu -- C ABI of the batched form: many independent Markov chains of
// uneven size advanced by one persistent launch (see tc_kernels.cu).
#include "tc_path.h"

struct hmc_batch {
    hmc::TcBatch* impl;
};

extern "C" {

int hmc_batch_create(const hmc_params* params, int n_chains, hmc_batch** out) {
    if (!params || !out || n_chains < 1 || n_chains > (1 << 20)) return HMC_ERR_BAD_ARG;
    *out = nullptr;
    hmc::TcBatch* impl = nullptr;
    const int st = hmc::tc_batch_create(params, n_chains, &impl);
    if (st != HMC_OK) return st;
    *out = new hmc_batch{impl};
    return HMC_OK;
}

int hmc_batch_destroy(hmc_batch* b) {
    if (!b) return HMC_OK;
    hmc::tc_batch_destroy(b->impl);
    delete b;
    return HMC_OK;
}

int hmc_batch_layout(const hmc_batch* b, int64_t* offsets, int n_offsets) {
    if (!b || !offsets || n_offsets < hmc::tc_batch_size(b->impl) + 1) return HMC_ERR_BAD_ARG;
    static_assert(sizeof(long long) == sizeof(int64_t), "offset width");
    hmc::tc_batch_offsets(b->impl, reinterpret_cast<long long*>(offsets));
    return HMC_OK;
}

int hmc_batch_trajectory(hmc_batch* b, double* phi, uint64_t seed, uint64_t traj_index,
                         hmc_traj_out* out, void* stream) {
    if (!b || !phi || !out) return HMC_ERR_BAD_ARG;
    return hmc::tc_batch_trajectory(b->impl, phi, seed, traj_index, out, (cudaStream_t)stream);
}

}  // extern "C"
