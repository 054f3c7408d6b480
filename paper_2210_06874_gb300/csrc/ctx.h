// ctx.h -- the opaque hmc_ctx and the per-chain device view handed to kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hmc.h"

namespace hmc {

// Device view of one chain: sizes, constants and the workspaces the
// persistent kernels use.  Passed by value to kernels.
struct ChainView {
    int L, V, Nt, N;            // N = V * Nt
    double delta, kappa, U;
    const double* E;            // V x V FP64, row-major, exactly symmetric
    // FP16 split of E for the tensor-core path (row-major, padded):
    //   E ~= (E_hi + E_lo * 2^-kLoShift) with rows and cols padded to Vp.
    const void* E_hi;           // __half [Vr][Vp]
    const void* E_lo;           // __half [Vr][Vp]
    int Vr, Vp;                 // padded rows (multiple of 128), cols (multiple of 64)
    // scaled FP16 split of the slice-major tensor-core tile:
    //   2^eE E ~= Ew_hi + Ew_lo (plain remainder), same padding; e_inv = 2^-eE
    const void* Ew_hi;          // __half [Vr][Vp]
    const void* Ew_lo;          // __half [Vr][Vp]
    float e_inv;
    // FP64 workspaces, double2 [Nt][V] each
    double2 *cis;               // exp(i phi)
    double2 *x, *r, *p, *q, *chi, *rho;
    double2 *xh;                // solution history for the mixed trajectory's guesses
    double2 *chi2, *phi2, *x2;  // mass preconditioning: second pseudofermion, M_g chi2,
                                // and its solve (allocated when hb_inner > 0)
    double *pi, *phi_old;       // double [Nt][V]
    // FP32 workspaces for the mixed path, float2 [Nt][V] each
    float2 *cis_f, *r_f, *p_f, *p2_f, *q_f, *x_f;
    // split-K CG (operand_mode 5): G = E p' carried per target slice, and
    // u = e^{i phi} q, the source of the M application
    float2 *g_f, *u_f;
    unsigned long long* gslots; // sequence-numbered partial sums and totals (tc_splitk.cuh)
    // team synchronisation
    unsigned* bar;              // 2 words
    int* status;                // device status block (kStatusBlockBytes): status
                                // word, then the wait limit (common.cuh)
    int team_pad;               // testing only: CTAs every team barrier expects
                                // beyond those launched (0 in normal use)
    double* partials;           // kSlots * kMaxTeam * kVals
    double* scalars;            // per-call scalar outputs (see kernels)
};

}  // namespace hmc

namespace hmc {
struct TcCtx;
}

struct hmc_ctx {
    hmc_params params;
    hmc::TcCtx* tc;             // tensor-core path state (tc_kernels.cu)
    int device;
    int num_sms;
    hmc::ChainView view;
    // owned device allocations (freed by hmc_ctx_destroy)
    void* allocs[64];
    int n_allocs;
    double* scalars_host;       // pinned, mirrors view.scalars
};
