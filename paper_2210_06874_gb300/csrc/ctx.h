// ctx.h -- the opaque hmc_ctx and the per-chain device view handed to kernels.
#pragma once

#include <cuda_fp16.h>
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
    // split-K CG (operand_mode 5): the sources of its applications with a
    // one-slice halo, rows [Nt + 2][V]: row t + 1 holds slice t, row 0 slice
    // Nt - 1 and row Nt + 1 slice 0, so every n-group's shifted source
    // slices are contiguous rows; u = e^{i phi} q (source of M) and r (source
    // of M^dag); sk_maps: their TMA maps in global memory (CUtensorMap[2]:
    // r, u; null when the context has no split-K shape)
    float2 *g_f, *u_f, *rh_f;
    // ... and their FP16 splits (plain remainder) at a team-uniform scale,
    // written by the owners, rows [2 (Nt + 2)][Vp] (row 2h: Re, 2h + 1: Im
    // of halo row h), in the order r hi, r lo, u hi, u lo
    __half_raw* sk_b16;
    // sk_maps: CUtensorMap[6] in global memory: [0] r, [1] u (FP32 halo
    // rows), [2] r hi, [3] r lo, [4] u hi, [5] u lo (FP16, boxes of sk_nn(ns)
    // rows, 128-byte swizzle); null when the context has no split-K shape
    const void* sk_maps;
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
