"""The mixed path against the plain FP64 GPU path on the same
seeded trajectories (L=12, Nt=64, U=3.8, beta=8), with the differences in
Delta H, the force and the CG solution stated and bounded."""
import numpy as np
import pytest
import torch

from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_mixed_vs_fp64_l12_nt64():
    w = synth.WORKLOADS["l12_nt64"]
    base = dict(L=w["L"], Nt=w["Nt"], kappa=w["kappa"], U=w["U"], beta=w["beta"], n_md=4,
                traj_length=0.25, cg_tol=1e-10)
    c64 = hmc.Context(hmc.Params(**base, precision=hmc.PREC_FP64))
    cmx = hmc.Context(hmc.Params(**base, precision=hmc.PREC_MIXED))
    V, Nt = c64.params.V, w["Nt"]
    delta = w["beta"] / Nt
    phi0 = torch.from_numpy(synth.gaussian_field(3, Nt, V, delta * w["U"], scale=0.3)).to(DEV)
    # CG solution and force at the start field
    chi = torch.from_numpy(synth.complex_gaussian(4, Nt, V)).to(DEV)
    x64, s64 = c64.cg_solve(phi0, chi, prec=hmc.PREC_FP64)
    xmx, smx = cmx.cg_solve(phi0, chi, prec=hmc.PREC_MIXED)
    assert s64.true_residual <= 1e-10 and smx.true_residual <= 1e-10
    err_x = (torch.linalg.vector_norm(xmx - x64) / torch.linalg.vector_norm(x64)).item()
    F64 = c64.force(phi0, x64)
    Fmx = cmx.force(phi0, xmx)
    err_F = (torch.linalg.vector_norm(Fmx - F64) / torch.linalg.vector_norm(F64)).item()
    # the same seeded trajectory on both paths
    a, b = phi0.clone(), phi0.clone()
    o64 = c64.trajectory(a, 11, 0)
    omx = cmx.trajectory(b, 11, 0)
    err_dH = abs(omx.dH - o64.dH)
    err_phi = (torch.linalg.vector_norm(b - a) / torch.linalg.vector_norm(a)).item()
    print("\nmixed vs FP64 (L=12, Nt=64): |dx|/|x| = %.2e, |dF|/|F| = %.2e, "
          "|d(Delta H)| = %.2e, |dphi|/|phi| = %.2e; CG iterations %d (FP64) vs %d (mixed, "
          "%d FP64 reliable updates)" % (err_x, err_F, err_dH, err_phi, s64.iterations,
                                          smx.iterations, smx.reliable_updates))
    assert err_x < 1e-8
    assert err_F < 1e-8
    assert err_dH < 1e-7
    assert err_phi < 1e-9
    assert o64.accept == omx.accept
