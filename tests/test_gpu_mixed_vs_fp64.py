"""The mixed path against the plain FP64 GPU path on the same seeded
trajectories of the two largest single-chain workloads at their full
trajectory length, from a field thermalised by mixed trajectories:

  L=12, Nt=64, U=3.8, beta=8, 20 leapfrog steps over tau=1
  L=24, Nt=96, U=4,   beta=12, 30 leapfrog steps over tau=1

Stated and bounded: the CG solution and the force built on it for the
heat-bath source chi = M rho of the thermalised field (both solves to the
FP64 true residual 1e-10), Delta H and the field after the same trajectory."""
import math

import pytest
import torch

from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


@pytest.mark.parametrize("name,n_therm", [("l12_nt64", 3), ("l24_nt96", 2)])
def test_mixed_vs_fp64_full_trajectory(name, n_therm):
    w = synth.WORKLOADS[name]
    base = dict(L=w["L"], Nt=w["Nt"], kappa=w["kappa"], U=w["U"], beta=w["beta"],
                n_md=w["n_md"], traj_length=w["traj_length"], cg_tol=w["cg_tol"],
                cg_max_iter=200000)
    c64 = hmc.Context(hmc.Params(**base, precision=hmc.PREC_FP64))
    cmx = hmc.Context(hmc.Params(**base, precision=hmc.PREC_MIXED))
    V, Nt = c64.params.V, w["Nt"]
    phi = torch.from_numpy(synth.start_field(name)).to(DEV)
    for k in range(n_therm):                   # thermalise from the cold start
        o = cmx.trajectory(phi, w["seed"], k)
        assert o.status == hmc.HMC_OK
    # CG solution and force for the heat-bath source of the thermalised field
    rho = torch.from_numpy(synth.complex_gaussian(5, Nt, V) / math.sqrt(2.0)).to(DEV)
    chi = c64.apply_M(phi, rho)
    x64, s64 = c64.cg_solve(phi, chi, prec=hmc.PREC_FP64)
    xmx, smx = cmx.cg_solve(phi, chi, prec=hmc.PREC_MIXED)
    assert s64.true_residual <= 1e-10 and smx.true_residual <= 1e-10
    err_x = rel(xmx, x64)
    err_F = rel(cmx.force(phi, xmx), c64.force(phi, x64))
    # the same seeded trajectory on both paths
    a, b = phi.clone(), phi.clone()
    o64 = c64.trajectory(a, w["seed"], 100)
    omx = cmx.trajectory(b, w["seed"], 100)
    assert o64.status == hmc.HMC_OK and omx.status == hmc.HMC_OK
    assert omx.max_true_residual <= 1e-10
    err_dH = abs(omx.dH - o64.dH)
    err_phi = rel(b, a)
    print("\nmixed vs FP64 (%s, %d x %.4f): |dx|/|x| = %.2e, |dF|/|F| = %.2e, "
          "|d(Delta H)| = %.2e (Delta H = %.4f), |dphi|/|phi| = %.2e; CG iterations of the "
          "solve %d (FP64) vs %d (mixed, %d FP64 reliable updates); trajectory %d vs %d"
          % (name, w["n_md"], w["traj_length"] / w["n_md"], err_x, err_F, err_dH, o64.dH,
             err_phi, s64.iterations, smx.iterations, smx.reliable_updates,
             o64.cg_iterations, omx.cg_iterations))
    assert err_x < 1e-8
    assert err_F < 1e-8
    assert err_dH < 1e-6
    assert err_phi < 1e-8
    assert o64.accept == omx.accept
