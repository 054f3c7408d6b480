"""Trajectories with the second-order minimum-norm (Omelyan) integrator
(hmc_params.integrator = 1) against the oracle's schedule, on the plain FP64
path (1e-10), the mixed tensor-core path and the mixed CUDA-core cluster mode
(Delta H to 1e-7, phi to 1e-8 relative, the mixed path's tolerances)."""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def oracle_E(L, Nt, beta, kappa=1.0):
    return ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_omelyan_fp64_matches_oracle():
    L, Nt, beta, U, n_md, tau = 3, 8, 2.0, 2.0, 5, 1.0
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=tau,
                               cg_tol=1e-12, precision=hmc.PREC_FP64, integrator=1))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(21, Nt, 18, delta * U, scale=0.5)
    phi = dev(phi_np)
    for traj in range(3):
        want = ohmc.trajectory(E, phi_np, delta, U, tau / n_md, n_md, 31, traj, 0, tol=1e-12,
                               integrator="omelyan")
        out = c.trajectory(phi, 31, traj)
        assert out.status == 0
        assert out.cg_solves == want["cg_solves"] == 2 * n_md + 1
        assert abs(out.dH - want["dH"]) < 1e-10 * max(1.0, abs(want["H0"]))
        assert bool(out.accept) == want["accept"]
        assert rel(phi.cpu().numpy(), want["phi"]) < 1e-10
        phi_np = want["phi"]


@pytest.mark.parametrize("shape", [dict(operand_mode=1), dict(operand_mode=2),
                                   dict(operand_mode=3, team_ctas=2, inner_ctas=2)])
def test_omelyan_mixed_matches_oracle(shape):
    L, Nt, beta, U, n_md, tau = 3, 8, 2.0, 2.0, 4, 1.0
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=tau,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, integrator=1, **shape))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(22, Nt, 18, delta * U, scale=0.5)
    phi = dev(phi_np)
    for traj in range(2):
        want = ohmc.trajectory(E, phi_np, delta, U, tau / n_md, n_md, 32, traj, 0, tol=1e-12,
                               integrator="omelyan")
        out = c.trajectory(phi, 32, traj)
        assert out.status == 0
        assert out.cg_solves == 2 * n_md + 1
        assert out.max_true_residual <= 1e-10
        assert abs(out.dH - want["dH"]) < 1e-7
        assert bool(out.accept) == want["accept"]
        assert rel(phi.cpu().numpy(), want["phi"]) < 1e-8
        phi_np = want["phi"]


def test_omelyan_smaller_delta_h_on_gpu():
    """Same seeded trajectories at L=6, Nt=32 (cluster mode): RMS Delta H of
    the minimum-norm integrator with 10 steps is well below leapfrog's with
    20 steps (both 21 force evaluations' worth of solves or fewer)."""
    L, Nt, beta, U = 6, 32, 4.0, 3.5
    V = 2 * L * L
    phi0 = dev(synth.gaussian_field(23, Nt, V, beta / Nt * U, scale=0.5))
    res = {}
    for integ, n_md in ((0, 20), (1, 10)):
        c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=1.0,
                                   cg_tol=1e-10, precision=hmc.PREC_MIXED, integrator=integ,
                                   operand_mode=3, team_ctas=8, inner_ctas=8))
        dh = []
        for traj in range(6):
            phi = phi0.clone()
            dh.append(c.trajectory(phi, 40, traj).dH)
        res[integ] = np.sqrt(np.mean(np.square(dh)))
    assert res[1] < 0.5 * res[0], res
