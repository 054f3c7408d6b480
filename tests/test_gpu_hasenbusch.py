"""Mass preconditioning with the nested leapfrog on the GPU against the
oracle, trajectory by trajectory: Delta H, the proposed field, the Metropolis
uniform and decision, and the number of solves of each level; g = 0 with one
inner step against the plain trajectory; a chain of trajectories following
the oracle's chain.  FP64 path: Delta H and the field to 1e-10.  Mixed path
(split-K tiles, the heavy operator's hop factor in their epilogues; every
solve to an FP64 true residual of 1e-10): Delta H 1e-7, the field 1e-8, as
the plain mixed trajectory."""
import numpy as np
import pytest
import torch

from oracle import hasenbusch as hb, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def params(L, Nt, beta, U, g, n_inner, n_md, tau, **kw):
    return hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=n_md, traj_length=tau, cg_tol=1e-12,
                      hb_gamma=g, hb_inner=n_inner, **kw)


@pytest.mark.parametrize("L,Nt,beta,U,g,n_inner,n_md", [
    (3, 8, 2.0, 2.0, 0.5, 3, 4), (3, 8, 2.0, 2.0, 0.8, 1, 5), (2, 5, 1.5, 3.0, 0.3, 2, 3),
    (6, 16, 2.0, 3.5, 0.6, 4, 3)])
def test_hasenbusch_trajectory_matches_oracle(L, Nt, beta, U, g, n_inner, n_md):
    V, delta, tau = 2 * L * L, beta / Nt, 0.6
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    phi = synth.gaussian_field(20 + L, Nt, V, delta * U, scale=0.5)
    ctx = hmc.Context(params(L, Nt, beta, U, g, n_inner, n_md, tau))
    t = torch.from_numpy(phi).to(DEV)
    out = ctx.trajectory(t, 13, 2, chain=1)
    want = hb.trajectory(E, phi, delta, U, g, tau / n_md, n_md, n_inner, 13, 2, chain=1,
                         tol=1e-13)
    assert out.status == hmc.HMC_OK
    assert abs(out.dH - want["dH"]) < 1e-10, (out.dH, want["dH"])
    assert out.u == want["u"] and bool(out.accept) == want["accept"]
    got = t.cpu().numpy()
    ref = want["phi_proposed"] if want["accept"] else phi
    assert np.abs(got - ref).max() < 1e-10
    assert out.cg_solves_outer == want["solves_outer"] == n_md + 1
    assert out.cg_solves - out.cg_solves_outer == want["solves_inner"] + 1   # + heat bath
    assert out.max_true_residual < 1e-11


def test_gamma_zero_single_inner_step_is_plain_fp64_trajectory():
    L, Nt, beta, U, n_md, tau = 3, 8, 2.0, 2.0, 6, 0.6
    V = 2 * L * L
    phi = synth.gaussian_field(5, Nt, V, beta / Nt * U, scale=0.5)
    a = torch.from_numpy(phi).to(DEV)
    b = a.clone()
    o_hb = hmc.Context(params(L, Nt, beta, U, 0.0, 1, n_md, tau)).trajectory(a, 9, 0)
    o_pl = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=n_md, traj_length=tau,
                                  cg_tol=1e-12)).trajectory(b, 9, 0)
    assert abs(o_hb.dH - o_pl.dH) < 1e-10
    assert torch.allclose(a, b, rtol=0, atol=1e-11)


def test_hasenbusch_chain_follows_oracle():
    L, Nt, beta, U, g, n_inner, n_md, tau = 3, 8, 2.0, 2.0, 0.5, 2, 5, 1.0
    V, delta = 2 * L * L, beta / Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    phi = synth.gaussian_field(31, Nt, V, delta * U, scale=0.5)
    ctx = hmc.Context(params(L, Nt, beta, U, g, n_inner, n_md, tau))
    t = torch.from_numpy(phi).to(DEV)
    acc = 0
    for traj in range(30):
        start = t.cpu().numpy()
        out = ctx.trajectory(t, 77, traj)
        want = hb.trajectory(E, start, delta, U, g, tau / n_md, n_md, n_inner, 77, traj,
                             tol=1e-13)
        assert abs(out.dH - want["dH"]) < 1e-9, traj
        assert bool(out.accept) == want["accept"], traj
        assert np.abs(t.cpu().numpy() - want["phi"]).max() < 1e-9, traj
        acc += out.accept
    assert acc >= 20


@pytest.mark.parametrize("mode", [0, 1, 3, 4])
def test_mixed_mass_preconditioning_needs_split_k_tiles(mode):
    ctx = hmc.Context(params(3, 8, 2.0, 2.0, 0.5, 2, 4, 0.5, precision=hmc.PREC_MIXED,
                             operand_mode=mode))
    t = torch.zeros((8, 18), dtype=torch.float64, device=DEV)
    with pytest.raises(hmc.HmcError) as e:
        ctx.trajectory(t, 1, 0)
    assert e.value.code == hmc.HMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("L,Nt,beta,U,g,n_inner,n_md,C", [
    (3, 8, 2.0, 2.0, 0.5, 3, 4, 2), (6, 16, 2.0, 3.5, 0.6, 4, 3, 4), (5, 12, 1.5, 3.0, 0.3, 2, 3, 2),
    (9, 16, 2.0, 3.5, 0.7, 3, 4, 4)])
def test_mixed_hasenbusch_trajectory_matches_oracle(L, Nt, beta, U, g, n_inner, n_md, C):
    V, delta, tau = 2 * L * L, beta / Nt, 0.6
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    phi = synth.gaussian_field(40 + L, Nt, V, delta * U, scale=0.4)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=n_md, traj_length=tau,
                                 cg_tol=1e-10, hb_gamma=g, hb_inner=n_inner,
                                 precision=hmc.PREC_MIXED, operand_mode=5, inner_ctas=C))
    t = torch.from_numpy(phi).to(DEV)
    out = ctx.trajectory(t, 13, 2, chain=1)
    want = hb.trajectory(E, phi, delta, U, g, tau / n_md, n_md, n_inner, 13, 2, chain=1,
                         tol=1e-13)
    assert out.status == hmc.HMC_OK and out.fp64_iterations == 0
    assert abs(out.dH - want["dH"]) < 1e-7, (out.dH, want["dH"])
    assert out.u == want["u"] and bool(out.accept) == want["accept"]
    ref = want["phi_proposed"] if want["accept"] else phi
    assert np.abs(t.cpu().numpy() - ref).max() < 1e-8
    assert out.cg_solves_outer == want["solves_outer"] == n_md + 1
    assert out.cg_solves - out.cg_solves_outer == want["solves_inner"] + 1   # + heat bath
    assert out.max_true_residual <= 1e-10
    # repeatable: the same trajectory again gives the same bits
    t2 = torch.from_numpy(phi).to(DEV)
    out2 = ctx.trajectory(t2, 13, 2, chain=1)
    assert out2.dH == out.dH and torch.equal(t2, t)


def test_mixed_hasenbusch_gamma_zero_single_inner_step_is_plain_mixed_physics():
    """g = 0 with one inner step: the same target and momenta schedule as the
    plain leapfrog; the mixed trajectory's Delta H agrees with the plain FP64
    one to the solver's accuracy (the mixed path's solves start from zero
    here, the plain mixed path extrapolates its guesses)."""
    L, Nt, beta, U, n_md, tau = 6, 16, 2.0, 3.5, 6, 0.6
    V = 2 * L * L
    phi = synth.gaussian_field(5, Nt, V, beta / Nt * U, scale=0.4)
    a = torch.from_numpy(phi).to(DEV)
    b = a.clone()
    o_hb = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=n_md, traj_length=tau,
                                  cg_tol=1e-10, hb_gamma=0.0, hb_inner=1,
                                  precision=hmc.PREC_MIXED, operand_mode=5)).trajectory(a, 9, 0)
    o_pl = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=n_md, traj_length=tau,
                                  cg_tol=1e-12)).trajectory(b, 9, 0)
    assert abs(o_hb.dH - o_pl.dH) < 1e-7
    assert torch.allclose(a, b, rtol=0, atol=1e-8)
