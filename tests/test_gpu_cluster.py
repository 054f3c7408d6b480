"""Inner CG team as one thread-block cluster (distributed-shared-memory
barriers and sums) against the global-memory team barriers and the oracle.

Both synchronisation paths sum the per-CTA partials in the same fixed order,
so for the same launch shape the two give bit-identical solutions; each is
also checked against the FP64 oracle operator (true residual 1e-10).
Resident E with more CTAs than 128-site blocks (extra CTAs take further slice
tiles of the same block) is covered by the same cases, and so is the
CUDA-core cluster mode for small lattices (operand_mode 3: E and the FP32
iterates in the cluster's shared memory, halo slices through distributed
shared memory), including ragged slice splits and one slice per CTA.
"""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def oracle_E(L, Nt, beta, kappa=1.0):
    return ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


# (L, Nt, team_ctas, inner_ctas, tile_slices, operand_mode)
SHAPES = [
    (6, 32, 12, 4, 8, 1),     # streamed E, 4 slice tiles on 4 CTAs
    (6, 32, 8, 4, 8, 2),      # resident E, 4 CTAs share the one site block
    (6, 32, 8, 2, 16, 2),
    (9, 16, 8, 4, 8, 2),      # V = 162: 2 site blocks x 2 slice-tile groups
    (12, 64, 16, 8, 16, 1),   # V = 288: 3 site blocks x 4 slice tiles on 8 CTAs
    (3, 24, 6, 3, 8, 1),      # odd cluster size
]


@pytest.mark.parametrize("L,Nt,team,inner,ns,mode", SHAPES)
def test_cg_cluster_matches_global_and_oracle(L, Nt, team, inner, ns, mode):
    beta, U = 0.125 * Nt, 3.5
    V = 2 * L * L
    phi = synth.gaussian_field(41 + L, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(42 + L, Nt, V)
    xs = []
    for cm in (1, 2):          # cluster required / never
        c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, team_ctas=team,
                                   inner_ctas=inner, tile_slices=ns, operand_mode=mode,
                                   cluster_mode=cm))
        x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
        assert st.status == 0
        assert st.true_residual <= 1e-10
        xs.append((x, st))
        c.close()
    (xa, sa), (xb, sb) = xs
    assert sa.iterations == sb.iterations
    assert torch.equal(xa, xb)
    E = oracle_E(L, Nt, beta)
    res = chi - ops.apply_MMdag(E, phi, xa.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10


def test_trajectory_cluster_matches_oracle():
    L, Nt, beta, U, n_md, tau = 6, 32, 4.0, 3.5, 3, 0.3
    delta = beta / Nt
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=tau,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, team_ctas=8,
                               inner_ctas=4, tile_slices=8, operand_mode=2, cluster_mode=1))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(9, Nt, V, delta * U, scale=0.5)
    phi = dev(phi_np)
    want = ohmc.trajectory(E, phi_np, delta, U, tau / n_md, n_md, 5, 0, 0, tol=1e-12)
    out = c.trajectory(phi, 5, 0)
    assert out.status == 0
    assert out.max_true_residual <= 1e-10
    assert abs(out.dH - want["dH"]) < 1e-7
    assert bool(out.accept) == want["accept"]
    assert np.linalg.norm(phi.cpu().numpy() - want["phi"]) <= 1e-8 * np.linalg.norm(want["phi"])


def test_cluster_required_without_multi_cta_team_is_refused():
    """cluster_mode = 1 with a one-CTA inner team is refused on the host."""
    L, Nt = 3, 8
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=1.0, U=3.0, team_ctas=2, inner_ctas=1,
                               cluster_mode=1))
    phi = torch.zeros((Nt, 18), dtype=torch.float64, device=DEV)
    chi = torch.ones((Nt, 18), dtype=torch.complex128, device=DEV)
    with pytest.raises(hmc.HmcError) as ei:
        c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert ei.value.code == -6


# CUDA-core cluster mode (operand_mode 3): (L, Nt, team_ctas, inner_ctas = cluster size)
SMALL = [
    (6, 32, 8, 8),     # 4 slices per CTA
    (6, 32, 12, 4),    # FP64 team larger than the cluster
    (6, 32, 1, 1),     # one CTA, 32 slices is above 16: refused (checked below)
    (3, 8, 2, 2),
    (1, 3, 1, 1),      # V = 2
    (5, 13, 4, 4),     # ragged split: 3, 3, 3, 4 slices
    (2, 5, 5, 5),      # one slice per CTA, odd cluster size
    (8, 64, 8, 8),     # V = 128
    (4, 16, 2, 2),     # 8 slices each, prev = next
]


@pytest.mark.parametrize("L,Nt,team,inner", [s for s in SMALL if s != (6, 32, 1, 1)])
def test_cg_small_cluster_mode(L, Nt, team, inner):
    beta, U = 0.125 * Nt, 3.5
    V = 2 * L * L
    phi = synth.gaussian_field(61 + L, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(62 + L, Nt, V)
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, team_ctas=team, inner_ctas=inner,
                               operand_mode=3))
    x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == 0
    assert st.true_residual <= 1e-10
    assert st.reliable_updates >= 1
    E = oracle_E(L, Nt, beta)
    res = chi - ops.apply_MMdag(E, phi, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10
    # same iteration count regime as the FP64 solver
    _, st64 = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_FP64)
    assert st.iterations < 3 * st64.iterations + 20


def test_cg_small_cluster_mode_deterministic():
    L, Nt = 6, 32
    V = 2 * L * L
    phi = dev(synth.gaussian_field(3, Nt, V, 0.4375, scale=0.5))
    chi = dev(synth.complex_gaussian(4, Nt, V))
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=4.0, U=3.5, team_ctas=8, inner_ctas=8,
                               operand_mode=3))
    x1, s1 = c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    x2, s2 = c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert s1.iterations == s2.iterations
    assert torch.equal(x1, x2)


def test_trajectory_small_cluster_mode_matches_oracle():
    L, Nt, beta, U, n_md, tau = 6, 32, 4.0, 3.5, 3, 0.3
    delta = beta / Nt
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=tau,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, team_ctas=8,
                               inner_ctas=8, operand_mode=3))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(10, Nt, V, delta * U, scale=0.5)
    phi = dev(phi_np)
    for traj in range(2):
        want = ohmc.trajectory(E, phi_np, delta, U, tau / n_md, n_md, 6, traj, 0, tol=1e-12)
        out = c.trajectory(phi, 6, traj)
        assert out.status == 0
        assert out.max_true_residual <= 1e-10
        assert abs(out.dH - want["dH"]) < 1e-7
        assert bool(out.accept) == want["accept"]
        got = phi.cpu().numpy()
        assert np.linalg.norm(got - want["phi"]) <= 1e-8 * np.linalg.norm(want["phi"])
        phi_np = want["phi"]


@pytest.mark.parametrize("kw", [dict(team_ctas=1, inner_ctas=1),        # 32 slices > 16
                                dict(team_ctas=8, inner_ctas=8, cluster_mode=2),
                                dict(team_ctas=6, inner_ctas=3, L=2, Nt=2)])
def test_small_cluster_mode_refusals(kw):
    p = dict(L=6, Nt=32, beta=4.0, U=3.5, operand_mode=3)
    p.update(kw)
    c = hmc.Context(hmc.Params(**p))
    V = 2 * p["L"] ** 2
    phi = torch.zeros((p["Nt"], V), dtype=torch.float64, device=DEV)
    chi = torch.ones((p["Nt"], V), dtype=torch.complex128, device=DEV)
    with pytest.raises(hmc.HmcError) as ei:
        c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert ei.value.code == -6


@pytest.mark.parametrize("L,Nt", [(6, 32), (8, 64), (5, 23)])
def test_cg_small_cluster_of_16(L, Nt):
    """A cluster of 16 CTAs (non-portable size; skipped where the device
    refuses it): 2 to 4 slices per CTA, ragged at Nt = 23."""
    beta, U = 0.125 * Nt, 3.5
    V = 2 * L * L
    phi = synth.gaussian_field(71 + L, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(72 + L, Nt, V)
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, team_ctas=16, inner_ctas=16,
                               operand_mode=3))
    try:
        x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    except hmc.HmcError as e:
        if e.code == -6:
            pytest.skip("device refuses a cluster of 16 CTAs")
        raise
    assert st.status == 0 and st.true_residual <= 1e-10
    E = oracle_E(L, Nt, beta)
    res = chi - ops.apply_MMdag(E, phi, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10
