"""Batched chains (one persistent launch, CUDA graph) against single-chain
trajectories of the same chains and against the oracle."""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# uneven sizes: ragged site blocks, Nt = 1 excluded only because of n_md
CHAINS = [(3, 8, 2.0), (2, 5, 3.0), (3, 16, 4.0), (6, 16, 3.5), (1, 4, 2.5), (4, 12, 3.0),
          (6, 8, 5.0)]


def params(L, Nt, U, **kw):
    return hmc.Params(L=L, Nt=Nt, U=U, beta=0.125 * Nt * 2, n_md=4, traj_length=0.5,
                      cg_tol=1e-10, precision=hmc.PREC_MIXED, **kw)


def start_fields():
    return [synth.gaussian_field(10 + i, Nt, 2 * L * L, 0.25 * U / 4, scale=0.5)
            for i, (L, Nt, U) in enumerate(CHAINS)]


def test_batch_matches_single_chain_runs():
    b = hmc.Batch([params(*c) for c in CHAINS])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = start_fields()
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    singles = [hmc.Context(params(*c, team_ctas=1, inner_ctas=1)) for c in CHAINS]
    sphi = [torch.from_numpy(f).to(DEV) for f in fields]
    for traj in range(2):                     # second call replays the graph
        outs = b.trajectory(phi, 99, traj)
        for i, c in enumerate(singles):
            o = c.trajectory(sphi[i], 99, traj, chain=i)
            assert outs[i].status == 0 and o.status == 0
            assert outs[i].dH == o.dH, (i, outs[i].dH, o.dH)     # same arithmetic, bitwise
            assert outs[i].accept == o.accept
            assert outs[i].cg_iterations == o.cg_iterations
            assert torch.equal(b.view(phi, i), sphi[i])


def test_batch_matches_oracle():
    sel = [0, 3, 4]
    chains = [CHAINS[i] for i in sel]
    b = hmc.Batch([params(*c) for c in chains])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = [start_fields()[i] for i in sel]
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    outs = b.trajectory(phi, 7, 0)
    for i, (L, Nt, U) in enumerate(chains):
        p = params(L, Nt, U)
        E = ops.transfer_matrix(lattice.hopping_matrix(L), p.delta)
        want = ohmc.trajectory(E, fields[i], p.delta, U, p.traj_length / p.n_md, p.n_md, 7, 0,
                               chain=i, tol=1e-12)
        assert outs[i].max_true_residual <= 1e-10
        assert abs(outs[i].dH - want["dH"]) < 1e-7
        assert bool(outs[i].accept) == want["accept"]
        got = b.view(phi, i).cpu().numpy()
        assert np.linalg.norm(got - want["phi"]) <= 1e-8 * np.linalg.norm(want["phi"])


def test_batch_rejects_fp64_chains():
    with pytest.raises(hmc.HmcError) as e:
        hmc.Batch([hmc.Params(L=2, Nt=4, precision=hmc.PREC_FP64)])
    assert e.value.code == hmc.HMC_ERR_UNSUPPORTED


# cluster teams in the batch: (L, Nt, U, operand_mode, team_ctas); team chains
# run on a cluster of 4 CTAs (slice-major, site-major and CUDA-core kinds),
# the rest on one CTA each
TEAM_CHAINS = [(9, 16, 3.0, 4, 4), (6, 16, 3.5, 1, 4), (6, 32, 3.0, 3, 4), (3, 8, 2.0, 4, 1),
               (12, 16, 3.0, 4, 4), (2, 5, 3.0, 1, 1), (6, 8, 5.0, 3, 1)]


def test_batch_cluster_teams_match_single_chains_and_oracle():
    def tparams(L, Nt, U, mode, team):
        return params(L, Nt, U, operand_mode=mode, team_ctas=team, inner_ctas=team)
    b = hmc.Batch([tparams(*c) for c in TEAM_CHAINS])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = [synth.gaussian_field(40 + i, Nt, 2 * L * L, 0.25 * U / 4, scale=0.5)
              for i, (L, Nt, U, _, _) in enumerate(TEAM_CHAINS)]
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    for traj in range(2):
        outs = b.trajectory(phi, 17, traj)
        for i, (L, Nt, U, mode, team) in enumerate(TEAM_CHAINS):
            single = hmc.Context(tparams(L, Nt, U, mode, team))
            sphi = torch.from_numpy(fields[i]).to(DEV)
            o = single.trajectory(sphi, 17, traj, chain=i)
            assert outs[i].status == 0 and o.status == 0, (i, outs[i].status, o.status)
            # same launch shape and summation order: bitwise
            assert outs[i].dH == o.dH, (i, outs[i].dH, o.dH)
            assert outs[i].cg_iterations == o.cg_iterations
            assert torch.equal(b.view(phi, i), sphi)
            p = params(L, Nt, U)
            E = ops.transfer_matrix(lattice.hopping_matrix(L), p.delta)
            want = ohmc.trajectory(E, fields[i], p.delta, U, p.traj_length / p.n_md, p.n_md,
                                   17, traj, chain=i, tol=1e-12)
            assert outs[i].max_true_residual <= 1e-10
            assert abs(outs[i].dH - want["dH"]) < 1e-7
            assert bool(outs[i].accept) == want["accept"]
            fields[i] = b.view(phi, i).cpu().numpy()


def test_batch_rejects_mixed_team_sizes():
    with pytest.raises(hmc.HmcError) as e:
        hmc.Batch([params(3, 8, 2.0, team_ctas=2), params(3, 8, 2.0, team_ctas=4)])
    assert e.value.code == hmc.HMC_ERR_UNSUPPORTED
