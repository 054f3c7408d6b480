"""The full batched workload (256 chains of uneven size, L in {3,6,9,12},
Nt in {16,32,48,64}) in the launch configuration the benchmark times: the
autotuned shapes, cluster teams of 4 for the chains that would finish last,
one persistent launch per trajectory.  Every chain must reach the mixed
path's true residual; a sample of chains (the cheapest one-CTA chain of each
L and the first team chain) is compared with the oracle's trajectory from the
same cold start, seed, trajectory index and chain id."""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import autotune, hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def workload_params():
    return [hmc.Params(L=c["L"], Nt=c["Nt"], kappa=c["kappa"], U=c["U"], beta=c["beta"],
                       n_md=c["n_md"], traj_length=c["traj_length"], cg_tol=c["cg_tol"],
                       cg_max_iter=200000, precision=hmc.PREC_MIXED)
            for c in synth.batch256()]


def sampled_chains(plist):
    picks = []
    for L in (3, 6, 9, 12):
        solo = [i for i, p in enumerate(plist) if p.L == L and p.team_ctas <= 1]
        if solo:
            picks.append(min(solo, key=lambda i: (plist[i].Nt, i)))
    teams = [i for i, p in enumerate(plist) if p.team_ctas > 1]
    if teams:
        picks.append(teams[0])
    return picks


def test_batch256_in_the_benchmark_shapes_matches_oracle_on_sampled_chains():
    plist = autotune.batch_shapes(workload_params(), csize=4)
    assert len(plist) == 256
    b = hmc.Batch(plist)
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)   # cold start
    seed, traj = synth.BASE_SEED + 3, 0
    outs = b.trajectory(phi, seed, traj)
    assert all(o.status == 0 for o in outs)
    assert max(o.max_true_residual for o in outs) <= 1e-10
    picks = sampled_chains(plist)
    assert len(picks) >= 4
    for i in picks:
        p = plist[i]
        E = ops.transfer_matrix(lattice.hopping_matrix(p.L), p.delta)
        want = ohmc.trajectory(E, np.zeros((p.Nt, p.V)), p.delta, p.U, p.traj_length / p.n_md,
                               p.n_md, seed, traj, chain=i, tol=1e-12)
        assert abs(outs[i].dH - want["dH"]) < 1e-7, (i, p.L, p.Nt, outs[i].dH, want["dH"])
        assert bool(outs[i].accept) == want["accept"]
        got = b.view(phi, i).cpu().numpy()
        assert np.linalg.norm(got - want["phi"]) <= 1e-8 * np.linalg.norm(want["phi"]), (i, p.L)
