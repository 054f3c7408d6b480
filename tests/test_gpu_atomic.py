"""Long GPU chains in the atomic limit (kappa = 0), through the C ABI.

The FP64 chain follows the oracle's chain trajectory by trajectory over 610
trajectories (same Philox draws, identical accept decisions, fields within
1e-9).  Both precisions reproduce <cos Phi_x> of the atomic-limit weight
N(0, beta U) x (2 + 2 cos Phi), the distribution pinned against the §1
Hamiltonian in test_oracle_atomic.py, within 4 standard errors.
"""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc
from test_oracle_atomic import ATOM, cos_phase_target

pytestmark = pytest.mark.gpu


def gpu_chain(precision, cg_tol):
    a = ATOM
    c = hmc.Context(hmc.Params(L=a["L"], Nt=a["Nt"], kappa=0.0, U=a["U"], beta=a["beta"],
                               n_md=a["n_md"], traj_length=a["eps"] * a["n_md"],
                               cg_tol=cg_tol, precision=precision))
    phi = torch.zeros((a["Nt"], 2 * a["L"] ** 2), dtype=torch.float64, device="cuda:0")
    fields, outs = [], []
    for traj in range(a["n_therm"] + a["n_traj"]):
        outs.append(c.trajectory(phi, a["seed"], traj))
        fields.append(phi.cpu().numpy().copy())
    return fields, outs


def cos_stats(fields):
    vals = np.array([np.cos(f.sum(axis=0)).mean() for f in fields[ATOM["n_therm"]:]])
    blocks = vals.reshape(20, -1).mean(axis=1)
    return vals.mean(), blocks.std(ddof=1) / np.sqrt(len(blocks))


def test_fp64_chain_follows_oracle_and_samples_atomic_limit():
    a = ATOM
    fields, outs = gpu_chain(hmc.PREC_FP64, 1e-12)
    delta = a["beta"] / a["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(a["L"]), 0.0)
    phi = np.zeros((a["Nt"], 2 * a["L"] ** 2))
    for traj, (f, o) in enumerate(zip(fields, outs)):
        want = ohmc.trajectory(E, phi, delta, a["U"], eps=a["eps"], n_md=a["n_md"],
                               seed=a["seed"], traj=traj, tol=1e-12)
        assert o.status == 0
        assert o.u == want["u"]
        assert bool(o.accept) == want["accept"], traj
        assert abs(o.dH - want["dH"]) < 1e-9, (traj, o.dH, want["dH"])
        assert np.abs(f - want["phi"]).max() < 1e-9, traj
        phi = want["phi"]
    mean, err = cos_stats(fields)
    assert abs(mean - cos_phase_target()) < 4.0 * err, (mean, err)


def test_mixed_chain_samples_atomic_limit():
    fields, outs = gpu_chain(hmc.PREC_MIXED, 1e-10)
    assert all(o.status == 0 for o in outs)
    assert np.mean([o.accept for o in outs]) > 0.9
    assert max(o.max_true_residual for o in outs) <= 1e-10
    mean, err = cos_stats(fields)
    assert err < 0.015
    assert abs(mean - cos_phase_target()) < 4.0 * err, (mean, err)
