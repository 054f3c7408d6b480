"""Split-K tensor-core tiles with the transfer matrix resident in shared
memory (operand_mode 5): the FP32 iterations of the mixed CG run on
thread-block clusters that split the contraction's K, sum the partials
through distributed shared memory and the team's norms through
sequence-numbered slots.  Checked against the oracle (CG solution, a
trajectory) and the plain FP64 GPU path (L=24), over cluster sizes, slices
per n-group, ragged site blocks (V = 18, 50, 162) and ragged n-groups."""
import math

import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_E(L, Nt, beta):
    return ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt)


# (L, Nt, beta, U, cluster CTAs, slices per n-group)
CASES = [(3, 8, 1.0, 3.0, 2, 0), (5, 12, 1.5, 3.0, 2, 5), (6, 32, 4.0, 3.5, 2, 0),
         (6, 32, 4.0, 3.5, 4, 12), (9, 48, 6.0, 3.5, 6, 0), (9, 48, 6.0, 3.5, 4, 20),
         (12, 64, 8.0, 3.8, 6, 0), (12, 64, 8.0, 3.8, 8, 32), (12, 64, 8.0, 3.8, 4, 0)]


@pytest.mark.parametrize("L,Nt,beta,U,C,ns", CASES)
def test_splitk_cg_matches_oracle(L, Nt, beta, U, C, ns):
    V = 2 * L * L
    phi = synth.gaussian_field(L * 10 + Nt, Nt, V, beta / Nt * U, scale=0.4)
    chi = synth.complex_gaussian(L * 10 + Nt + 1, Nt, V)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, precision=hmc.PREC_MIXED,
                                 operand_mode=5, inner_ctas=C, tile_slices=ns))
    tphi, tchi = torch.from_numpy(phi).to(DEV), torch.from_numpy(chi).to(DEV)
    x, st = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == hmc.HMC_OK and st.true_residual <= 1e-10
    # the FP32 iteration itself converged (no switch to FP64 CG after a stall)
    assert st.fp64_iterations == 0
    xo, _, _ = ohmc.cg_solve(oracle_E(L, Nt, beta), phi, chi, tol=1e-14, max_iter=100000)
    assert rel(x.cpu().numpy(), xo) < 1e-8
    # deterministic: the same solve gives the same bits
    x2, st2 = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert st2.iterations == st.iterations and torch.equal(x, x2)


@pytest.mark.parametrize("L,Nt,C", [(3, 8, 2), (6, 16, 4)])
def test_splitk_trajectory_matches_oracle(L, Nt, C):
    beta, U = 0.125 * Nt * 2, 3.0
    V = 2 * L * L
    phi = synth.gaussian_field(7 + L, Nt, V, beta / Nt * U, scale=0.4)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, n_md=4, traj_length=0.5,
                                 cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=5,
                                 inner_ctas=C))
    t = torch.from_numpy(phi).to(DEV)
    out = ctx.trajectory(t, 31, 0)
    want = ohmc.trajectory(oracle_E(L, Nt, beta), phi, beta / Nt, U, 0.125, 4, 31, 0,
                           tol=1e-12)
    assert out.status == hmc.HMC_OK and out.max_true_residual <= 1e-10
    assert abs(out.dH - want["dH"]) < 1e-7
    assert bool(out.accept) == want["accept"]
    assert rel(t.cpu().numpy(), want["phi"]) < 1e-8


@pytest.mark.parametrize("C,ns", [(6, 0), (6, 48)])
def test_splitk_l24_matches_fp64_path(C, ns):
    w = synth.WORKLOADS["l24_nt96"]
    L, Nt, beta, U = w["L"], w["Nt"], w["beta"], w["U"]
    V = 2 * L * L
    base = dict(L=L, Nt=Nt, beta=beta, U=U, cg_tol=1e-10, cg_max_iter=200000)
    c64 = hmc.Context(hmc.Params(**base))
    csk = hmc.Context(hmc.Params(**base, precision=hmc.PREC_MIXED, operand_mode=5,
                                 inner_ctas=C, tile_slices=ns))
    phi = torch.from_numpy(synth.gaussian_field(91, Nt, V, beta / Nt * U, scale=0.3)).to(DEV)
    rho = torch.from_numpy(synth.complex_gaussian(92, Nt, V) / math.sqrt(2.0)).to(DEV)
    chi = c64.apply_M(phi, rho)
    x64, s64 = c64.cg_solve(phi, chi, prec=hmc.PREC_FP64)
    xsk, ssk = csk.cg_solve(phi, chi, prec=hmc.PREC_MIXED)
    print("\nL=24 split-K C=%d: iterations %d (+%d FP64 updates), FP64 path %d" %
          (C, ssk.iterations, ssk.reliable_updates, s64.iterations))
    assert ssk.status == hmc.HMC_OK and ssk.true_residual <= 1e-10
    err = (torch.linalg.vector_norm(xsk - x64) / torch.linalg.vector_norm(x64)).item()
    assert err < 1e-8


# Standalone applications on split-K tiles (k_apply_sk): pre-split source by
# TMA, E's rows x K range by TMA, cluster K split summed through distributed
# shared memory.  Tolerance 2e-6 (22-bit operands, FP32 sums), normwise and
# for the largest element error against the largest element.
APPLY_SIZES = [(3, 8, 0, 0), (3, 9, 0, 0), (5, 13, 0, 0), (6, 32, 0, 0), (7, 9, 0, 0),
               (6, 1, 0, 0), (9, 48, 0, 0), (12, 64, 0, 0), (24, 96, 0, 0), (12, 64, 8, 32),
               (9, 48, 4, 20), (24, 96, 8, 0), (24, 96, 6, 32), (12, 16, 4, 0),
               (12, 64, 4, 0), (24, 96, 7, 40)]


@pytest.mark.parametrize("L,Nt,C,ns", APPLY_SIZES)
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_splitk_apply_matches_oracle(L, Nt, C, ns, mu):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    delta = beta / Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta, delta * mu)
    phi = synth.gaussian_field(L * 100 + Nt + 7, Nt, V, delta * U)
    psi = torch.from_numpy(synth.complex_gaussian(L * 1000 + Nt + 7, Nt, V)).to(
        DEV, torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, mu=mu, precision=hmc.PREC_MIXED,
                                 operand_mode=5, inner_ctas=C, tile_slices=ns))
    tphi = torch.from_numpy(phi).to(DEV)
    for dag, want in ((False, ops.apply_M(E, phi, psi_in)), (True, ops.apply_Mdag(E, phi, psi_in))):
        f = ctx.apply_Mdag if dag else ctx.apply_M
        got = f(tphi, psi, prec=hmc.PREC_MIXED).cpu().numpy()
        assert rel(got, want) < 2e-6, dag
        assert np.abs(got - want).max() < 2e-6 * np.abs(want).max(), dag
        again = f(tphi, psi, prec=hmc.PREC_MIXED).cpu().numpy()
        assert np.array_equal(got, again)


# Clusters whose CTAs hold different numbers of K chunks (e.g. V = 288 split
# over 4 CTAs: 4, 5, 4 and 5 steps of 16 sites, 1 or 2 chunks of 64): the
# members read each other's staged partials, so their shared-memory layout
# must agree.  The FP32 iteration must converge on its own (no FP64
# fallback) in about as many iterations as the FP64 CG.
@pytest.mark.parametrize("L,Nt,C,ns", [(12, 16, 4, 0), (12, 32, 4, 0), (12, 64, 4, 0),
                                       (12, 48, 4, 0), (9, 16, 4, 0), (12, 64, 6, 0)])
def test_splitk_cg_converges_in_fp32(L, Nt, C, ns):
    V = 2 * L * L
    beta = Nt / 8
    phi = synth.gaussian_field(L * 7 + Nt, Nt, V, beta / Nt * 3.9, scale=0.3)
    chi = synth.complex_gaussian(L * 7 + Nt + 1, Nt, V)
    tphi, tchi = torch.from_numpy(phi).to(DEV), torch.from_numpy(chi).to(DEV)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=3.9, precision=hmc.PREC_MIXED,
                                 operand_mode=5, inner_ctas=C, tile_slices=ns))
    x, st = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == hmc.HMC_OK and st.true_residual <= 1e-10
    assert st.fp64_iterations == 0
    x64, st64 = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_FP64)
    assert st.iterations <= 1.3 * st64.iterations + 20
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) < 1e-8
