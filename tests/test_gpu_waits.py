"""Bounded device waits and the mixed solver's safeguards, on the GPU.

* Timeout path: with the context's wait limit at 5 ms and every team barrier
  expecting one CTA more than the launch has (host-side injection), the
  first barrier never completes; the kernel must give up, report
  HMC_ERR_TIMEOUT and leave the context usable for a following good solve.
* Reliable-update trigger by iteration count: with a residual-drop threshold
  that never fires, the FP32 iteration still reaches FP64 residual checks
  every ru_every iterations and the solve converges.
* FP64 fallback: a reliable update after every FP32 iteration cannot halve
  the true residual each time, so two updates in a row count as a stall and
  the rest of the solve runs as FP64 CG; it must converge to the FP64 path's
  solution.
"""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(L, Nt, beta, U, seed):
    V = 2 * L * L
    phi = synth.gaussian_field(seed, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(seed + 1, Nt, V)
    E = ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt)
    return E, phi, chi


# (precision, operand_mode): the FP64 kernel, the CUDA-core cluster mode (the
# automatic choice at this size), site-major and slice-major tensor-core tiles
CASES = [(hmc.PREC_FP64, 0), (hmc.PREC_MIXED, 0), (hmc.PREC_MIXED, 1), (hmc.PREC_MIXED, 4)]


@pytest.mark.parametrize("prec,mode", CASES)
def test_timeout_then_good_solve(prec, mode):
    L, Nt, beta, U = 3, 8, 2.0, 2.0
    E, phi, chi = problem(L, Nt, beta, U, 301)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, precision=prec,
                                 operand_mode=mode, cg_tol=1e-10))
    tphi, tchi = torch.from_numpy(phi).to(DEV), torch.from_numpy(chi).to(DEV)
    ctx.set_wait_limit(0.005)
    ctx.debug_team_padding(1)
    for _ in range(2):                       # the failure repeats, the context survives
        with pytest.raises(hmc.HmcError) as e:
            ctx.cg_solve(tphi, tchi, tol=1e-10, prec=prec)
        assert e.value.code == hmc.HMC_ERR_TIMEOUT
    with pytest.raises(hmc.HmcError) as e:
        ctx.trajectory(tphi.clone(), 5, 0)
    assert e.value.code == hmc.HMC_ERR_TIMEOUT
    ctx.debug_team_padding(0)
    ctx.set_wait_limit(0)
    x, st = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=prec)
    assert st.status == hmc.HMC_OK and st.true_residual <= 1e-10
    xo, _, _ = ohmc.cg_solve(E, phi, chi, tol=1e-14)
    assert rel(x.cpu().numpy(), xo) < 1e-8


def test_bad_wait_arguments():
    ctx = hmc.Context(hmc.Params(L=2, Nt=4))
    for bad in (-1.0, float("nan"), 1e6):
        with pytest.raises(hmc.HmcError) as e:
            ctx.set_wait_limit(bad)
        assert e.value.code == hmc.HMC_ERR_BAD_ARG
    with pytest.raises(hmc.HmcError):
        ctx.debug_team_padding(-1)


@pytest.mark.parametrize("mode", [0, 1, 4])
def test_reliable_update_by_iteration_count(mode):
    L, Nt, beta, U = 6, 32, 4.0, 3.5
    E, phi, chi = problem(L, Nt, beta, U, 311)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, precision=hmc.PREC_MIXED,
                                 operand_mode=mode, ru_delta=1e-30, ru_every=40))
    x, st = ctx.cg_solve(torch.from_numpy(phi).to(DEV), torch.from_numpy(chi).to(DEV),
                         tol=1e-10, prec=hmc.PREC_MIXED)
    print("iterations", st.iterations, "reliable updates", st.reliable_updates,
          "fp64 iterations", st.fp64_iterations)
    assert st.status == hmc.HMC_OK and st.true_residual <= 1e-10
    # ru_delta never fires: updates come from the count (and the last check)
    assert st.reliable_updates >= st.iterations // 40
    xo, _, _ = ohmc.cg_solve(E, phi, chi, tol=1e-14)
    assert rel(x.cpu().numpy(), xo) < 1e-8


@pytest.mark.parametrize("mode", [0, 1, 4])
def test_stall_switches_to_fp64(mode):
    L, Nt, beta, U = 6, 4, 1.0, 3.78          # delta = 0.25
    E, phi, chi = problem(L, Nt, beta, U, 321)
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, precision=hmc.PREC_MIXED,
                                 operand_mode=mode, ru_every=1))
    tphi, tchi = torch.from_numpy(phi).to(DEV), torch.from_numpy(chi).to(DEV)
    x, st = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_MIXED)
    print("iterations", st.iterations, "reliable updates", st.reliable_updates,
          "fp64 iterations", st.fp64_iterations)
    assert st.fp64_iterations > 0
    assert st.status == hmc.HMC_OK and st.true_residual <= 1e-10
    x64, _ = ctx.cg_solve(tphi, tchi, tol=1e-10, prec=hmc.PREC_FP64)
    assert rel(x.cpu().numpy(), x64.cpu().numpy()) < 1e-8
    # a trajectory whose solves all stall and fall back still matches the oracle
    ctx2 = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, precision=hmc.PREC_MIXED,
                                  operand_mode=mode, ru_every=1, n_md=2, traj_length=0.5,
                                  cg_tol=1e-10))
    out = ctx2.trajectory(tphi.clone(), 17, 0)
    assert out.status == hmc.HMC_OK and out.fp64_iterations > 0
    want = ohmc.trajectory(E, phi, beta / Nt, U, 0.25, 2, 17, 0, tol=1e-12)
    assert abs(out.dH - want["dH"]) < 1e-7
