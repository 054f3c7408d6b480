"""GPU parity of the mixed-precision path (FP16-split tensor-core contraction,
FP32 CG with FP64 reliable updates) against the FP64 oracle.

Tolerances, derived from the arithmetic: the split keeps 22 bits of E and of
the (power-of-two scaled) vector, products are exact in FP32 and summed in
FP32, so one application is accurate to a few 1e-7 relative (normwise); the
solver must reach the FP64 true residual 1e-10 and the force built on its
solution 1e-8 relative.
"""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
APPLY_TOL = 2e-6


def oracle_E(L, Nt, beta, kappa=1.0):
    return ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def elementwise_ok(got, want, tol):
    """Every element within tol of the oracle, relative to its own magnitude
    plus the vector's RMS (small entries come from sums that cancel; their
    absolute error is that of the whole sum)."""
    rms = np.sqrt(np.mean(np.abs(want) ** 2))
    return bool(np.all(np.abs(got - want) <= tol * (np.abs(want) + rms)))


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype else t).to(DEV)


SIZES = [(1, 1), (1, 3), (2, 5), (3, 8), (5, 13), (6, 32), (7, 9), (9, 48), (12, 64), (24, 96)]


@pytest.mark.parametrize("L,Nt", SIZES)
def test_apply_mixed(L, Nt):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(L * 100 + Nt, Nt, V, beta / Nt * U)
    psi64 = synth.complex_gaussian(L * 1000 + Nt, Nt, V)
    psi = dev(psi64, torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)        # what the kernel sees
    got = c.apply_M(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    want = ops.apply_M(E, phi, psi_in)
    assert rel(got, want) < APPLY_TOL and elementwise_ok(got, want, APPLY_TOL)
    got = c.apply_Mdag(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    want = ops.apply_Mdag(E, phi, psi_in)
    assert rel(got, want) < APPLY_TOL and elementwise_ok(got, want, APPLY_TOL)


def test_apply_mixed_scale_invariance():
    """The power-of-two vector scaling keeps tiny and huge inputs accurate."""
    L, Nt = 3, 8
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=1.0, U=3.0))
    E = oracle_E(L, Nt, 1.0)
    phi = synth.gaussian_field(1, Nt, 18, 0.3)
    for s in (1e-30, 1e-6, 1.0, 1e6, 1e30):
        psi = dev(synth.complex_gaussian(2, Nt, 18) * s, torch.complex64)
        got = c.apply_M(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
        want = ops.apply_M(E, phi, psi.cpu().numpy().astype(np.complex128))
        assert rel(got, want) < APPLY_TOL, s


def test_apply_mixed_zero_vector():
    c = hmc.Context(hmc.Params(L=2, Nt=4, beta=0.5, U=3.0))
    psi = torch.zeros((4, 8), dtype=torch.complex64, device=DEV)
    phi = torch.zeros((4, 8), dtype=torch.float64, device=DEV)
    assert torch.count_nonzero(c.apply_M(phi, psi, prec=hmc.PREC_MIXED)) == 0


@pytest.mark.parametrize("mode", [1, 2])       # streamed E / resident E
@pytest.mark.parametrize("L,Nt,beta,U", [(1, 2, 1.0, 2.0), (3, 8, 2.0, 2.0), (6, 32, 4.0, 3.5),
                                         (9, 16, 2.0, 3.0), (12, 64, 8.0, 3.8)])
def test_cg_mixed_reaches_fp64_residual(L, Nt, beta, U, mode):
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, operand_mode=mode))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(11, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(12, Nt, V)
    x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == 0
    assert st.true_residual <= 1e-10
    assert st.reliable_updates >= 1
    # independent FP64 check of the residual with the oracle operator
    xn = x.cpu().numpy()
    res = chi - ops.apply_MMdag(E, phi, xn)
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10
    x64, st64 = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_FP64)
    # same residual target: iteration counts of the two solvers are comparable
    assert st.iterations < 3 * st64.iterations + 20


@pytest.mark.parametrize("L,Nt", [(3, 8), (6, 32)])
def test_force_from_mixed_solution(L, Nt):
    """Force relative error 1e-8 against the oracle's analytic gradient."""
    beta, U = 0.125 * Nt, 3.5
    V = 2 * L * L
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(31, Nt, V, delta * U, scale=0.5)
    chi = synth.complex_gaussian(32, Nt, V)
    x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    F = c.force(dev(phi), x).cpu().numpy()
    xo, _, _ = ohmc.cg_solve(E, phi, chi, tol=1e-14, max_iter=100000)
    Fo = ohmc.force_from_solution(E, phi, xo, delta, U)
    assert rel(F, Fo) < 1e-8


@pytest.mark.parametrize("mode", [1, 2])
def test_trajectory_mixed_matches_oracle(mode):
    L, Nt, beta, U, n_md = 3, 8, 2.0, 2.0, 10
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=1.0,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=mode))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(5, Nt, 18, delta * U, scale=0.5)
    phi = dev(phi_np)
    for traj in range(3):
        want = ohmc.trajectory(E, phi_np, delta, U, 1.0 / n_md, n_md, 77, traj, 0, tol=1e-12)
        out = c.trajectory(phi, 77, traj)
        assert out.status == 0
        assert out.max_true_residual <= 1e-10
        assert out.reliable_updates >= out.cg_solves
        assert abs(out.dH - want["dH"]) < 1e-7
        assert bool(out.accept) == want["accept"]
        assert rel(phi.cpu().numpy(), want["phi"]) < 1e-8
        phi_np = want["phi"]


def test_trajectory_mixed_deterministic():
    c = hmc.Context(hmc.Params(L=6, Nt=32, U=3.5, beta=4.0, n_md=4, traj_length=0.5,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED))
    a = torch.zeros((32, 72), dtype=torch.float64, device=DEV)
    b = a.clone()
    o1 = [c.trajectory(a, 3, t).dH for t in range(2)]
    o2 = [c.trajectory(b, 3, t).dH for t in range(2)]
    assert o1 == o2 and torch.equal(a, b)


@pytest.mark.parametrize("L,Nt,ns", [(5, 13, 16), (6, 40, 32), (3, 20, 32), (9, 21, 16)])
def test_apply_mixed_ragged_last_tile(L, Nt, ns):
    """Standalone applications with 16 or 32 slices per tile and a ragged
    last tile (fewer slices, same TMA box for the pre-split operand)."""
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, tile_slices=ns))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(L * 7 + Nt, Nt, V, beta / Nt * U)
    psi = dev(synth.complex_gaussian(L * 11 + Nt, Nt, V), torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)
    for dag, op in ((False, ops.apply_M), (True, ops.apply_Mdag)):
        fn = c.apply_Mdag if dag else c.apply_M
        got = fn(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
        assert rel(got, op(E, phi, psi_in)) < APPLY_TOL
