"""The adjoint force behind torch.autograd against the oracle gradient and
central finite differences (the L=6, Nt=32, U=3.5, beta=4 workload,
16 random fields)."""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth
from paper_2210_06874_gb300.autograd import pseudofermion_action

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
L, NT, U, BETA = 6, 32, 3.5, 4.0
V = 2 * L * L
DELTA = BETA / NT


@pytest.fixture(scope="module")
def setup():
    c = hmc.Context(hmc.Params(L=L, Nt=NT, U=U, beta=BETA, cg_tol=1e-12))
    E = ops.transfer_matrix(lattice.hopping_matrix(L), DELTA)
    return c, E


@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_MIXED])
def test_autograd_matches_oracle_gradient_16_fields(setup, prec):
    c, E = setup
    worst = 0.0
    for k in range(16):
        phi_np = synth.gaussian_field(1000 + k, NT, V, DELTA * U, scale=0.5)
        chi_np = synth.complex_gaussian(2000 + k, NT, V)
        phi = torch.from_numpy(phi_np).to(DEV).requires_grad_(True)
        chi = torch.from_numpy(chi_np).to(DEV)
        S = pseudofermion_action(phi, chi, c, prec=prec, tol=1e-12 if prec == hmc.PREC_FP64
                                 else 1e-10)
        S.backward()
        xo, _, _ = ohmc.cg_solve(E, phi_np, chi_np, tol=1e-14, max_iter=100000)
        Fo = ohmc.force_from_solution(E, phi_np, xo, DELTA, U)
        So = ohmc.bosonic_action(phi_np, DELTA, U) + np.vdot(chi_np, xo).real
        g = phi.grad.cpu().numpy()
        worst = max(worst, np.linalg.norm(g - Fo) / np.linalg.norm(Fo))
        assert abs(S.item() - So) < 1e-9 * abs(So)
    assert worst < 1e-8, worst


def test_autograd_matches_finite_differences(setup):
    c, E = setup
    phi_np = synth.gaussian_field(77, NT, V, DELTA * U, scale=0.5)
    chi = torch.from_numpy(synth.complex_gaussian(78, NT, V)).to(DEV)
    phi = torch.from_numpy(phi_np).to(DEV).requires_grad_(True)
    S = pseudofermion_action(phi, chi, c, tol=1e-13)
    S.backward()
    g = phi.grad.cpu().numpy()
    h = 1e-5
    for (t, x) in [(0, 0), (5, 17), (NT - 1, V - 1), (16, 40)]:
        p1, p2 = phi_np.copy(), phi_np.copy()
        p1[t, x] += h
        p2[t, x] -= h
        s1 = pseudofermion_action(torch.from_numpy(p1).to(DEV), chi, c, tol=1e-13).item()
        s2 = pseudofermion_action(torch.from_numpy(p2).to(DEV), chi, c, tol=1e-13).item()
        fd = (s1 - s2) / (2 * h)
        assert abs(fd - g[t, x]) < 1e-5 * max(1.0, abs(g[t, x])), (t, x, fd, g[t, x])


def test_backward_does_not_resolve(setup):
    c, _ = setup
    phi = torch.from_numpy(synth.gaussian_field(5, NT, V, DELTA * U, scale=0.5)).to(DEV)
    phi.requires_grad_(True)
    chi = torch.from_numpy(synth.complex_gaussian(6, NT, V)).to(DEV)
    S = pseudofermion_action(phi, chi, c)
    calls = []
    orig = c.cg_solve
    c.cg_solve = lambda *a, **k: calls.append(1) or orig(*a, **k)
    try:
        S.backward()
    finally:
        c.cg_solve = orig
    assert calls == []
    assert torch.isfinite(phi.grad).all()
