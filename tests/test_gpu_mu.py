"""Chemical potential mu (the sign-problem setting of the paper's
tensor-network section, p ~ det(M[phi,mu] M[phi,-mu]^dag)): the context's
operator is the particles' one, E = exp(delta (kappa h - mu)).
Parity against the FP64 oracle at the tolerances of the mu = 0 tests: FP64
operator 1e-13, mixed operator 2e-6 (both tensor-core tile kinds), CG true
residual 1e-10, mixed trajectory Delta H 1e-7."""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def oracle_E(L, Nt, beta, mu, kappa=1.0):
    delta = beta / Nt
    return ops.transfer_matrix(lattice.hopping_matrix(L), delta * kappa, delta * mu)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype else t).to(DEV)


@pytest.mark.parametrize("L,Nt,mu", [(3, 8, 0.5), (6, 32, -0.8), (9, 16, 1.3)])
def test_transfer_matrix_and_fp64_apply_with_mu(L, Nt, mu):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, mu=mu))
    E = oracle_E(L, Nt, beta, mu)
    assert np.abs(c.transfer_matrix().numpy() - E).max() <= 1e-13 * np.abs(E).max()
    phi = synth.gaussian_field(L + Nt, Nt, V, beta / Nt * U)
    psi = synth.complex_gaussian(L * 3 + Nt, Nt, V)
    got = c.apply_M(dev(phi), dev(psi)).cpu().numpy()
    assert rel(got, ops.apply_M(E, phi, psi)) < 1e-13
    got = c.apply_Mdag(dev(phi), dev(psi)).cpu().numpy()
    assert rel(got, ops.apply_Mdag(E, phi, psi)) < 1e-13


@pytest.mark.parametrize("mode", [1, 4])
@pytest.mark.parametrize("L,Nt,mu", [(6, 32, 0.9), (12, 64, -0.6)])
def test_mixed_apply_and_cg_with_mu(L, Nt, mu, mode):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, mu=mu, operand_mode=mode))
    E = oracle_E(L, Nt, beta, mu)
    phi = synth.gaussian_field(L * 5 + Nt, Nt, V, beta / Nt * U, scale=0.5)
    psi = dev(synth.complex_gaussian(L * 7 + Nt, Nt, V), torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)
    got = c.apply_M(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    assert rel(got, ops.apply_M(E, phi, psi_in)) < 2e-6
    got = c.apply_Mdag(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    assert rel(got, ops.apply_Mdag(E, phi, psi_in)) < 2e-6
    chi = synth.complex_gaussian(L * 9 + Nt, Nt, V)
    x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == 0 and st.true_residual <= 1e-10
    res = chi - ops.apply_MMdag(E, phi, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10


def test_mixed_trajectory_with_mu_matches_oracle():
    L, Nt, beta, U, n_md, tau, mu = 6, 32, 4.0, 3.5, 3, 0.3, 0.7
    delta = beta / Nt
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=tau,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=4, mu=mu))
    E = oracle_E(L, Nt, beta, mu)
    phi_np = synth.gaussian_field(12, Nt, V, delta * U, scale=0.5)
    phi = dev(phi_np)
    want = ohmc.trajectory(E, phi_np, delta, U, tau / n_md, n_md, 8, 0, 0, tol=1e-12)
    out = c.trajectory(phi, 8, 0)
    assert out.status == 0
    assert out.max_true_residual <= 1e-10
    assert abs(out.dH - want["dH"]) < 1e-7
    assert bool(out.accept) == want["accept"]
    assert rel(phi.cpu().numpy(), want["phi"]) < 1e-8


def test_batch_chains_differing_only_in_mu():
    """Chains of one lattice and delta*kappa but different mu must not share
    the transfer matrix: each batch chain matches its own single-chain run."""
    chains = [(6, 16, 0.0), (6, 16, 0.6), (6, 16, -0.6)]

    def p(L, Nt, mu, **kw):
        return hmc.Params(L=L, Nt=Nt, U=3.0, beta=0.125 * Nt, n_md=3, traj_length=0.3,
                          cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=4, mu=mu, **kw)
    b = hmc.Batch([p(*c) for c in chains])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = [synth.gaussian_field(70 + i, Nt, 2 * L * L, 0.375, scale=0.5)
              for i, (L, Nt, _) in enumerate(chains)]
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    outs = b.trajectory(phi, 4, 0)
    for i, (L, Nt, mu) in enumerate(chains):
        single = hmc.Context(p(L, Nt, mu, team_ctas=1, inner_ctas=1))
        sphi = torch.from_numpy(fields[i]).to(DEV)
        o = single.trajectory(sphi, 4, 0, chain=i)
        assert outs[i].status == 0 and o.status == 0
        assert outs[i].dH == o.dH, (i, outs[i].dH, o.dH)
        assert torch.equal(b.view(phi, i), sphi)
