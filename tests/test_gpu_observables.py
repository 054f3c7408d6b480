"""Observables from M^{-1} sources against the oracle.  The zero-momentum
single-particle correlator (hmc_correlator_k0) against the oracle's dense
solve and, at phi = 0, the closed form with Fermi factors: FP64 CG to 1e-12
-> C(t) to 1e-10 relative (norm over t); mixed CG to 1e-10 (FP64 true
residual) -> 1e-8.  The staggered spin traces (hmc_spin_traces) per noise
sample against the oracle's dense solves, and at full size against the
particle-hole identities."""
import numpy as np
import pytest
import torch

from oracle import lattice, observables as obs, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("prec,tol,bound", [(hmc.PREC_FP64, 1e-12, 1e-10),
                                            (hmc.PREC_MIXED, 1e-10, 1e-8)])
@pytest.mark.parametrize("L,Nt,mu", [(2, 6, 0.0), (3, 8, 0.0), (6, 16, 0.5)])
def test_correlator_matches_oracle(L, Nt, mu, prec, tol, bound):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, mu=mu))
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta, delta * mu)
    phi = synth.gaussian_field(L * 13 + Nt, Nt, V, delta * U, scale=0.5)
    C, st = c.correlator_k0(torch.from_numpy(phi).to(DEV), tol=tol, prec=prec)
    assert st.status == 0
    want = obs.correlator_k0(E, phi)
    got = C.cpu().numpy()
    assert np.linalg.norm(got - want) <= bound * np.linalg.norm(want)


def test_free_correlator_closed_form():
    L, Nt, beta = 6, 32, 4.0
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=3.0))
    C, st = c.correlator_k0(torch.zeros((Nt, 2 * L * L), dtype=torch.float64, device=DEV),
                            tol=1e-12)
    t = np.arange(Nt)
    want = 0.5 * sum(np.exp(t * delta * e) / (1.0 + np.exp(beta * e)) for e in (3.0, -3.0))
    assert st.status == 0
    assert np.allclose(C.cpu().numpy(), want, rtol=1e-10, atol=1e-13)


# ------------------------------------------------------- staggered spin traces
# Per-sample Z2-noise estimates (hmc_spin_traces) against the oracle's dense
# solves on the same Philox noise: FP64 CG to 1e-13 -> 1e-10 relative,
# mixed CG to 1e-10 (FP64 true residual) -> 1e-8 (norm over the samples).
@pytest.mark.parametrize("prec,tol,bound", [(hmc.PREC_FP64, 1e-13, 1e-10),
                                            (hmc.PREC_MIXED, 1e-10, 1e-8)])
@pytest.mark.parametrize("L,Nt,chain", [(1, 4, 0), (2, 6, 3), (3, 8, 1), (6, 16, 7)])
def test_spin_traces_match_oracle(L, Nt, chain, prec, tol, bound):
    beta, U, n_noise, seed = 0.125 * Nt, 3.0, 3, 2210068777
    V, N = 2 * L * L, 2 * L * L * Nt
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U))
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    phi = synth.gaussian_field(L * 17 + Nt, Nt, V, delta * U, scale=0.5)
    samples, mean, st = c.spin_traces(torch.from_numpy(phi).to(DEV), n_noise, seed, chain,
                                      tol=tol, prec=prec)
    # the FP64 solver stops on its recursive residual, the true one may sit a
    # little above tol; the mixed solver stops on the FP64 true residual
    assert st.status == 0 and st.true_residual <= (100 * tol if prec == hmc.PREC_FP64 else tol)
    want = obs.spin_trace_samples(E, phi, n_noise, seed, chain)
    got = samples.cpu().numpy()
    assert np.linalg.norm(got - want) <= bound * np.linalg.norm(want)
    m = mean.cpu().numpy()
    assert np.allclose(m[:3], want.mean(axis=0), rtol=bound, atol=bound * np.abs(want).max())
    chi = obs.staggered_susceptibility(want[:, 1].mean(), want[:, 2].mean(), N)
    assert abs(m[3].real - chi) <= bound * abs(chi) and m[3].imag == 0.0


def test_spin_traces_repeatable_and_refusals():
    L, Nt = 3, 8
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=1.0, U=3.0))
    phi = torch.from_numpy(synth.gaussian_field(5, Nt, 2 * L * L, 0.375, scale=0.5)).to(DEV)
    a = c.spin_traces(phi, 2, 11, 0, tol=1e-12)
    b = c.spin_traces(phi, 2, 11, 0, tol=1e-12)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert not torch.equal(a[0], c.spin_traces(phi, 2, 12, 0, tol=1e-12)[0])
    with pytest.raises(hmc.HmcError) as e:
        c.spin_traces(phi, 0, 11)
    assert e.value.code == hmc.HMC_ERR_BAD_ARG
    cmu = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=1.0, U=3.0, mu=0.3))
    with pytest.raises(hmc.HmcError) as e:
        cmu.spin_traces(phi, 1, 11)
    assert e.value.code == hmc.HMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [hmc.PREC_MIXED])
def test_spin_traces_full_size_particle_hole_identities(prec):
    """L=24, Nt=96 (N = 110592): per sample, Re(eta^T eps G eta) = sum(eps)/2 = 0
    and T_u - T_ss = |M^{-1} eta|^2 = eta^dag (M M^dag)^{-1} eta, real (the
    identity eps G eps = 1 - G^dag at mu = 0); the right side comes from a
    separate hmc_cg_solve of the same noise (drawn with hmc_rng_draw)."""
    L, Nt, beta, U = 24, 96, 12.0, 4.0
    V, N = 2 * L * L, 2 * L * L * Nt
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U))
    phi = torch.from_numpy(synth.gaussian_field(24, Nt, V, delta * U, scale=0.3)).to(DEV)
    samples, mean, st = c.spin_traces(phi, 2, 99, 0, tol=1e-10, prec=prec)
    assert st.status == 0 and st.true_residual <= 1e-10
    s = samples.cpu().numpy()
    for k in range(2):
        raw, _, _ = hmc.rng_draw(99, 4, k, 0, N)
        eta = (1 - 2 * (raw[:, 0] & 1)).to(torch.complex128).view(Nt, V)
        x, cst = c.cg_solve(phi, eta, tol=1e-10, prec=hmc.PREC_MIXED)
        assert cst.status == 0
        norm2 = torch.vdot(eta.flatten(), x.flatten()).item()
        d = s[k, 1] - s[k, 2]
        assert abs(s[k, 0].real) <= 1e-8 * abs(s[k, 1])
        assert abs(d.imag) <= 1e-8 * abs(d.real)
        assert abs(d.real - norm2.real) <= 1e-8 * norm2.real
    assert abs(mean.cpu().numpy()[3].real - (s[:, 1] - s[:, 2]).real.mean() / (2 * N)) <= \
        1e-12 * abs(mean.cpu().numpy()[3].real)
