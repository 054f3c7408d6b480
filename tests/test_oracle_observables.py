"""Pins of the zero-momentum single-particle correlator (oracle/observables.py)."""
import numpy as np
import pytest

from oracle import lattice, observables as obs, operators as ops


@pytest.mark.parametrize("L,Nt,beta,kappa,mu", [(1, 4, 1.0, 1.0, 0.0), (2, 6, 2.0, 1.0, 0.0),
                                                (3, 8, 2.0, 1.0, 0.4), (4, 5, 3.0, -0.7, -0.3)])
def test_free_correlator_closed_form(L, Nt, beta, kappa, mu):
    """phi = 0: M^{-1}'s (t, 0) block is E^t (1 + E^Nt)^{-1}; the k = 0 states
    of the two sublattices mix through h with energies +-3 kappa (each site
    has three neighbours), so C(t) = 1/2 sum_{e = +-3 kappa}
    e^{t delta (e - mu)} / (1 + e^{beta (e - mu)}): Fermi factors of the
    particles (energies -e + mu)."""
    delta = beta / Nt
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta * kappa, delta * mu)
    got = obs.correlator_k0(E, np.zeros((Nt, V)))
    t = np.arange(Nt)
    want = 0.5 * sum(np.exp(t * delta * (e - mu)) / (1.0 + np.exp(beta * (e - mu)))
                     for e in (3.0 * kappa, -3.0 * kappa))
    assert np.allclose(got, want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("L,Nt", [(1, 4), (2, 3)])
def test_correlator_kappa_zero_closed_form(L, Nt):
    """kappa = 0: the sites decouple; with Phi_t(x) = sum_{t' < t} phi_t'(x),
    C(t) = V_A^{-1} sum_{x in A} e^{i Phi_t(x)} / (1 + e^{i Phi_Nt(x)})."""
    rng = np.random.default_rng(21)
    V = 2 * L * L
    VA = V // 2
    phi = rng.normal(0.0, 1.0, size=(Nt, V))
    got = obs.correlator_k0(np.eye(V), phi)
    Phi = np.vstack([np.zeros((1, V)), np.cumsum(phi, axis=0)])
    want = np.array([np.mean(np.exp(1j * Phi[t, :VA]) / (1.0 + np.exp(1j * Phi[Nt, :VA])))
                     for t in range(Nt)])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-14)
