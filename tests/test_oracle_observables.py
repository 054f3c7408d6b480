"""Pins of oracle/observables.py: the zero-momentum single-particle
correlator, the staggered spin traces and the staggered susceptibility."""
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


# ---------------------------------------------------------------- spin traces
def random_field(L, Nt, seed=4, s=0.6):
    return np.random.default_rng(seed).normal(0.0, s, size=(Nt, 2 * L * L))


def bloch_energies(L):
    """Tight-binding spectrum +-|1 + e^{i theta_1} + e^{i theta_2}| (§1)."""
    m = np.arange(L)
    th1, th2 = np.meshgrid(2 * np.pi * m / L, 2 * np.pi * m / L, indexing="ij")
    f = np.abs(1.0 + np.exp(1j * th1) + np.exp(1j * th2)).ravel()
    return np.concatenate([f, -f])


@pytest.mark.parametrize("L,Nt", [(1, 4), (2, 5)])
def test_spin_traces_kappa_zero_closed_form(L, Nt):
    """kappa = 0: the sites decouple; with Z_x = e^{i Phi_x} each diagonal
    entry of M^{-1} is 1 / (1 + Z_x), and the single-site loop
    sum_{t t'} G_tt' G_t't is (Nt - Nt (Nt - 1) Z_x) / (1 + Z_x)^2
    (off-diagonal pairs wrap the antiperiodic slice once)."""
    V = 2 * L * L
    phi = random_field(L, Nt)
    Ts, Tu, Tss = obs.spin_traces_exact(np.eye(V), phi)
    Z = np.exp(1j * phi.sum(axis=0))
    eps = obs.sublattice_signs(V)
    assert np.isclose(Ts, np.sum(eps * Nt / (1 + Z)), rtol=1e-12)
    assert np.isclose(Tu, np.sum(Nt / (1 + Z)), rtol=1e-12)
    assert np.isclose(Tss, np.sum((Nt - Nt * (Nt - 1) * Z) / (1 + Z) ** 2), rtol=1e-12)


@pytest.mark.parametrize("L,Nt,beta,kappa", [(2, 6, 2.0, 1.0), (3, 4, 1.5, 1.0), (3, 7, 3.0, -0.8)])
def test_free_spin_traces_closed_form(L, Nt, beta, kappa):
    """phi = 0: M is diagonal in antiperiodic frequencies w_n = (2n+1) pi / Nt
    and in the eigenbasis of h, with symbol 1 - e^{-i w} e^{delta kappa lam};
    on the bipartite lattice eps h eps = -h, so eps G eps has the symbol at
    -lam and T_ss = sum_{w, lam} g_lam(w) g_{-lam}(w), T_u = sum g_lam(w),
    lam over the Bloch spectrum."""
    delta = beta / Nt
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta * kappa)
    _, Tu, Tss = obs.spin_traces_exact(E, np.zeros((Nt, V)))
    w = (2 * np.arange(Nt) + 1) * np.pi / Nt
    lam = bloch_energies(L)

    def g(sign):
        return 1.0 / (1.0 - np.exp(-1j * w)[:, None] * np.exp(sign * delta * kappa * lam)[None, :])
    assert np.isclose(Tu, g(1).sum(), rtol=1e-12)
    assert np.isclose(Tss, (g(1) * g(-1)).sum(), rtol=1e-12)
    # a loop without the second sublattice sign is a different number
    assert not np.isclose(Tss, (g(1) ** 2).sum(), rtol=1e-6)


def test_planted_periodic_sign_breaks_spin_traces(monkeypatch):
    monkeypatch.setattr(ops, "time_signs", lambda Nt: np.ones(Nt))
    V, Nt = 2, 4
    phi = random_field(1, Nt)
    _, Tu, _ = obs.spin_traces_exact(np.eye(V), phi)
    Z = np.exp(1j * phi.sum(axis=0))
    assert not np.isclose(Tu, np.sum(Nt / (1 + Z)), rtol=1e-6)


@pytest.mark.parametrize("L,Nt,beta", [(2, 6, 2.0), (3, 4, 1.0)])
def test_particle_hole_symmetry_of_the_traces(L, Nt, beta):
    """mu = 0: Re T_s = 0 and Re T_u = N/2 for every field (the staggered
    density vanishes, the filling is one half), and M[-phi] = conj(M[phi])
    conjugates every trace; at phi = 0, T_u = N/2 exactly."""
    V, N = 2 * L * L, 2 * L * L * Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt)
    phi = random_field(L, Nt)
    Ts, Tu, Tss = obs.spin_traces_exact(E, phi)
    assert abs(Ts.real) < 1e-10 and abs(Tu.real - N / 2) < 1e-10
    m = obs.spin_traces_exact(E, -phi)
    assert np.allclose(m, np.conj([Ts, Tu, Tss]), rtol=1e-10, atol=1e-10)
    assert np.isclose(obs.spin_traces_exact(E, np.zeros((Nt, V)))[1], N / 2, rtol=1e-12)


@pytest.mark.parametrize("L,Nt,beta,kappa", [(2, 6, 2.0, 1.0), (3, 4, 1.0, -0.6)])
def test_particle_hole_identity_of_the_propagator(L, Nt, beta, kappa):
    """mu = 0: eps h eps = -h makes eps E eps = E^{-1}; with the antiperiodic
    sign this gives eps G eps = 1 - G^dag for every field, hence per real noise
    vector Re(eta^T eps G eta) = sum(eps)/2 = 0 and T_u - T_ss = |G eta|^2
    (chi_s = |G|_F^2 / (2N)).  With mu != 0 the identity fails."""
    V, N = 2 * L * L, 2 * L * L * Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa)
    phi = random_field(L, Nt, seed=L + Nt)
    G = np.linalg.inv(ops.dense_M(E, phi))
    eps = np.tile(obs.sublattice_signs(V), Nt)
    assert np.allclose(eps[:, None] * G * eps[None, :], np.eye(N) - G.conj().T, atol=1e-12)
    s = obs.spin_trace_samples(E, phi, 3, 8)
    for k in range(3):
        v = G @ obs.z2_noise(8, k, 0, Nt, V).ravel()
        assert abs(s[k, 0].real) < 1e-10
        assert np.isclose(s[k, 1] - s[k, 2], np.vdot(v, v), rtol=1e-12)
    _, Tu, Tss = obs.spin_traces_exact(E, phi)
    assert np.isclose(obs.staggered_susceptibility(Tu, Tss, N),
                      np.linalg.norm(G) ** 2 / (2 * N), rtol=1e-12)
    Emu = ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa, beta / Nt * 0.4)
    Gmu = np.linalg.inv(ops.dense_M(Emu, phi))
    assert not np.allclose(eps[:, None] * Gmu * eps[None, :], np.eye(N) - Gmu.conj().T,
                           atol=1e-6)


def test_traces_at_kappa_zero_depend_on_the_time_sum_only():
    """kappa = 0: a site's traces depend on its field only through
    Phi_x = sum_t phi_{x,t} (a diagonal unitary change of basis moves the
    phases between slices and commutes with eps)."""
    Nt, V = 3, 2
    phi = random_field(1, Nt, seed=11)
    flat = np.tile(phi.sum(axis=0) / Nt, (Nt, 1))
    assert np.allclose(obs.spin_traces_exact(np.eye(V), phi),
                       obs.spin_traces_exact(np.eye(V), flat), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("Nt,beta,U", [(2, 1.0, 2.0), (3, 2.0, 3.0), (4, 1.5, 4.0)])
def test_atomic_limit_staggered_susceptibility(Nt, beta, U):
    """kappa = 0, mu = 0: each site of the section 1 Hamiltonian (U/2) rho^2 has
    the empty and doubly occupied states (spin 0, weight e^{-beta U/2}) and the
    two singly occupied ones (spin +-1/2, weight 1), and S^3 commutes with H,
    so the space-time staggered susceptibility is Nt <S^2> =
    Nt / (2 (2 + 2 e^{-beta U / 2})).  The ensemble average of
    chi_s = (Re T_u - Re T_ss) / (2N) under |det M|^2 e^{-S_B}, with
    Phi_x ~ N(0, beta U) the only field variable (previous test), by
    Gauss-Hermite quadrature over the two sites' Phi, equals it."""
    V, N = 2, 2 * Nt
    x, wq = np.polynomial.hermite_e.hermegauss(70)
    Phi = np.sqrt(beta * U) * x
    num = den = loop_only = flipped = 0.0
    for i in range(len(x)):
        for j in range(len(x)):
            phi = np.tile(np.array([Phi[i], Phi[j]]) / Nt, (Nt, 1))
            w = wq[i] * wq[j] * abs(np.linalg.det(ops.dense_M(np.eye(V), phi))) ** 2
            _, Tu, Tss = obs.spin_traces_exact(np.eye(V), phi)
            num += w * obs.staggered_susceptibility(Tu, Tss, N)
            loop_only += w * (-Tss.real) / (2.0 * N)
            flipped += w * (Tu.real + Tss.real) / (2.0 * N)
            den += w
    want = Nt / (2.0 * (2.0 + 2.0 * np.exp(-beta * U / 2.0)))
    assert np.isclose(num / den, want, rtol=1e-10)
    # the loop without the contact term, or with the wrong sign, is not it
    assert not np.isclose(loop_only / den, want, rtol=1e-3)
    assert not np.isclose(flipped / den, want, rtol=1e-3)


def test_noise_estimates_are_exact_on_a_full_basis_and_unbiased():
    """With the unit vectors of the space-time basis in place of noise the
    estimator sums the diagonal exactly; with Z2 noise the estimates of the
    three traces fall within 5 standard errors of the exact values."""
    L, Nt, beta = 2, 4, 1.5
    V, N = 2 * L * L, 2 * L * L * Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt)
    phi = random_field(L, Nt, seed=9)
    exact = np.array(obs.spin_traces_exact(E, phi))
    G = np.linalg.inv(ops.dense_M(E, phi))
    eps = np.tile(obs.sublattice_signs(V), Nt)
    full = sum(b @ (eps * (G @ (eps * (G @ b)))) for b in np.eye(N))
    assert np.isclose(full, exact[2], rtol=1e-12)
    n = 1500
    vals = obs.spin_trace_samples(E, phi, n, 77, chain=0)
    mean = vals.mean(axis=0)
    assert np.allclose(mean, obs.spin_traces_noise(E, phi, n, 77, chain=0), rtol=1e-12)
    se_re = np.sqrt(vals.real.var(axis=0) / n)
    se_im = np.sqrt(vals.imag.var(axis=0) / n)
    for j in range(3):
        assert abs(mean[j].real - exact[j].real) < 5 * se_re[j] + 1e-12, j
        assert abs(mean[j].imag - exact[j].imag) < 5 * se_im[j] + 1e-12, j


def test_z2_noise_values_and_streams():
    """Entries are exactly +-1 (real), about half of each sign, and the
    samples, chains and seeds give different vectors."""
    a = obs.z2_noise(5, 0, 0, 8, 18)
    assert set(np.unique(a.real)) == {-1.0, 1.0} and not a.imag.any()
    assert abs(a.real.mean()) < 0.2
    for b in (obs.z2_noise(5, 1, 0, 8, 18), obs.z2_noise(5, 0, 1, 8, 18), obs.z2_noise(6, 0, 0, 8, 18)):
        assert (a != b).any()
