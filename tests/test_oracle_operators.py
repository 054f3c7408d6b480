"""Pins of the oracle's lattice and fermion matrices against what the paper and
the mathematics fix (CPU only).

  * tight-binding spectrum of h: +-|1 + e^{i th1} + e^{i th2}| (the U = 0
    analytic solution the paper points to in §1, Fig. 2)
  * E = exp(delta kappa h) against scipy's Pade expm, and E 1 = e^{3 delta kappa} 1
  * free-theory determinant of the exponential form in closed form
  * reduced determinant det M = det(1 + E D_{Nt-1} ... E D_0)
  * kappa = 0: det M = prod_x (1 + exp(i sum_t phi_{x,t}))
  * Eq. (2.2) at phi = 0: |det M| = prod_{k,n} |2 - 2 cos w_n + delta^2 kappa^2 |f_k|^2|
  * dense vs matrix-free, adjoint identity
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import lattice, operators as ops


def bloch_moduli(L):
    th = 2.0 * np.pi * np.arange(L) / L
    return np.abs(1.0 + np.exp(1j * th)[:, None] + np.exp(1j * th)[None, :]).ravel()


@pytest.mark.parametrize("L", [1, 2, 3, 4, 6])
def test_hopping_structure_and_spectrum(L):
    h = lattice.hopping_matrix(L)
    V = 2 * L * L
    assert h.shape == (V, V)
    assert np.array_equal(h, h.T)
    assert np.allclose(h.sum(axis=1), 3.0)                  # three neighbours
    A = L * L
    assert not h[:A, :A].any() and not h[A:, A:].any()      # bipartite
    f = bloch_moduli(L)
    want = np.sort(np.concatenate([f, -f]))
    got = np.linalg.eigvalsh(h)
    assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("L,dk", [(2, 0.25), (3, 0.125), (6, 0.125), (4, 0.5)])
def test_transfer_matrix(L, dk):
    h = lattice.hopping_matrix(L)
    E = ops.transfer_matrix(h, dk)
    assert np.allclose(E, scipy.linalg.expm(dk * h), rtol=0, atol=1e-14)
    assert np.allclose(E.sum(axis=1), np.exp(3.0 * dk), atol=1e-13)
    assert np.allclose(E, E.T, atol=1e-15)


def random_field(rng, Nt, V, scale):
    return rng.normal(0.0, scale, size=(Nt, V))


def random_vec(rng, Nt, V):
    return rng.normal(size=(Nt, V)) + 1j * rng.normal(size=(Nt, V))


@pytest.mark.parametrize("L,Nt", [(1, 1), (1, 3), (2, 2), (2, 5), (3, 8)])
def test_dense_vs_matrix_free(L, Nt):
    rng = np.random.default_rng(10 * L + Nt)
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), 0.3)
    phi = random_field(rng, Nt, V, 0.7)
    psi = random_vec(rng, Nt, V)
    Md = ops.dense_M(E, phi)
    assert np.allclose(Md @ psi.ravel(), ops.apply_M(E, phi, psi).ravel(), atol=1e-13)
    assert np.allclose(Md.conj().T @ psi.ravel(), ops.apply_Mdag(E, phi, psi).ravel(),
                       atol=1e-13)


@pytest.mark.parametrize("L,Nt", [(3, 8), (6, 32)])
def test_adjoint_identity(L, Nt):
    rng = np.random.default_rng(99)
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), 0.125)
    phi = random_field(rng, Nt, V, 0.6)
    u, v = random_vec(rng, Nt, V), random_vec(rng, Nt, V)
    lhs = np.vdot(u, ops.apply_M(E, phi, v))
    rhs = np.vdot(ops.apply_Mdag(E, phi, u), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("L,Nt,beta,kappa", [(1, 4, 1.0, 1.0), (2, 6, 2.0, 1.0),
                                             (3, 8, 2.0, 1.0), (3, 5, 3.0, -0.7)])
def test_free_determinant_closed_form(L, Nt, beta, kappa):
    """phi = 0: det M = prod over eigenvalues lam of h of (1 + e^{beta kappa lam})."""
    delta = beta / Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta * kappa)
    sign, logdet = np.linalg.slogdet(ops.dense_M(E, np.zeros((Nt, 2 * L * L))))
    f = bloch_moduli(L)
    lam = np.concatenate([f, -f])
    want = np.sum(np.log1p(np.exp(beta * kappa * lam)))
    assert abs(logdet - want) < 1e-11
    assert abs(sign - 1.0) < 1e-12


@pytest.mark.parametrize("L,Nt", [(1, 3), (2, 4), (3, 6)])
def test_reduced_determinant(L, Nt):
    rng = np.random.default_rng(5)
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), 0.25)
    phi = random_field(rng, Nt, V, 0.8)
    s1, l1 = np.linalg.slogdet(ops.dense_M(E, phi))
    s2, l2 = np.linalg.slogdet(ops.reduced_matrix(E, phi))
    assert abs(l1 - l2) < 1e-11
    assert abs(s1 - s2) < 1e-11


@pytest.mark.parametrize("L,Nt", [(1, 4), (2, 3)])
def test_kappa_zero_closed_form(L, Nt):
    """kappa = 0 decouples the sites: det M = prod_x (1 + e^{i sum_t phi_{x,t}})."""
    rng = np.random.default_rng(6)
    V = 2 * L * L
    E = np.eye(V)
    phi = random_field(rng, Nt, V, 1.0)
    want = np.prod(1.0 + np.exp(1j * phi.sum(axis=0)))
    got = np.linalg.det(ops.dense_M(E, phi))
    assert abs(got - want) <= 1e-12 * abs(want)


def test_single_slice():
    """Nt = 1: the antiperiodic wrap gives M = 1 + E D_0."""
    rng = np.random.default_rng(8)
    L, V = 2, 8
    E = ops.transfer_matrix(lattice.hopping_matrix(L), 0.4)
    phi = random_field(rng, 1, V, 1.0)
    want = np.eye(V) + E * np.exp(1j * phi[0])[None, :]
    assert np.allclose(ops.dense_M(E, phi), want, atol=1e-15)


@pytest.mark.parametrize("L,Nt,beta", [(1, 4, 1.0), (2, 4, 2.0), (3, 8, 2.0)])
def test_brs_free_closed_form(L, Nt, beta):
    """Eq. (2.2) at phi = 0, Fourier in space and antiperiodic time."""
    kappa = 1.0
    delta = beta / Nt
    V = 2 * L * L
    M = ops.dense_M_brs(L, np.zeros((Nt, V)), delta, kappa)
    _, logdet = np.linalg.slogdet(M)
    f = bloch_moduli(L)
    w = (2 * np.arange(Nt) + 1) * np.pi / Nt
    want = np.sum(np.log(np.abs(2 - 2 * np.cos(w)[:, None]
                                + (delta * kappa * f[None, :]) ** 2)))
    assert abs(logdet - want) < 1e-11


def brs_kappa_zero_det(L, phi):
    """det of Eq. (2.2) at kappa = 0: every site is a cyclic bidiagonal
    Nt x Nt block.  A site: -diag(e^{i phi_t}) plus the forward shift with
    the wrap -1, det = (-1)^Nt (1 + e^{i Phi}); B site: 1 minus the
    backward shift weighted by e^{-i phi_t} with the wrap -1,
    det = 1 + e^{-i Phi}; Phi = sum_t phi_t.  Sites x < L^2 are A."""
    Nt, V = phi.shape
    Phi = phi.sum(axis=0)
    a = (-1.0) ** Nt * (1.0 + np.exp(1j * Phi[:V // 2]))
    b = 1.0 + np.exp(-1j * Phi[V // 2:])
    return np.prod(a) * np.prod(b)


@pytest.mark.parametrize("L,Nt", [(1, 3), (2, 4), (2, 5)])
def test_brs_kappa_zero_closed_form(L, Nt):
    rng = np.random.default_rng(23)
    V = 2 * L * L
    phi = random_field(rng, Nt, V, 1.0)
    got = np.linalg.det(ops.dense_M_brs(L, phi, 0.25, 0.0))
    want = brs_kappa_zero_det(L, phi)
    assert abs(got - want) <= 1e-12 * abs(want)


def test_planted_brs_sublattice_swap_is_caught(monkeypatch):
    """The phases of Eq. (2.2) on the wrong sublattices (A backward with
    e^{-i phi}, B forward with e^{+i phi}) change the complex determinant."""
    L, Nt = 2, 4
    rng = np.random.default_rng(23)
    V = 2 * L * L
    phi = random_field(rng, Nt, V, 1.0)
    real = lattice.sublattice
    monkeypatch.setattr(lattice, "sublattice", lambda L_: 1 - real(L_))
    got = np.linalg.det(ops.dense_M_brs(L, phi, 0.25, 0.0))
    assert abs(got - brs_kappa_zero_det(L, phi)) > 1e-3 * abs(got)


@pytest.mark.parametrize("L,Nt", [(1, 2), (2, 3), (3, 4)])
def test_brs_dense_vs_matrix_free(L, Nt):
    rng = np.random.default_rng(3)
    V = 2 * L * L
    phi = random_field(rng, Nt, V, 0.9)
    psi = random_vec(rng, Nt, V)
    M = ops.dense_M_brs(L, phi, 0.25, 1.0)
    assert np.allclose(M @ psi.ravel(), ops.apply_M_brs(L, phi, psi, 0.25, 1.0).ravel(),
                       atol=1e-13)


@pytest.mark.parametrize("L,Nt", [(1, 2), (2, 3), (3, 4)])
def test_brs_adjoint_dense(L, Nt):
    """The matrix-free adjoint of Eq. (2.2) is the conjugate transpose of the
    dense matrix built from the equation."""
    rng = np.random.default_rng(13)
    V = 2 * L * L
    phi = random_field(rng, Nt, V, 0.9)
    psi = random_vec(rng, Nt, V)
    M = ops.dense_M_brs(L, phi, 0.25, 1.0)
    assert np.allclose(M.conj().T @ psi.ravel(),
                       ops.apply_Mdag_brs(L, phi, psi, 0.25, 1.0).ravel(), atol=1e-13)


def test_brs_adjoint_identity_large():
    rng = np.random.default_rng(14)
    L, Nt = 6, 16
    V = 2 * L * L
    phi = random_field(rng, Nt, V, 0.7)
    u, v = random_vec(rng, Nt, V), random_vec(rng, Nt, V)
    lhs = np.vdot(u, ops.apply_M_brs(L, phi, v, 0.125, 1.0))
    rhs = np.vdot(ops.apply_Mdag_brs(L, phi, u, 0.125, 1.0), v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# chemical potential (sign-problem setting, p ~ det(M[phi,mu] M[phi,-mu]^dag)):
# the §1 Hamiltonian's + mu sum_x rho_x gives the particles' transfer matrix
# E = exp(delta (kappa h - mu))

@pytest.mark.parametrize("L,Nt,beta,kappa,mu", [(1, 4, 1.0, 1.0, 0.3), (2, 6, 2.0, 1.0, -0.5),
                                                (3, 8, 2.0, 1.0, 0.7), (3, 5, 3.0, -0.7, 1.1)])
def test_free_determinant_with_mu_closed_form(L, Nt, beta, kappa, mu):
    """phi = 0: det M[0, mu] = prod over eigenvalues lam of h of
    (1 + e^{beta (kappa lam - mu)}) -- the free partition function of the
    particles, single-particle energies -kappa lam + mu."""
    delta = beta / Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta * kappa, delta * mu)
    sign, logdet = np.linalg.slogdet(ops.dense_M(E, np.zeros((Nt, 2 * L * L))))
    f = bloch_moduli(L)
    lam = np.concatenate([f, -f])
    want = np.sum(np.log1p(np.exp(beta * (kappa * lam - mu))))
    assert abs(logdet - want) < 1e-11
    assert abs(sign - 1.0) < 1e-12


@pytest.mark.parametrize("L,Nt,mu", [(1, 4, 0.4), (2, 3, -0.9)])
def test_kappa_zero_with_mu_closed_form(L, Nt, mu):
    """kappa = 0: det M = prod_x (1 + e^{-beta mu} e^{i sum_t phi_{x,t}}): the
    one-site trace over the particle's occupations n = 0, 1 of
    e^{-beta mu n} e^{i Phi n} (energy + mu per particle, §1)."""
    rng = np.random.default_rng(16)
    V = 2 * L * L
    beta = 1.5
    E = ops.transfer_matrix(lattice.hopping_matrix(L), 0.0, beta / Nt * mu)
    phi = random_field(rng, Nt, V, 1.0)
    want = np.prod(1.0 + np.exp(-beta * mu) * np.exp(1j * phi.sum(axis=0)))
    got = np.linalg.det(ops.dense_M(E, phi))
    assert abs(got - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("L,Nt,beta,kappa,mu", [(2, 4, 1.0, 1.0, 0.8), (3, 6, 2.0, 0.7, -0.4)])
def test_particle_hole_identity_with_mu(L, Nt, beta, kappa, mu):
    """det M[phi,-mu] = e^{i sum phi} e^{beta mu V} conj(det M[phi,mu]).
    With B the product of the Nt slices' E D_t, det M[phi,mu] =
    det(1 + e^{-beta mu} B); pulling B out of det(1 + e^{beta mu} B) leaves
    det B e^{beta mu V} det(1 + e^{-beta mu} B^{-1}), det B = e^{i sum phi}
    (tr h = 0), and B^{-1} is conj(B) transposed and conjugated by the
    sublattice signs (h bipartite: P h P = -h).  Hence
    |p[phi]| = e^{beta mu V} |det M[phi,mu]|^2: an HMC on |det M[phi,mu]|^2
    samples the reweighting ensemble of §3."""
    rng = np.random.default_rng(19)
    V = 2 * L * L
    delta = beta / Nt
    h = lattice.hopping_matrix(L)
    phi = random_field(rng, Nt, V, 1.0)
    dp = np.linalg.det(ops.dense_M(ops.transfer_matrix(h, delta * kappa, delta * mu), phi))
    dm = np.linalg.det(ops.dense_M(ops.transfer_matrix(h, delta * kappa, -delta * mu), phi))
    want = np.exp(1j * phi.sum()) * np.exp(beta * mu * V) * np.conj(dp)
    assert abs(dm - want) <= 1e-12 * abs(dm)


def test_sign_problem_weight():
    """det(M[phi,mu] M[phi,-mu]^dag) is real and positive at mu = 0 (it is
    |det M|^2) and picks up a non-trivial phase at mu != 0."""
    rng = np.random.default_rng(17)
    L, Nt, delta = 2, 4, 0.25
    V = 2 * L * L
    h = lattice.hopping_matrix(L)
    phi = random_field(rng, Nt, V, 1.0)

    def weight(mu):
        Mp = ops.dense_M(ops.transfer_matrix(h, delta, delta * mu), phi)
        Mm = ops.dense_M(ops.transfer_matrix(h, delta, -delta * mu), phi)
        return np.linalg.det(Mp) * np.conj(np.linalg.det(Mm))

    w0 = weight(0.0)
    assert abs(w0.imag) <= 1e-12 * abs(w0) and w0.real > 0
    w1 = weight(0.8)
    assert abs(np.angle(w1)) > 1e-3
