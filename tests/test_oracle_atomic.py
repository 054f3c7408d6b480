"""Atomic-limit pins of the oracle's weight and sampler (CPU only).

At kappa = 0 the Hamiltonian of §1 in the particle-hole basis,
H = (U/2) sum_x rho_x^2 + mu sum_x rho_x with rho_x = p^dag p - h^dag h,
falls apart into independent sites with four states each: rho = 0 twice,
rho = +1 and rho = -1, so every site contributes

    Z_atom = 2 + exp(-beta (U/2 + mu)) + exp(-beta (U/2 - mu))
           = 2 + 2 cosh(beta mu) exp(-beta U / 2).

Without hopping the Trotter splitting is exact and the Gaussian
auxiliary-field integral of Eq. (2.1) reproduces this for any Nt: the
weight exp(-S_B) det(M[phi, mu] M[phi, -mu]^dag), averaged over the
Gaussian exp(-S_B) alone, is the product over sites of Z_atom evaluated
at that site's field.  A site held at phi = 0 contributes
(1 + e^{beta mu})(1 + e^{-beta mu}) = 2 + 2 cosh(beta mu).

These facts come from the Hamiltonian, not from the oracle's formulas, so
they pin the coefficient of the bosonic action (delta U), the phase
convention, the antiperiodic boundary and the way mu enters, all at once.
The second half checks that the oracle's HMC samples this weight.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import hmc, lattice, operators as ops, philox


def gaussian_average_of_weight(Nt, beta, U, mu=0.0, n=81, width=8.0):
    """<det(M[phi,mu] M[phi,-mu]^dag)> over exp(-S_B) at kappa = 0, L = 1,
    by trapezoidal quadrature over the Nt field components of site 0 (site 1
    stays at phi = 0).  The oracle's bosonic action is the weight; the
    nodes span +-width standard deviations of a N(0, delta U) component
    (wide enough for any reasonable coefficient; the integrand is smooth, so
    the trapezoidal rule converges geometrically)."""
    delta = beta / Nt
    h = lattice.hopping_matrix(1)
    E_p = ops.transfer_matrix(h, 0.0, delta * mu)
    E_m = ops.transfer_matrix(h, 0.0, -delta * mu)
    nodes = np.linspace(-width, width, n) * np.sqrt(delta * U)
    num = 0.0
    den = 0.0
    for idx in np.ndindex(*(n,) * Nt):
        phi = np.zeros((Nt, 2))
        phi[:, 0] = nodes[list(idx)]
        w = np.exp(-hmc.bosonic_action(phi, delta, U))
        d = np.linalg.det(ops.dense_M(E_p, phi)) * np.conj(np.linalg.det(ops.dense_M(E_m, phi)))
        num += w * d
        den += w
    return num / den


def z_atom(beta, U, mu=0.0):
    return 2.0 + 2.0 * np.cosh(beta * mu) * np.exp(-0.5 * beta * U)


@pytest.mark.parametrize("Nt,beta,U,mu,n", [
    (2, 1.0, 2.0, 0.0, 81),
    (2, 0.8, 3.0, 0.7, 81),     # chemical potential
    (3, 1.0, 2.0, 0.0, 33),     # delta = beta/3: the variance adds up over slices
])
def test_atomic_limit_partition_function(Nt, beta, U, mu, n):
    got = gaussian_average_of_weight(Nt, beta, U, mu, n=n)
    want = (2.0 + 2.0 * np.cosh(beta * mu)) * z_atom(beta, U, mu)
    assert abs(got.imag) < 1e-12 * want
    assert abs(got.real - want) < 1e-12 * want, (got, want)


def test_planted_bosonic_coefficient_is_caught(monkeypatch):
    """S_B = sum phi^2 / (2U) (delta dropped) gives the atom at the wrong
    temperature."""
    monkeypatch.setattr(hmc, "bosonic_action",
                        lambda phi, delta, U: float(np.sum(phi * phi) / (2.0 * U)))
    got = gaussian_average_of_weight(2, 1.0, 2.0)
    assert abs(got.real - 4.0 * z_atom(1.0, 2.0)) > 1e-2


def test_planted_periodic_boundary_is_caught(monkeypatch):
    """Periodic fermions turn 1 + e^{i Phi} into 1 - e^{i Phi}: the atom's
    weight becomes 2 - 2 cos Phi."""
    monkeypatch.setattr(ops, "time_signs", lambda Nt: np.ones(Nt))
    got = gaussian_average_of_weight(2, 1.0, 2.0)
    assert abs(got.real - 4.0 * z_atom(1.0, 2.0)) > 1e-2


# ---------------------------------------------------------------------------
# the HMC samples the atomic-limit weight
# ---------------------------------------------------------------------------
# L = 1, Nt = 4, beta = 1, U = 1 (delta = 1/4).  The bosonic term alone
# makes each field mode oscillate with angular frequency sqrt(delta/U) = 1/2
# in molecular-dynamics time, so trajectories of length 3 (6 steps of 1/2)
# take the field about a quarter period: successive measurements are
# nearly independent.
ATOM = dict(L=1, Nt=4, beta=1.0, U=1.0, eps=0.5, n_md=6, n_traj=600, n_therm=10, seed=11)


def sample_cos_phase():
    """HMC chain from phi = 0; per trajectory the site average of
    cos(Phi_x), Phi_x = sum_t phi_{x,t}.  Returns (mean, error of the mean
    from 20 blocks, acceptance)."""
    a = ATOM
    delta = a["beta"] / a["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(a["L"]), 0.0)
    phi = np.zeros((a["Nt"], 2 * a["L"] ** 2))
    vals, acc = [], 0
    for traj in range(a["n_therm"] + a["n_traj"]):
        out = hmc.trajectory(E, phi, delta, a["U"], eps=a["eps"], n_md=a["n_md"],
                             seed=a["seed"], traj=traj, tol=1e-12)
        phi = out["phi"]
        if traj >= a["n_therm"]:
            vals.append(np.cos(phi.sum(axis=0)).mean())
            acc += out["accept"]
    vals = np.asarray(vals)
    blocks = vals.reshape(20, -1).mean(axis=1)
    return vals.mean(), blocks.std(ddof=1) / np.sqrt(len(blocks)), acc / a["n_traj"]


def cos_phase_target():
    """<cos Phi> under the atomic weight: Phi ~ N(0, beta U) times
    |1 + e^{i Phi}|^2 = 2 + 2 cos Phi.  The weight vanishes at Phi = +-pi
    and the pseudofermion action diverges there, so a chain started at
    phi = 0 stays in (-pi, pi); the integral is taken over that interval
    (at beta U = 1 it differs from the one over the real line by 1e-4)."""
    bu = ATOM["beta"] * ATOM["U"]

    def w(p):
        return np.exp(-p * p / (2.0 * bu)) * (1.0 + np.cos(p))
    num = integrate.quad(lambda p: np.cos(p) * w(p), -np.pi, np.pi)[0]
    return num / integrate.quad(w, -np.pi, np.pi)[0]


def test_hmc_samples_atomic_limit():
    mean, err, acc = sample_cos_phase()
    target = cos_phase_target()
    assert err < 0.015
    assert acc > 0.9
    assert abs(mean - target) < 4.0 * err, (mean, err, target)
    # the determinant matters: the Gaussian alone gives exp(-beta U / 2)
    assert abs(mean - np.exp(-0.5 * ATOM["beta"] * ATOM["U"])) > 6.0 * err


def test_planted_pseudofermion_variance_is_caught(monkeypatch):
    """Re and Im of the pseudofermion noise with variance 1 instead of 1/2
    (exp(-rho^dag rho/2) in place of exp(-rho^dag rho)) breaks the heat
    bath: the chain then samples another weight."""
    real = philox.pseudofermion_noise
    monkeypatch.setattr(philox, "pseudofermion_noise",
                        lambda *a: np.sqrt(2.0) * real(*a))
    mean, err, _ = sample_cos_phase()
    assert abs(mean - cos_phase_target()) > 4.0 * err, (mean, err)


def test_planted_momentum_variance_is_caught(monkeypatch):
    """Momenta of variance 2 while the Hamiltonian keeps pi^2/2."""
    real = philox.momenta
    monkeypatch.setattr(philox, "momenta", lambda *a: np.sqrt(2.0) * real(*a))
    mean, err, _ = sample_cos_phase()
    assert abs(mean - cos_phase_target()) > 4.0 * err, (mean, err)
