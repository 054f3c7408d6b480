"""Pins of the oracle's mass preconditioning with a nested integrator
(Hasenbusch 2001; Sexton and Weingarten 1992), on CPU.

* g = 0 with one inner step reduces to the plain leapfrog HMC of the same
  seeds (M_0 = 1: S_1 is constant, F_1 = 0, chi_2 = M rho_2, and the merged
  kicks are those of the plain leapfrog);
* at the start S_1 + S_2 = rho_1^dag rho_1 + rho_2^dag rho_2 exactly;
* the forces are the derivative of S_B + S_1 + S_2 (central differences);
  dropped or sign-flipped terms are caught;
* the nested schedule is symmetric and integrates each force over the whole
  trajectory; the molecular dynamics is reversible and Delta H falls as
  eps^2;
* at kappa = 0 the chain samples the atomic-limit weight of the §1
  Hamiltonian (Creutz <exp(-Delta H)> = 1 as well); a planted wrong second
  pseudofermion (chi_2 = M rho_2, dropping M_g^{-1}) breaks Creutz's
  identity, and correlated noise of the two pseudofermions biases the
  sampled weight.
"""
import numpy as np
import pytest

from oracle import hasenbusch as hb, hmc, lattice, operators as ops, philox
from paper_2210_06874_gb300 import synth

from test_oracle_atomic import ATOM, cos_phase_target

L, NT, BETA, U = 3, 8, 2.0, 2.0
V, DELTA = 2 * L * L, BETA / NT


def setup(seed=3, scale=0.5):
    E = ops.transfer_matrix(lattice.hopping_matrix(L), DELTA)
    phi = synth.gaussian_field(seed, NT, V, DELTA * U, scale=scale)
    return E, phi


def noise(seed):
    rng = np.random.default_rng(seed)
    return [(rng.normal(size=(NT, V)) + 1j * rng.normal(size=(NT, V))) / np.sqrt(2.0)
            for _ in range(2)]


def test_gamma_zero_is_plain_leapfrog():
    E, phi = setup()
    a = hb.trajectory(E, phi, DELTA, U, 0.0, 0.1, 10, 1, 7, 0, tol=1e-14)
    b = hmc.trajectory(E, phi, DELTA, U, 0.1, 10, 7, 0, tol=1e-14)
    assert abs(a["dH"] - b["dH"]) < 1e-10
    assert np.abs(a["phi_proposed"] - b["phi_proposed"]).max() < 1e-12
    assert a["accept"] == b["accept"] and a["u"] == b["u"]


@pytest.mark.parametrize("g", [0.3, 0.8])
def test_start_action_is_noise_norm(g):
    E, phi = setup()
    rho1, rho2 = noise(1)
    chi1, chi2 = hb.pseudofermions(E, phi, rho1, rho2, g)
    S = hb.action(E, phi, chi1, chi2, DELTA, U, g) - hmc.bosonic_action(phi, DELTA, U)
    want = float(np.vdot(rho1, rho1).real + np.vdot(rho2, rho2).real)
    assert abs(S - want) < 1e-10 * want


def fd_check(force_fn, g=0.6, points=((0, 0), (3, 5), (7, 17), (5, 9))):
    E, phi = setup()
    rho1, rho2 = noise(2)
    chi1, chi2 = hb.pseudofermions(E, phi, rho1, rho2, g)
    F = force_fn(E, phi, chi1, chi2, g)
    h, worst = 1e-5, 0.0
    for t, x in points:
        pp, pm = phi.copy(), phi.copy()
        pp[t, x] += h
        pm[t, x] -= h
        fd = (hb.action(E, pp, chi1, chi2, DELTA, U, g) -
              hb.action(E, pm, chi1, chi2, DELTA, U, g)) / (2 * h)
        worst = max(worst, abs(F[t, x] - fd) / max(1.0, abs(fd)))
    return worst


def total_force(E, phi, chi1, chi2, g, ratio=hb.force_ratio):
    x1, _, _ = hb.heavy_solve(E, phi, chi1, g, 1e-14, 100000)
    phi2 = ops.apply_M(g * E, phi, chi2)
    x2, _, _ = hmc.cg_solve(E, phi, phi2, 1e-14, 100000)
    return hb.force_heavy(E, phi, x1, DELTA, U, g) + ratio(E, phi, x2, chi2, g)


def test_forces_match_finite_differences():
    assert fd_check(total_force) < 1e-6


def test_planted_force_mistakes_are_caught():
    def dropped(E, phi, x2, chi2, g):      # the M_g dependence of phi_2 left out
        y = ops.apply_Mdag(E, phi, x2)
        return 2.0 * np.imag(x2 * np.conj(y))

    def flipped(E, phi, x2, chi2, g):      # wrong sign of that term
        y = ops.apply_Mdag(E, phi, x2)
        w = ops.apply_Mdag(g * E, phi, x2) - x2
        return 2.0 * np.imag(x2 * np.conj(y)) + 2.0 * np.imag(np.conj(w) * chi2)

    for bad in (dropped, flipped):
        assert fd_check(lambda E, p, c1, c2, g: total_force(E, p, c1, c2, g, bad)) > 1e-3


@pytest.mark.parametrize("n_outer,n_inner", [(1, 1), (3, 2), (5, 4)])
def test_schedule_is_symmetric_and_complete(n_outer, n_inner):
    s = hb.nested_schedule(n_outer, n_inner)
    assert s == s[::-1]
    tot = {k: sum(c for kk, c in s if kk == k) for k in ("outer", "inner", "drift")}
    assert all(abs(v - n_outer) < 1e-12 for v in tot.values())
    # no two kicks of the inner level in a row, every drift between kicks
    assert all(not (a[0] == "inner" and b[0] == "inner") for a, b in zip(s, s[1:]))
    assert sum(1 for k, _ in s if k == "outer") == n_outer + 1


def test_md_is_reversible():
    E, phi = setup()
    rho1, rho2 = noise(3)
    g = 0.5
    chi1, chi2 = hb.pseudofermions(E, phi, rho1, rho2, g)
    pi = philox.momenta(5, 0, 0, NT, V)
    p1, q1, *_ = hb.md(E, phi, pi, chi1, chi2, DELTA, U, g, 0.2, 5, 3, tol=1e-14)
    p2, q2, *_ = hb.md(E, p1, -q1, chi1, chi2, DELTA, U, g, 0.2, 5, 3, tol=1e-14)
    assert np.abs(p2 - phi).max() < 1e-11
    assert np.abs(q2 + pi).max() < 1e-10


def test_delta_h_falls_as_eps_squared():
    E, phi = setup()
    n = np.array([4, 8, 16, 32])
    dh = [abs(hb.trajectory(E, phi, DELTA, U, 0.5, 1.0 / k, int(k), 2, 7, 0,
                            tol=1e-14)["dH"]) for k in n]
    slope = -np.polyfit(np.log(n), np.log(dh), 1)[0]
    assert abs(slope - 2.0) < 0.15, (slope, dh)


# ---------------------------------------------------------------- atomic limit
def sample_cos_phase_hb(g, n_inner=2):
    a = ATOM
    delta = a["beta"] / a["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(a["L"]), 0.0)
    phi = np.zeros((a["Nt"], 2 * a["L"] ** 2))
    vals, boltz = [], []
    for traj in range(a["n_therm"] + a["n_traj"]):
        out = hb.trajectory(E, phi, delta, a["U"], g, a["eps"], a["n_md"], n_inner,
                            a["seed"], traj, tol=1e-12)
        phi = out["phi"]
        if traj >= a["n_therm"]:
            vals.append(np.cos(phi.sum(axis=0)).mean())
            boltz.append(np.exp(-out["dH"]))
    vals = np.asarray(vals)
    blocks = vals.reshape(20, -1).mean(axis=1)
    return vals.mean(), blocks.std(ddof=1) / np.sqrt(len(blocks)), np.mean(boltz)


@pytest.mark.slow
def test_hasenbusch_chain_samples_atomic_limit():
    mean, err, creutz = sample_cos_phase_hb(0.5)
    assert err < 0.015
    assert abs(mean - cos_phase_target()) < 4.0 * err, (mean, err)
    assert abs(creutz - 1.0) < 0.05


@pytest.mark.slow
def test_planted_wrong_second_pseudofermion_is_caught(monkeypatch):
    """chi_2 = M rho_2 (M_g^{-1} dropped): the start action no longer equals
    the noise norm, Creutz's identity fails."""
    def wrong(E, phi, rho1, rho2, g, tol=1e-14, max_iter=100000):
        return ops.apply_M(g * E, phi, rho1), ops.apply_M(E, phi, rho2)
    monkeypatch.setattr(hb, "pseudofermions", wrong)
    _, _, creutz = sample_cos_phase_hb(0.5)
    assert abs(creutz - 1.0) > 0.2, creutz


@pytest.mark.slow
def test_planted_correlated_noise_is_caught(monkeypatch):
    """rho_1 drawn from rho_2's stream: the two pseudofermions are no longer
    independent and the chain samples a different weight."""
    monkeypatch.setattr(hb, "heavy_noise", lambda seed, traj, chain, Nt, V:
                        philox.pseudofermion_noise(seed, traj, chain, Nt, V))
    mean, err, _ = sample_cos_phase_hb(0.5)
    assert abs(mean - cos_phase_target()) > 4.0 * err, (mean, err)
