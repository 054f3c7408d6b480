"""Pins of the oracle's solver, action, force and integrator (CPU only).

  * CG against a dense LU solve; the true residual reaches the tolerance
  * pseudofermion identity: for chi = M rho, chi^dag (M M^dag)^{-1} chi = rho^dag rho
  * force against central finite differences of the action Eq. (2.1)
  * leapfrog reversibility and Delta H = O(eps^2)
  * Creutz equality <exp(-Delta H)> = 1 (exactness of the HMC, §2)
  * planted mistakes in the oracle are caught by these pins

Fields are drawn with half the width of the free auxiliary-field Gaussian
N(0, delta U): an i.i.d. draw at full width lands far from the
determinant-weighted distribution, where M is nearly singular and the
molecular dynamics is chaotic (reversibility then fails at the 1e-2 level).
"""
import numpy as np
import pytest

from oracle import hmc, lattice, operators as ops, philox


def setup(L=3, Nt=8, beta=2.0, U=2.0, scale=0.5, seed=1):
    delta = beta / Nt
    V = 2 * L * L
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    rng = np.random.default_rng(seed)
    phi = scale * rng.normal(0.0, np.sqrt(delta * U), size=(Nt, V))
    return E, phi, delta, U, rng


def test_cg_matches_dense_solve():
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    chi = rng.normal(size=(Nt, V)) + 1j * rng.normal(size=(Nt, V))
    x, it, res = hmc.cg_solve(E, phi, chi, tol=1e-13)
    M = ops.dense_M(E, phi)
    want = np.linalg.solve(M @ M.conj().T, chi.ravel()).reshape(Nt, V)
    assert res < 1e-12
    assert np.linalg.norm(x - want) <= 1e-10 * np.linalg.norm(want)
    assert 0 < it < 10000


def test_pseudofermion_identity():
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    rho = philox.pseudofermion_noise(11, 0, 0, Nt, V)
    chi = ops.apply_M(E, phi, rho)
    x, _, _ = hmc.cg_solve(E, phi, chi, tol=1e-14)
    assert abs(np.vdot(chi, x).real - np.vdot(rho, rho).real) < 1e-10 * np.vdot(rho, rho).real


def fd_gradient(E, phi, chi, delta, U, comps, h=1e-5):
    out = []
    for (t, x) in comps:
        p1, p2 = phi.copy(), phi.copy()
        p1[t, x] += h
        p2[t, x] -= h
        out.append((hmc.action(E, p1, chi, delta, U, tol=1e-14)
                    - hmc.action(E, p2, chi, delta, U, tol=1e-14)) / (2 * h))
    return np.array(out)


def test_force_matches_finite_differences():
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    rho = philox.pseudofermion_noise(5, 0, 0, Nt, V)
    chi = ops.apply_M(E, phi, rho)
    x, _, _ = hmc.cg_solve(E, phi, chi, tol=1e-14)
    F = hmc.force_from_solution(E, phi, x, delta, U)
    comps = [(0, 0), (0, V - 1), (3, 5), (Nt - 1, 9), (Nt - 1, V - 1)]
    fd = fd_gradient(E, phi, chi, delta, U, comps)
    an = np.array([F[c] for c in comps])
    assert np.allclose(an, fd, rtol=1e-6, atol=1e-6 * np.abs(F).max())


def test_leapfrog_reversible():
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    pi = rng.normal(size=(Nt, V))
    chi = ops.apply_M(E, phi, philox.pseudofermion_noise(3, 0, 0, Nt, V))
    p1, q1, _, _, _ = hmc.leapfrog(E, phi, pi, chi, delta, U, 0.1, 10, tol=1e-14)
    p2, q2, _, _, _ = hmc.leapfrog(E, p1, -q1, chi, delta, U, 0.1, 10, tol=1e-14)
    assert np.abs(p2 - phi).max() < 1e-10
    assert np.abs(q2 + pi).max() < 1e-10


def test_delta_h_scales_as_eps_squared():
    E, phi, delta, U, rng = setup(seed=4)
    Nt, V = phi.shape
    pi = philox.momenta(9, 0, 0, Nt, V)
    rho = philox.pseudofermion_noise(9, 0, 0, Nt, V)
    chi = ops.apply_M(E, phi, rho)
    H0 = hmc.bosonic_action(phi, delta, U) + np.vdot(rho, rho).real + 0.5 * np.sum(pi ** 2)
    tau = 1.0
    eps_list, dh = [], []
    for n in (4, 8, 16, 32):
        eps = tau / n
        p1, q1, x1, _, _ = hmc.leapfrog(E, phi, pi, chi, delta, U, eps, n, tol=1e-14)
        H1 = hmc.bosonic_action(p1, delta, U) + np.vdot(chi, x1).real + 0.5 * np.sum(q1 ** 2)
        eps_list.append(eps)
        dh.append(abs(H1 - H0))
    slope = np.polyfit(np.log(eps_list), np.log(dh), 1)[0]
    assert abs(slope - 2.0) < 0.15, (slope, dh)


def test_creutz_equality():
    """<exp(-Delta H)> = 1 for an exact HMC; coarse steps so Delta H = O(0.1)."""
    L, Nt, beta, U = 3, 8, 2.0, 2.0
    delta = beta / Nt
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta)
    phi = np.zeros((Nt, 2 * L * L))
    w, dh = [], []
    for traj in range(250):
        out = hmc.trajectory(E, phi, delta, U, eps=0.25, n_md=4, seed=77, traj=traj,
                             tol=1e-12)
        if traj >= 20:                     # after thermalisation from phi = 0
            w.append(np.exp(-out["dH"]))
            dh.append(abs(out["dH"]))
        phi = out["phi"]
    w = np.array(w)
    err = w.std() / np.sqrt(len(w))
    assert abs(w.mean() - 1.0) < 4 * err + 1e-3, (w.mean(), err)
    assert np.median(dh) > 0.02            # Delta H was not trivially 0


# ---------------------------------------------------------------------------
# planted mistakes (in the oracle, on the CPU) must fail the pins above
# ---------------------------------------------------------------------------
def test_planted_periodic_sign_is_caught(monkeypatch):
    monkeypatch.setattr(ops, "time_signs", lambda Nt: np.ones(Nt))
    E, _, _, _, _ = setup(L=2, Nt=4)
    _, logdet = np.linalg.slogdet(ops.dense_M(E, np.zeros((4, 8))))
    th = 2 * np.pi * np.arange(2) / 2
    f = np.abs(1 + np.exp(1j * th)[:, None] + np.exp(1j * th)[None, :]).ravel()
    want = np.sum(np.log1p(np.exp(2.0 * np.concatenate([f, -f]))))
    assert abs(logdet - want) > 1e-3


def test_planted_force_sign_is_caught(monkeypatch):
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    chi = ops.apply_M(E, phi, philox.pseudofermion_noise(5, 0, 0, Nt, V))
    x, _, _ = hmc.cg_solve(E, phi, chi, tol=1e-14)
    y = ops.apply_Mdag(E, phi, x)
    wrong = phi / (delta * U) - 2.0 * np.imag(x * np.conj(y))
    fd = fd_gradient(E, phi, chi, delta, U, [(3, 5)])
    assert abs(wrong[3, 5] - fd[0]) > 1e-3 * abs(fd[0])


def test_planted_adjoint_phase_is_caught(monkeypatch):
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    u = rng.normal(size=(Nt, V)) + 1j * rng.normal(size=(Nt, V))
    v = rng.normal(size=(Nt, V)) + 1j * rng.normal(size=(Nt, V))
    real = ops.apply_Mdag
    monkeypatch.setattr(ops, "apply_Mdag",
                        lambda E_, p_, s_: real(E_, -p_, s_))  # conj phase dropped
    lhs = np.vdot(u, ops.apply_M(E, phi, v))
    rhs = np.vdot(ops.apply_Mdag(E, phi, u), v)
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)


# ---------------------------------------------------------------------------
# second-order minimum-norm (Omelyan) integrator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["leapfrog", "omelyan"])
def test_integrator_schedule_consistency(kind):
    """Both move phi and pi over the same total time n_md*eps and are
    palindromic (time-reversible by construction)."""
    for n in (1, 3, 7):
        kicks, drift = hmc.integrator_schedule(kind, n)
        assert abs(sum(kicks) - n) < 1e-14
        assert abs(drift * (len(kicks) - 1) - n) < 1e-14
        assert np.allclose(kicks, kicks[::-1], rtol=0, atol=1e-15)


def test_omelyan_reversible():
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    pi = rng.normal(size=(Nt, V))
    chi = ops.apply_M(E, phi, philox.pseudofermion_noise(3, 0, 0, Nt, V))
    p1, q1, _, _, _ = hmc.leapfrog(E, phi, pi, chi, delta, U, 0.2, 5, tol=1e-14,
                                   integrator="omelyan")
    p2, q2, _, _, _ = hmc.leapfrog(E, p1, -q1, chi, delta, U, 0.2, 5, tol=1e-14,
                                   integrator="omelyan")
    assert np.abs(p2 - phi).max() < 1e-10
    assert np.abs(q2 + pi).max() < 1e-10


def _delta_h(E, phi, pi, rho, delta, U, eps, n, kind):
    chi = ops.apply_M(E, phi, rho)
    H0 = hmc.bosonic_action(phi, delta, U) + np.vdot(rho, rho).real + 0.5 * np.sum(pi ** 2)
    p1, q1, x1, _, _ = hmc.leapfrog(E, phi, pi, chi, delta, U, eps, n, tol=1e-14,
                                    integrator=kind)
    H1 = hmc.bosonic_action(p1, delta, U) + np.vdot(chi, x1).real + 0.5 * np.sum(q1 ** 2)
    return H1 - H0


def test_omelyan_delta_h_scales_as_eps_squared():
    E, phi, delta, U, rng = setup(seed=4)
    Nt, V = phi.shape
    pi = philox.momenta(9, 0, 0, Nt, V)
    rho = philox.pseudofermion_noise(9, 0, 0, Nt, V)
    eps_list, dh = [], []
    for n in (2, 4, 8, 16):
        eps = 1.0 / n
        eps_list.append(eps)
        dh.append(abs(_delta_h(E, phi, pi, rho, delta, U, eps, n, "omelyan")))
    slope = np.polyfit(np.log(eps_list), np.log(dh), 1)[0]
    assert abs(slope - 2.0) < 0.2, (slope, dh)


def test_omelyan_beats_leapfrog_at_equal_step():
    """At the same step size the minimum-norm integrator's energy violation
    is several times smaller than leapfrog's (its leading error
    coefficients are minimised): RMS of Delta H over 8 momenta draws (a
    single draw can make either one accidentally small)."""
    E, phi, delta, U, rng = setup(seed=5)
    Nt, V = phi.shape
    lf, om = [], []
    for k in range(8):
        pi = philox.momenta(20 + k, 0, 0, Nt, V)
        rho = philox.pseudofermion_noise(20 + k, 0, 0, Nt, V)
        lf.append(_delta_h(E, phi, pi, rho, delta, U, 0.1, 10, "leapfrog"))
        om.append(_delta_h(E, phi, pi, rho, delta, U, 0.1, 10, "omelyan"))
    ratio = np.sqrt(np.mean(np.square(om)) / np.mean(np.square(lf)))
    assert ratio < 0.3, (ratio, lf, om)


def test_planted_asymmetric_schedule_is_caught(monkeypatch):
    """A schedule that is not a palindrome (last kick 2 lam instead of lam)
    must break reversibility."""
    real = hmc.integrator_schedule

    def broken(kind, n):
        kicks, drift = real(kind, n)
        kicks = list(kicks)
        kicks[-1] = 2.0 * hmc.OMELYAN_LAMBDA
        return kicks, drift
    monkeypatch.setattr(hmc, "integrator_schedule", broken)
    E, phi, delta, U, rng = setup()
    Nt, V = phi.shape
    pi = rng.normal(size=(Nt, V))
    chi = ops.apply_M(E, phi, philox.pseudofermion_noise(3, 0, 0, Nt, V))
    p1, q1, _, _, _ = hmc.leapfrog(E, phi, pi, chi, delta, U, 0.2, 5, tol=1e-14,
                                   integrator="omelyan")
    p2, q2, _, _, _ = hmc.leapfrog(E, p1, -q1, chi, delta, U, 0.2, 5, tol=1e-14,
                                   integrator="omelyan")
    assert np.abs(p2 - phi).max() > 1e-6 or np.abs(q2 + pi).max() > 1e-6
