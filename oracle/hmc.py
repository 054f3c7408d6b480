"""Pseudofermion HMC on the exponential-hopping fermion matrix
(oracle; test infrastructure only).

Paper §2: effective Hamiltonian Eq. (2.1)
    H = delta/(2U) phi_paper^2 + chi^dag (M M^dag)^{-1} chi + pi^2/2,
momenta pi ~ exp(-pi^2/2), rho ~ exp(-rho^dag rho), chi = M rho, a molecular
dynamics trajectory, acceptance min(1, exp(-Delta H)).  The stored field is the
phase angle phi = delta * phi_paper, so the bosonic term reads
sum(phi^2)/(2 delta U).  The momenta stay conjugate to phi_paper as in
Eq. (2.1), hence in terms of the stored phi
    d phi / d tau = delta * pi,     d pi / d tau = -delta * dS/dphi.

Force (derived, not printed in the paper): with x = (M M^dag)^{-1} chi and
y = M^dag x,  dS/dphi_{x,t} = phi_{x,t}/(delta U) + 2 Im(x_{x,t} conj(y_{x,t})).

Integrator (the paper does not name one): leapfrog
    kick(eps/2) [drift(eps) kick(eps)]^(n-1) drift(eps) kick(eps/2)
with drift phi += eps*delta*pi and kick pi -= eps*delta*dS/dphi; as an
option, among the HMC improvements the paper refers to, the second-order
minimum-norm integrator of Omelyan, Mryglod and Folk (2003) (see
integrator_schedule).
CG: plain conjugate gradient on A = M M^dag from x0 = 0, stopping when the
recursive residual satisfies |r| <= tol |chi|.
"""
import numpy as np

from . import operators as ops
from . import philox


def bosonic_action(phi, delta, U):
    return float(np.sum(phi * phi) / (2.0 * delta * U))


def cg_solve(E, phi, chi, tol=1e-12, max_iter=10000):
    """Solve (M M^dag) x = chi.  Returns (x, iterations, true relative residual)."""
    x = np.zeros_like(chi)
    r = chi.copy()
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    chi_norm = np.sqrt(float(np.vdot(chi, chi).real))
    it = 0
    if chi_norm == 0.0:
        return x, 0, 0.0
    while it < max_iter:
        q = ops.apply_Mdag(E, phi, p)
        qq = float(np.vdot(q, q).real)         # p^dag M M^dag p = |M^dag p|^2
        alpha = rr / qq
        x = x + alpha * p
        r = r - alpha * ops.apply_M(E, phi, q)
        rr_new = float(np.vdot(r, r).real)
        it += 1
        if np.sqrt(rr_new) <= tol * chi_norm:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    res = chi - ops.apply_MMdag(E, phi, x)
    return x, it, float(np.sqrt(np.vdot(res, res).real) / chi_norm)


def force_from_solution(E, phi, x, delta, U):
    """dS/dphi given the kept solve x = (M M^dag)^{-1} chi."""
    y = ops.apply_Mdag(E, phi, x)
    return phi / (delta * U) + 2.0 * np.imag(x * np.conj(y))


def action(E, phi, chi, delta, U, tol=1e-13, max_iter=10000):
    x, _, _ = cg_solve(E, phi, chi, tol, max_iter)
    return bosonic_action(phi, delta, U) + float(np.vdot(chi, x).real)


# Minimum-norm parameter of the second-order integrator of Omelyan, Mryglod
# and Folk (Comput. Phys. Commun. 151 (2003) 272), the value that minimises
# the norm of its leading error terms.
OMELYAN_LAMBDA = 0.1931833275037836


def integrator_schedule(kind, n_md):
    """(kicks, drift) of a symmetric second-order integrator of n_md steps
    of length eps: the update is kick(kicks[0] eps), then for m = 1 .. M
    drift(drift eps) followed by kick(kicks[m] eps).
      leapfrog:  M = n_md, drift 1, kicks 1/2, 1, ..., 1, 1/2
      omelyan:   M = 2 n_md, drift 1/2, kicks lam, 1-2lam, 2lam, 1-2lam, ...,
                 2lam, 1-2lam, lam  (two force evaluations per step)"""
    if kind == "leapfrog":
        kicks = [0.5] + [1.0] * (n_md - 1) + [0.5]
        return kicks, 1.0
    if kind == "omelyan":
        lam = OMELYAN_LAMBDA
        kicks = [lam]
        for m in range(1, 2 * n_md):
            kicks.append(1.0 - 2.0 * lam if m % 2 == 1 else 2.0 * lam)
        kicks.append(lam)
        return kicks, 0.5
    raise ValueError(kind)


def leapfrog(E, phi, pi, chi, delta, U, eps, n_md, tol=1e-12, max_iter=10000,
             integrator="leapfrog"):
    """Molecular dynamics of n_md steps with the given integrator (leapfrog
    by default, see integrator_schedule).  Returns (phi, pi, x_final, total
    CG iterations, number of solves).  x_final is the solve at the final phi."""
    kicks, drift = integrator_schedule(integrator, n_md)
    phi = phi.copy()
    pi = pi.copy()
    iters, solves = 0, 0
    for m, k in enumerate(kicks):
        if m > 0:
            phi = phi + drift * eps * delta * pi
        x, it, _ = cg_solve(E, phi, chi, tol, max_iter)
        iters += it
        solves += 1
        pi = pi - k * eps * delta * force_from_solution(E, phi, x, delta, U)
    return phi, pi, x, iters, solves


def trajectory(E, phi0, delta, U, eps, n_md, seed, traj, chain=0,
               tol=1e-12, max_iter=10000, integrator="leapfrog"):
    """One HMC update (§2).  Random draws come from the Philox streams.
    Returns a dict with the new field and the diagnostics."""
    Nt, V = phi0.shape
    pi0 = philox.momenta(seed, traj, chain, Nt, V)
    rho = philox.pseudofermion_noise(seed, traj, chain, Nt, V)
    chi = ops.apply_M(E, phi0, rho)
    # chi^dag (M M^dag)^{-1} chi = rho^dag rho exactly at the start field
    H0 = (bosonic_action(phi0, delta, U) + float(np.vdot(rho, rho).real)
          + 0.5 * float(np.sum(pi0 * pi0)))
    phi1, pi1, x1, iters, solves = leapfrog(E, phi0, pi0, chi, delta, U, eps,
                                            n_md, tol, max_iter, integrator)
    H1 = (bosonic_action(phi1, delta, U) + float(np.vdot(chi, x1).real)
          + 0.5 * float(np.sum(pi1 * pi1)))
    dH = H1 - H0
    u = philox.metropolis_uniform(seed, traj, chain)
    accept = bool(u < np.exp(-dH))
    return {
        "phi": phi1 if accept else phi0.copy(),
        "phi_proposed": phi1,
        "pi_final": pi1,
        "dH": dH,
        "H0": H0,
        "H1": H1,
        "accept": accept,
        "u": u,
        "cg_iters": iters,
        "cg_solves": solves,
        "chi": chi,
        "x_final": x1,
    }
