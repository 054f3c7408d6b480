"""Hasenbusch mass preconditioning with a two-level nested integrator
(oracle; test infrastructure only).

The paper (§2) credits its HMC's speed to improvements it cites but does not
print.  This module follows two published methods, restated from their
definitions: the determinant split of M. Hasenbusch, Phys. Lett. B 519
(2001) 177, and the multiple-time-scale leapfrog of J. C. Sexton and
D. H. Weingarten, Nucl. Phys. B 380 (1992) 665.

Heavy operator.  M_g = 1 - g S E D, i.e. the fermion matrix with the
transfer matrix scaled by g in [0, 1): its slice-to-slice hop is damped, so
M_g M_g^dag is well conditioned.  With
    det(M M^dag) = det(M_g M_g^dag) * det(M M^dag) / det(M_g M_g^dag)
two pseudofermions replace one:
    S_1 = chi_1^dag (M_g M_g^dag)^{-1} chi_1,            chi_1 = M_g rho_1
    S_2 = phi_2^dag (M M^dag)^{-1} phi_2,  phi_2 = M_g chi_2,
                                           chi_2 = M_g^{-1} M rho_2
(rho_1, rho_2 ~ exp(-rho^dag rho)); integrating chi_1 and chi_2 out gives
det(M_g M_g^dag) and det(M M^dag)/det(M_g M_g^dag), so the target density
is that of the plain HMC.  At the start S_1 = rho_1^dag rho_1 and
S_2 = rho_2^dag rho_2 exactly.

Forces (derived here; the paper prints none).  With dM/dphi_j = i (M - 1) P_j
(P_j the projector on space-time point j, acting on the source slice) and the
same for M_g:
    F_B = phi / (delta U)
    F_1 = 2 Im(x_1 conj(M_g^dag x_1)),                 x_1 = (M_g M_g^dag)^{-1} chi_1
    F_2 = 2 Im(x_2 conj(M^dag x_2)) - 2 Im(conj(M_g^dag x_2 - x_2) chi_2),
                                                       x_2 = (M M^dag)^{-1} phi_2
Nested integrator: outer leapfrog of n_outer steps of eps on S_2 (the small,
expensive ratio force), each drift replaced by n_inner leapfrog steps of
eps / n_inner on S_B + S_1 (the large, cheap forces).  Drift phi += c delta pi,
kick pi -= c delta F, the momenta conjugate to phi_paper as in the plain HMC.
Random numbers: momenta stream 0, rho_2 stream 1 (the plain pseudofermion's),
rho_1 stream 3, the Metropolis uniform stream 2.
"""
import numpy as np

from . import hmc
from . import operators as ops
from . import philox


def heavy_noise(seed, traj, chain, Nt, V):
    """rho_1 ~ exp(-rho^dag rho) from Philox stream 3."""
    z0, z1 = philox.normal_pair(seed, philox.STREAM_HEAVY, traj, chain, Nt * V)
    return ((z0 + 1j * z1) / np.sqrt(2.0)).reshape(Nt, V)


def nested_schedule(n_outer, n_inner):
    """Steps of the two-level leapfrog in units of the outer step eps, as a
    list of (kind, coefficient), kind in {"outer", "inner", "drift"}:
    outer(1/2), then n_outer times [ n_inner times (inner(h/2) drift(h)
    inner(h/2)), outer(1 or, the last time, 1/2) ], h = 1/n_inner, with
    consecutive inner kicks (at the same field) merged into one."""
    h = 1.0 / n_inner
    raw = [("outer", 0.5)]
    for k in range(n_outer):
        for _ in range(n_inner):
            raw += [("inner", 0.5 * h), ("drift", h), ("inner", 0.5 * h)]
        raw.append(("outer", 1.0 if k < n_outer - 1 else 0.5))
    steps = []
    for kind, c in raw:
        if steps and kind == "inner" and steps[-1][0] == "inner":
            steps[-1] = ("inner", steps[-1][1] + c)
        else:
            steps.append((kind, c))
    return steps


def heavy_solve(E, phi, b, g, tol, max_iter):
    """(M_g M_g^dag) x = b: the plain CG with the transfer matrix g E."""
    return hmc.cg_solve(g * E, phi, b, tol, max_iter)


def force_heavy(E, phi, x1, delta, U, g):
    """F_B + F_1 given x_1 = (M_g M_g^dag)^{-1} chi_1."""
    y = ops.apply_Mdag(g * E, phi, x1)
    return phi / (delta * U) + 2.0 * np.imag(x1 * np.conj(y))


def force_ratio(E, phi, x2, chi2, g):
    """F_2 given x_2 = (M M^dag)^{-1} M_g chi_2."""
    y = ops.apply_Mdag(E, phi, x2)
    w = ops.apply_Mdag(g * E, phi, x2) - x2
    return 2.0 * np.imag(x2 * np.conj(y)) - 2.0 * np.imag(np.conj(w) * chi2)


def pseudofermions(E, phi, rho1, rho2, g, tol=1e-14, max_iter=100000):
    """chi_1 = M_g rho_1 and chi_2 = M_g^{-1} M rho_2 = M_g^dag (M_g M_g^dag)^{-1} M rho_2."""
    chi1 = ops.apply_M(g * E, phi, rho1)
    w, _, _ = heavy_solve(E, phi, ops.apply_M(E, phi, rho2), g, tol, max_iter)
    chi2 = ops.apply_Mdag(g * E, phi, w)
    return chi1, chi2


def action(E, phi, chi1, chi2, delta, U, g, tol=1e-14, max_iter=100000):
    """S_B + S_1 + S_2 for fixed pseudofermions."""
    x1, _, _ = heavy_solve(E, phi, chi1, g, tol, max_iter)
    phi2 = ops.apply_M(g * E, phi, chi2)
    x2, _, _ = hmc.cg_solve(E, phi, phi2, tol, max_iter)
    return (hmc.bosonic_action(phi, delta, U) + float(np.vdot(chi1, x1).real)
            + float(np.vdot(phi2, x2).real))


def md(E, phi, pi, chi1, chi2, delta, U, g, eps, n_outer, n_inner, tol=1e-12,
       max_iter=100000):
    """The nested molecular dynamics from (phi, pi) with fixed pseudofermions.
    Returns (phi, pi, x1, x2, phi2, iterations by level, solves by level);
    x1, x2 and phi2 belong to the final field (the last kick of each level
    is there)."""
    phi, pi = phi.copy(), pi.copy()
    it = {"inner": 0, "outer": 0}
    solves = {"inner": 0, "outer": 0}
    x1 = x2 = phi2 = None
    for kind, c in nested_schedule(n_outer, n_inner):
        if kind == "drift":
            phi = phi + c * eps * delta * pi
        elif kind == "inner":
            x1, n, _ = heavy_solve(E, phi, chi1, g, tol, max_iter)
            it["inner"] += n
            solves["inner"] += 1
            pi = pi - c * eps * delta * force_heavy(E, phi, x1, delta, U, g)
        else:
            phi2 = ops.apply_M(g * E, phi, chi2)
            x2, n, _ = hmc.cg_solve(E, phi, phi2, tol, max_iter)
            it["outer"] += n
            solves["outer"] += 1
            pi = pi - c * eps * delta * force_ratio(E, phi, x2, chi2, g)
    return phi, pi, x1, x2, phi2, it, solves


def trajectory(E, phi0, delta, U, g, eps, n_outer, n_inner, seed, traj, chain=0,
               tol=1e-12, max_iter=100000):
    """One HMC update with the two pseudofermions and the nested integrator
    (eps = tau / n_outer).  Returns the new field and the diagnostics, with
    the CG iterations and solves of each level."""
    Nt, V = phi0.shape
    pi0 = philox.momenta(seed, traj, chain, Nt, V)
    rho2 = philox.pseudofermion_noise(seed, traj, chain, Nt, V)
    rho1 = heavy_noise(seed, traj, chain, Nt, V)
    chi1, chi2 = pseudofermions(E, phi0, rho1, rho2, g, tol, max_iter)
    H0 = (hmc.bosonic_action(phi0, delta, U) + float(np.vdot(rho1, rho1).real)
          + float(np.vdot(rho2, rho2).real) + 0.5 * float(np.sum(pi0 * pi0)))
    phi, pi, x1, x2, phi2, it, solves = md(E, phi0, pi0, chi1, chi2, delta, U, g, eps,
                                           n_outer, n_inner, tol, max_iter)
    H1 = (hmc.bosonic_action(phi, delta, U) + float(np.vdot(chi1, x1).real)
          + float(np.vdot(phi2, x2).real) + 0.5 * float(np.sum(pi * pi)))
    dH = H1 - H0
    u = philox.metropolis_uniform(seed, traj, chain)
    accept = bool(u < np.exp(-dH))
    return {"phi": phi if accept else phi0.copy(), "phi_proposed": phi, "pi_final": pi,
            "dH": dH, "H0": H0, "H1": H1, "accept": accept, "u": u,
            "cg_iters_inner": it["inner"], "cg_iters_outer": it["outer"],
            "solves_inner": solves["inner"], "solves_outer": solves["outer"],
            "chi1": chi1, "chi2": chi2}
