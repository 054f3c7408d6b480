"""Observables from M^{-1} sources (oracle; test infrastructure only).

The paper (§2) measures the single-particle gap Delta from the decay of a
single-particle correlator; it names the observable, not its estimator.
Reading taken: the zero-momentum correlator on sublattice A from one
source b = V_A^{-1/2} on the A sites of slice 0,
    C(t) = V_A^{-1/2} sum_{x in A} (M^{-1} b)_t(x),   t = 0 .. Nt-1,
computed here by a dense LU solve of M (small lattices only).
"""
import numpy as np

from . import operators as ops


def correlator_k0(E, phi):
    Nt, V = phi.shape
    VA = V // 2
    b = np.zeros((Nt, V), dtype=np.complex128)
    b[0, :VA] = 1.0 / np.sqrt(VA)
    g = np.linalg.solve(ops.dense_M(E, phi), b.ravel()).reshape(Nt, V)
    return g[:, :VA].sum(axis=1) / np.sqrt(VA)


# ---------------------------------------------------------------------------
# Staggered spin correlations.  The paper's §2 names the staggered
# magnetisation, with the gap, as an order parameter of the transition; its
# estimator is cited, not printed.
#
# Reading taken.  In the particle-hole basis of §1 (spin up = particles p,
# spin down = holes h) the spin is S^3_x = (n^p_x + n^h_x - 1) / 2.  For one
# field, G = M[phi]^{-1} is the particle propagator on space-time points, and
# at mu = 0 the holes' matrix is M[-phi] = conj(M[phi]) (E is real), so the
# holes' propagator is conj(G).  With eps_x = +1 on sublattice A and -1 on B
# (on every slice), three space-time traces carry the spin structure:
#     T_s  = tr(eps G)          staggered density; Re T_s = 0 for every field
#                               at mu = 0, so the disconnected part of the
#                               staggered correlation vanishes
#     T_u  = tr(G)              filling; Re T_u = N / 2 (half filling)
#     T_ss = tr(eps G eps G)    the fermion loop of the staggered spin-spin
#                               correlation over all space-time pairs
# Wick's theorem for one field gives the connected density correlation
# <n_a n_b> - <n_a><n_b> = delta_ab G_aa - G_ab G_ba for each species, so the
# staggered space-time susceptibility of one field is
#     chi_s = (1/N) sum_{a,b} eps_a eps_b <S_a S_b> = (Re T_u - Re T_ss) / (2N),
# N = V Nt, whose ensemble average is the space-time integrated staggered
# spin correlation (its equal-time pairs depend on the time ordering the
# discretisation gives equal-time products; they are 1/Nt of the sum).
# At mu = 0 on the bipartite lattice (eps E eps = E^{-1}) the particle-hole
# symmetry reads eps G eps = 1 - G^dag, so T_ss = T_u - tr(G^dag G) and
# chi_s = |G|_F^2 / (2N); per real noise vector, T_u - T_ss = |M^{-1} eta|^2.
# Stochastic estimates use Z2 noise eta_k = +-1 (the lowest bit of Philox
# word 0 of element e, stream 4, trajectory counter k, the chain id):
# eta^dag eps M^{-1} eta, eta^dag M^{-1} eta and eta^dag eps M^{-1} eps
# M^{-1} eta are unbiased for the three traces.
# ---------------------------------------------------------------------------
from . import philox


def sublattice_signs(V):
    """eps_x: +1 on sublattice A (x < V/2), -1 on B."""
    return np.where(np.arange(V) < V // 2, 1.0, -1.0)


def z2_noise(seed, sample, chain, Nt, V):
    """eta(e) = 1 - 2 (word0 & 1) for e = t V + x, Philox stream 4."""
    x0 = philox._raw(seed, philox.STREAM_Z2, sample, chain, Nt * V)[0]
    return (1.0 - 2.0 * (x0 & np.uint64(1)).astype(np.float64)).reshape(Nt, V) + 0j


def spin_traces_exact(E, phi):
    """(T_s, T_u, T_ss) by a dense inverse of M."""
    Nt, V = phi.shape
    G = np.linalg.inv(ops.dense_M(E, phi))
    eps = np.tile(sublattice_signs(V), Nt)
    eG = eps[:, None] * G
    return complex(np.trace(eG)), complex(np.trace(G)), complex(np.trace(eG @ eG))


def spin_trace_samples(E, phi, n_noise, seed, chain=0, solve=None):
    """Per-sample Z2-noise estimates, array [n_noise, 3] of
    (eta^dag eps v, eta^dag v, eta^dag eps w) with v = M^{-1} eta_k and
    w = M^{-1} (eps v); dense solves of M unless `solve` is given."""
    Nt, V = phi.shape
    eps = sublattice_signs(V)
    if solve is None:
        Md = ops.dense_M(E, phi)

        def solve(b):
            return np.linalg.solve(Md, b.ravel()).reshape(Nt, V)
    out = np.zeros((n_noise, 3), dtype=np.complex128)
    for k in range(n_noise):
        eta = z2_noise(seed, k, chain, Nt, V)
        v = solve(eta)
        w = solve(eps * v)
        out[k] = (np.vdot(eta * eps, v), np.vdot(eta, v), np.vdot(eta * eps, w))
    return out


def spin_traces_noise(E, phi, n_noise, seed, chain=0, solve=None):
    """Means of the per-sample estimates of (T_s, T_u, T_ss)."""
    m = spin_trace_samples(E, phi, n_noise, seed, chain, solve).mean(axis=0)
    return complex(m[0]), complex(m[1]), complex(m[2])


def staggered_susceptibility(T_u, T_ss, N):
    """chi_s = (Re T_u - Re T_ss) / (2N) of one field at mu = 0."""
    return (np.real(T_u) - np.real(T_ss)) / (2.0 * N)
