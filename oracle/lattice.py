"""Honeycomb lattice and its hopping matrix h (oracle; test infrastructure only).

Paper: §1 and Fig. 1 -- two triangular sublattices (red A, blue B), every
nearest neighbour of a site lies on the other sublattice; the hopping term of
the Hamiltonian Eq. (1.1) couples nearest-neighbour pairs <x,y>.  Periodic
boundaries (§4 names them for the HMC).

Unit cell (m1, m2), 0 <= m1, m2 < L, holds an A site and a B site.  The A site
of cell (m1, m2) bonds to the B sites of cells (m1, m2), (m1-1, m2) and
(m1, m2-1), all indices mod L.  For L = 1 the three bonds join the same pair,
so h counts bond multiplicity (h[A,B] = 3); this keeps the Bloch spectrum
+-|1 + e^{i theta1} + e^{i theta2}| valid for every L.
"""
import numpy as np


def n_sites(L):
    """V = 2 L^2 sites for L x L unit cells."""
    return 2 * L * L


def site_index(s, m1, m2, L):
    """Sublattice-major site index x = s*L*L + (m1 mod L)*L + (m2 mod L)."""
    return s * L * L + (m1 % L) * L + (m2 % L)


def bonds(L):
    """List of (a, b) nearest-neighbour bonds, a on A, b on B (with multiplicity)."""
    out = []
    for m1 in range(L):
        for m2 in range(L):
            a = site_index(0, m1, m2, L)
            for d1, d2 in ((0, 0), (-1, 0), (0, -1)):
                out.append((a, site_index(1, m1 + d1, m2 + d2, L)))
    return out


def hopping_matrix(L):
    """Dense V x V real symmetric adjacency h (bond multiplicity counted)."""
    V = n_sites(L)
    h = np.zeros((V, V), dtype=np.float64)
    for a, b in bonds(L):
        h[a, b] += 1.0
        h[b, a] += 1.0
    return h


def sublattice(L):
    """Array of length V: 0 for A sites, 1 for B sites."""
    V = n_sites(L)
    return (np.arange(V) >= L * L).astype(np.int64)
