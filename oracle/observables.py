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
