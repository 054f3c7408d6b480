"""FP64 CPU oracle for the honeycomb-Hubbard HMC hot path (arXiv:2210.06874, §2).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
NumPy restatement of what the GPU library computes.  It exists to check the
CUDA path; it is never part of it.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py`` may import it.  It shares
no code with ``paper_2210_06874_gb300`` and imports nothing from it.

Modules
-------
lattice    honeycomb lattice and nearest-neighbour hopping matrix h (§1, Fig. 1)
operators  E = exp(delta*kappa*h); the fermion matrix M[phi] and M^dagger[phi]
           in the exponential-hopping form and in the printed mixed-differencing
           form of Eq. (2.2); dense builds for tiny lattices
hmc        CG on M M^dagger, action Eq. (2.1), force, leapfrog, Metropolis (§2)
philox     Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
           the Box-Muller normals drawn from it
hasenbusch mass preconditioning (Hasenbusch 2001) with a two-level nested
           leapfrog (Sexton and Weingarten 1992): heavy operator, the two
           pseudofermions, their forces, the nested schedule, a trajectory
observables zero-momentum single-particle correlator from one M^{-1} source;
           staggered spin traces of M^{-1} (dense and by Z2 noise) and the
           staggered susceptibility built from them

Conventions (readings of the paper where it leaves a choice):
  * field phi is the product delta*phi_paper, so phases are exp(+i phi) and the
    bosonic action is sum(phi^2) / (2 delta U)
  * site index x = s*L*L + m1*L + m2 (s=0: sublattice A, s=1: sublattice B)
  * space-time vectors are arrays of shape (Nt, V), time-major
  * (M psi)_t = psi_t - s_t * E * diag(exp(i phi_{t-1})) * psi_{t-1},
    s_0 = -1 (antiperiodic), s_t = +1 otherwise, t-1 taken mod Nt
"""
