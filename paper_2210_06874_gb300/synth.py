"""Seeded synthetic inputs and the named workloads (no method arithmetic).

This module only draws random numbers and lists sizes: both the CUDA path
(through tests and bench.py) and the CPU oracle take their inputs from here,
and neither side's arithmetic lives here.  Random numbers the method itself
draws (momenta, pseudofermion noise, the Metropolis uniform) are not made
here: each side generates them from the shared Philox stream definition.

Workloads (the paper publishes no dataset; all inputs are synthetic):
  l3_nt8     L=3 (18 sites), kappa=1, U=2, beta=2, Nt=8, 10 leapfrog steps of
             0.1, CG to 1e-12, FP64; start field phi ~ N(0, delta U)
  l6_nt32    L=6 (72 sites), U=3.5, beta=4, Nt=32, 20 steps over tau=1,
             complex64 CG vectors (mixed path), true residual 1e-10
  l12_nt64   L=12 (288 sites), U=3.8, beta=8, Nt=64, 20 steps, mixed vs FP64
  batch256   256 chains, L in {3,6,9,12}, Nt in {16,32,48,64}, U in [2,5],
             beta = Nt/8
  l24_nt96   L=24 (1152 sites), U=4, beta=12, Nt=96, 30 steps of 1/30
phi is the phase angle delta*phi_paper; its free (bosonic-only) distribution
is N(0, delta U).  Start fields other than l3_nt8 are cold (phi = 0) or
thermalised by warm-up trajectories: an i.i.d. N(0, delta U) draw on the larger
lattices lands on nearly singular M (condition numbers of M M^dag ~ 1e9 at
L=6), far from the determinant-weighted distribution.
"""
import numpy as np

BASE_SEED = 2210068740

WORKLOADS = {
    "l3_nt8": dict(L=3, Nt=8, kappa=1.0, U=2.0, beta=2.0, n_md=10, traj_length=1.0,
                   cg_tol=1e-12, precision="fp64", n_traj=200, start="gaussian",
                   seed=BASE_SEED + 0),
    "l6_nt32": dict(L=6, Nt=32, kappa=1.0, U=3.5, beta=4.0, n_md=20, traj_length=1.0,
                    cg_tol=1e-10, precision="mixed", n_traj=500, start="cold",
                    seed=BASE_SEED + 1),
    "l12_nt64": dict(L=12, Nt=64, kappa=1.0, U=3.8, beta=8.0, n_md=20, traj_length=1.0,
                     cg_tol=1e-10, precision="mixed", n_traj=100, start="cold",
                     seed=BASE_SEED + 2),
    "l24_nt96": dict(L=24, Nt=96, kappa=1.0, U=4.0, beta=12.0, n_md=30, traj_length=1.0,
                     cg_tol=1e-10, precision="mixed", n_traj=100, start="cold",
                     seed=BASE_SEED + 4),
}


def batch256(seed=BASE_SEED + 3, n_chains=256):
    """Per-chain sizes of the batched workload: L, Nt uniform from the sets,
    U/kappa uniform in [2, 5], beta = Nt * 0.125 (delta = 1/8)."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([3, 6, 9, 12], size=n_chains)
    Nts = rng.choice([16, 32, 48, 64], size=n_chains)
    Us = rng.uniform(2.0, 5.0, size=n_chains)
    return [dict(L=int(L), Nt=int(Nt), kappa=1.0, U=float(U), beta=Nt * 0.125, n_md=20,
                 traj_length=1.0, cg_tol=1e-10) for L, Nt, U in zip(Ls, Nts, Us)]


def n_sites(L):
    return 2 * L * L


def gaussian_field(seed, Nt, V, variance, scale=1.0):
    """phi ~ N(0, variance) i.i.d., times `scale`, shape (Nt, V), float64."""
    rng = np.random.default_rng(seed)
    return scale * rng.normal(0.0, np.sqrt(variance), size=(Nt, V))


def complex_gaussian(seed, Nt, V):
    """psi with independent N(0,1) real and imaginary parts, (Nt, V) complex128."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(Nt, V)) + 1j * rng.normal(size=(Nt, V))


def start_field(name, seed=None):
    w = WORKLOADS[name]
    V, Nt = n_sites(w["L"]), w["Nt"]
    delta = w["beta"] / Nt
    seed = w["seed"] if seed is None else seed
    if w["start"] == "gaussian":
        return gaussian_field(seed, Nt, V, delta * w["U"])
    return np.zeros((Nt, V))
