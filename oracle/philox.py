"""Philox4x32-10 counter-based generator and the HMC draws made from it
(oracle; test infrastructure only).

Generator: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, the Philox-4x32 bijection with 10 rounds.  One round maps
counter (c0, c1, c2, c3) under key (k0, k1) to
    (hi(B*c2) ^ c1 ^ k0,  lo(B*c2),  hi(A*c0) ^ c3 ^ k1,  lo(A*c0))
with A = 0xD2511F53, B = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85).

Stream layout shared with the GPU library (each side implements it on its own):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (element e, stream id, trajectory index mod 2^32, chain id)
    u1 = ((x0 << 32 | x1) >> 11 + 0.5) * 2^-53        in (0, 1)
    u2 = ((x2 << 32 | x3) >> 11 + 0.5) * 2^-53
    Box-Muller: z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2)
Streams: 0 momenta pi_e = z0; 1 pseudofermion noise rho_e = (z0 + i z1)/sqrt(2)
(density exp(-rho^dag rho), §2); 2 the Metropolis uniform u1 of element 0;
3 the second pseudofermion's noise under mass preconditioning (as stream 1);
4 Z2 noise 1 - 2 (x0 & 1) of the stochastic trace estimates.
"""
import numpy as np

PHILOX_A = np.uint64(0xD2511F53)
PHILOX_B = np.uint64(0xCD9E8D57)
WEYL_0 = 0x9E3779B9
WEYL_1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_MOMENTUM = 0
STREAM_PSEUDOFERMION = 1
STREAM_METROPOLIS = 2
STREAM_HEAVY = 3          # second pseudofermion of mass preconditioning
STREAM_Z2 = 4             # Z2 noise of the stochastic trace estimates


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Counters: uint32-valued arrays (broadcast),
    key: two Python ints.  Returns four uint64 arrays holding uint32 values."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + WEYL_0) & 0xFFFFFFFF
            k1 = (k1 + WEYL_1) & 0xFFFFFFFF
        p0 = PHILOX_A * c0                      # < 2^64, exact in uint64
        p1 = PHILOX_B * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def _raw(seed, stream, traj, chain, n):
    e = np.arange(n, dtype=np.uint64)
    return philox4x32_10(e, stream, traj & 0xFFFFFFFF, chain,
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def uniform_pair(seed, stream, traj, chain, n):
    """(u1, u2) for elements 0..n-1, each in the open interval (0, 1)."""
    x0, x1, x2, x3 = _raw(seed, stream, traj, chain, n)
    a = ((x0 << np.uint64(32)) | x1) >> np.uint64(11)
    b = ((x2 << np.uint64(32)) | x3) >> np.uint64(11)
    scale = 2.0 ** -53
    return (a.astype(np.float64) + 0.5) * scale, (b.astype(np.float64) + 0.5) * scale


def normal_pair(seed, stream, traj, chain, n):
    """Box-Muller pair (z0, z1) per element, standard normal each."""
    u1, u2 = uniform_pair(seed, stream, traj, chain, n)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def momenta(seed, traj, chain, Nt, V):
    """pi ~ exp(-pi^2/2) on every (t, x) (§2)."""
    z0, _ = normal_pair(seed, STREAM_MOMENTUM, traj, chain, Nt * V)
    return z0.reshape(Nt, V)


def pseudofermion_noise(seed, traj, chain, Nt, V):
    """rho ~ exp(-rho^dag rho): real and imaginary parts N(0, 1/2) (§2)."""
    z0, z1 = normal_pair(seed, STREAM_PSEUDOFERMION, traj, chain, Nt * V)
    return ((z0 + 1j * z1) / np.sqrt(2.0)).reshape(Nt, V)


def metropolis_uniform(seed, traj, chain):
    u1, _ = uniform_pair(seed, STREAM_METROPOLIS, traj, chain, 1)
    return float(u1[0])
