"""Pins of the oracle's Philox4x32-10 generator and the draws built on it."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def load_kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([int(v, 16) for v in line.split()])
    return rows


def test_known_answer_vectors():
    rows = load_kat()
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(v) for v in out] == r[6:10]


def test_vectorised_matches_scalar():
    e = np.arange(7)
    vec = philox.philox4x32_10(e, 1, 2, 3, 0x1234, 0x5678)
    for i in range(7):
        one = philox.philox4x32_10(i, 1, 2, 3, 0x1234, 0x5678)
        assert [int(v[i]) for v in vec] == [int(v) for v in one]


def test_uniform_range_and_normal_moments():
    u1, u2 = philox.uniform_pair(42, 0, 0, 0, 200000)
    assert (u1 > 0).all() and (u1 < 1).all() and (u2 > 0).all() and (u2 < 1).all()
    z0, z1 = philox.normal_pair(42, 1, 3, 0, 200000)
    for z in (z0, z1):
        assert abs(z.mean()) < 0.01
        assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z0 * z1)) < 0.01


def test_streams_and_noise_normalisation():
    rho = philox.pseudofermion_noise(7, 0, 0, 64, 1000)
    # e^{-rho^dag rho}: <|rho|^2> = 1 per component
    assert abs(np.mean(np.abs(rho) ** 2) - 1.0) < 0.01
    a = philox.momenta(7, 0, 0, 4, 5)
    b = philox.momenta(7, 1, 0, 4, 5)
    c = philox.momenta(7, 0, 1, 4, 5)
    assert not np.allclose(a, b) and not np.allclose(a, c)
    assert np.array_equal(a, philox.momenta(7, 0, 0, 4, 5))
