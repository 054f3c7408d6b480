"""GPU parity of the printed operator Eq. (2.2) (mixed differencing) and its
adjoint against the oracle: FP64 to 1e-13, FP32 to 1e-6 (single rounding of
a handful of terms)."""
import numpy as np
import pytest
import torch

from oracle import operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("L,Nt", [(1, 1), (1, 4), (2, 3), (3, 8), (5, 13), (6, 32), (12, 16)])
@pytest.mark.parametrize("dagger", [False, True])
def test_brs_fp64_and_fp32(L, Nt, dagger):
    V = 2 * L * L
    beta, kappa = 0.125 * Nt, 1.0
    dk = beta / Nt * kappa
    phi = synth.gaussian_field(L * 7 + Nt, Nt, V, 0.4)
    psi = synth.complex_gaussian(L * 11 + Nt, Nt, V)
    f = ops.apply_Mdag_brs if dagger else ops.apply_M_brs
    want = f(L, phi, psi, beta / Nt, kappa)
    c64, c32 = hmc.brs_phases(L, Nt, torch.from_numpy(phi).to(DEV))
    got = hmc.apply_brs(L, Nt, dk, c64, torch.from_numpy(psi).to(DEV), dagger=dagger)
    assert rel(got.cpu().numpy(), want) < 1e-13
    p32 = torch.from_numpy(psi).to(DEV).to(torch.complex64)
    got32 = hmc.apply_brs(L, Nt, dk, c32, p32, dagger=dagger)
    want32 = f(L, phi, p32.cpu().numpy().astype(np.complex128), beta / Nt, kappa)
    assert rel(got32.cpu().numpy(), want32) < 1e-6


def test_brs_adjoint_identity_large():
    """L = 48 (the dense oracle is too large): <u, M v> = <M^dag u, v> on the GPU
    and sampled rows of M v recomputed from the equation."""
    L, Nt = 48, 32
    V = 2 * L * L
    dk = 0.125
    phi = torch.from_numpy(synth.gaussian_field(3, Nt, V, 0.4)).to(DEV)
    u = torch.from_numpy(synth.complex_gaussian(4, Nt, V)).to(DEV)
    v = torch.from_numpy(synth.complex_gaussian(5, Nt, V)).to(DEV)
    c64, _ = hmc.brs_phases(L, Nt, phi)
    Mv = hmc.apply_brs(L, Nt, dk, c64, v)
    Mdu = hmc.apply_brs(L, Nt, dk, c64, u, dagger=True)
    lhs = torch.vdot(u.flatten(), Mv.flatten()).item()
    rhs = torch.vdot(Mdu.flatten(), v.flatten()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # sampled entries from Eq. (2.2) directly
    ph, vn, Mvn = phi.cpu().numpy(), v.cpu().numpy(), Mv.cpu().numpy()
    rng = np.random.default_rng(0)
    for _ in range(50):
        t, x = int(rng.integers(Nt)), int(rng.integers(V))
        s, c = divmod(x, L * L)
        m1, m2 = divmod(c, L)
        if s == 0:
            nbs = [L * L + c, L * L + ((m1 - 1) % L) * L + m2, L * L + m1 * L + (m2 - 1) % L]
            fwd = vn[(t + 1) % Nt, x] * (-1 if t + 1 == Nt else 1)
            want = fwd - np.exp(1j * ph[t, x]) * vn[t, x]
        else:
            nbs = [c, ((m1 + 1) % L) * L + m2, m1 * L + (m2 + 1) % L]
            bwd = vn[(t - 1) % Nt, x] * (-1 if t == 0 else 1)
            want = vn[t, x] - np.exp(-1j * ph[t, x]) * bwd
        want -= dk * sum(vn[t, y] for y in nbs)
        assert abs(Mvn[t, x] - want) < 1e-12 * (1 + abs(want))


@pytest.mark.parametrize("L,Nt", [(2, 5), (48, 32), (102, 8)])
@pytest.mark.parametrize("dagger", [False, True])
def test_brs_fp32_pairs_vs_fp64(L, Nt, dagger):
    """Even L takes the paired FP32 kernel (two sites per 16-byte access);
    against the FP64 kernel (itself pinned to the oracle above) it agrees to
    single-precision rounding, at sizes the dense oracle cannot reach."""
    V = 2 * L * L
    dk = 0.125
    phi = torch.from_numpy(synth.gaussian_field(L + 21, Nt, V, 0.4)).to(DEV)
    psi = torch.from_numpy(synth.complex_gaussian(L + 22, Nt, V)).to(DEV)
    c64, c32 = hmc.brs_phases(L, Nt, phi)
    p32 = psi.to(torch.complex64)
    want = hmc.apply_brs(L, Nt, dk, c64, p32.to(torch.complex128), dagger=dagger)
    got = hmc.apply_brs(L, Nt, dk, c32, p32, dagger=dagger)
    assert rel(got.cpu().numpy(), want.cpu().numpy()) < 1e-6


def test_brs_fp32_unaligned_buffers():
    """Buffers 8 bytes off a 16-byte boundary take the one-site kernel and give
    the same result as aligned ones."""
    L, Nt = 6, 8
    V = 2 * L * L
    N = Nt * V
    phi = torch.from_numpy(synth.gaussian_field(31, Nt, V, 0.4)).to(DEV)
    psi = torch.from_numpy(synth.complex_gaussian(32, Nt, V)).to(DEV).to(torch.complex64)
    _, c32 = hmc.brs_phases(L, Nt, phi)
    base = hmc.apply_brs(L, Nt, 0.125, c32, psi)
    cb = torch.empty(N + 1, dtype=torch.complex64, device=DEV)
    pb = torch.empty(N + 1, dtype=torch.complex64, device=DEV)
    ob = torch.empty(N + 1, dtype=torch.complex64, device=DEV)
    cu, pu, ou = cb[1:].view(Nt, V), pb[1:].view(Nt, V), ob[1:].view(Nt, V)
    cu.copy_(c32)
    pu.copy_(psi)
    hmc.apply_brs(L, Nt, 0.125, cu, pu, out=ou)
    assert rel(ou.cpu().numpy(), base.cpu().numpy()) < 1e-6
