"""Slice-major tensor-core tiles (operand_mode 4): 64 time slices x {re, im}
as the MMA's M = 128 and up to 288 sites as its N, one FP32 accumulator of
the 2^eE-scaled FP16 split of E, against the FP64 oracle.

Tolerances, from the arithmetic: the split keeps 22 bits of E and of the
power-of-two scaled vector (the plain fp16 remainder of a value below 2^15
is exact to 2^-24 absolute, far below the 2^-22 relative of the split),
products are exact in FP32 and summed in FP32, so one application is
accurate to a few 1e-7 relative (normwise; tested at 2e-6 like the
site-major tile); the solver must reach the FP64 true residual 1e-10 and a
trajectory the oracle's Delta H within 1e-7.  Covered: one and several site
tiles (V up to 288 in one tile, above it tiles of 288 or 144 with a ragged
last tile), one and several slice tiles (ragged), one CTA and teams.
"""
import numpy as np
import pytest
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
APPLY_TOL = 2e-6


def oracle_E(L, Nt, beta, kappa=1.0):
    return ops.transfer_matrix(lattice.hopping_matrix(L), beta / Nt * kappa)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype else t).to(DEV)


# (L, Nt, tile_slices): V from 2 to 1152; 0 = automatic slices per tile
APPLY = [(1, 1, 0), (1, 3, 0), (2, 5, 0), (3, 8, 0), (5, 13, 0), (6, 32, 0), (7, 9, 0),
         (9, 48, 0), (12, 64, 0), (13, 20, 0), (12, 64, 64), (9, 70, 64), (6, 33, 5),
         (24, 96, 0)]


@pytest.mark.parametrize("L,Nt,ns", APPLY)
def test_apply_slice_major(L, Nt, ns):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, operand_mode=4, tile_slices=ns))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(L * 100 + Nt, Nt, V, beta / Nt * U)
    psi = dev(synth.complex_gaussian(L * 1000 + Nt, Nt, V), torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)
    got = c.apply_M(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    assert rel(got, ops.apply_M(E, phi, psi_in)) < APPLY_TOL
    got = c.apply_Mdag(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
    assert rel(got, ops.apply_Mdag(E, phi, psi_in)) < APPLY_TOL


def test_apply_slice_major_scale_and_zero():
    """Per-slice power-of-two scales: tiny, huge and zero slices in one vector."""
    L, Nt = 6, 8
    V = 72
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=1.0, U=3.0, operand_mode=4))
    E = oracle_E(L, Nt, 1.0)
    phi = synth.gaussian_field(1, Nt, V, 0.3)
    psi64 = synth.complex_gaussian(2, Nt, V)
    psi64[1] *= 1e-30
    psi64[2] *= 1e30
    psi64[5] = 0.0
    psi = dev(psi64, torch.complex64)
    psi_in = psi.cpu().numpy().astype(np.complex128)
    for dag, op in ((False, ops.apply_M), (True, ops.apply_Mdag)):
        fn = c.apply_Mdag if dag else c.apply_M
        got = fn(dev(phi), psi, prec=hmc.PREC_MIXED).cpu().numpy()
        want = op(E, phi, psi_in)
        for t in range(Nt):       # slice by slice: each has its own scale
            if np.linalg.norm(want[t]) > 0:
                assert rel(got[t], want[t]) < APPLY_TOL, (dag, t)
    zero = torch.zeros((Nt, V), dtype=torch.complex64, device=DEV)
    assert torch.count_nonzero(c.apply_M(dev(phi), zero, prec=hmc.PREC_MIXED)) == 0


# (L, Nt, beta, U, team_ctas, inner_ctas, tile_slices)
CG = [(1, 2, 1.0, 2.0, 0, 0, 0), (3, 8, 2.0, 2.0, 0, 0, 0), (6, 32, 4.0, 3.5, 0, 0, 0),
      (9, 16, 2.0, 3.0, 0, 0, 0), (12, 64, 8.0, 3.8, 0, 0, 0), (13, 20, 2.5, 3.0, 0, 0, 0),
      (5, 70, 8.75, 3.0, 0, 0, 0), (12, 64, 8.0, 3.8, 8, 4, 16), (6, 32, 4.0, 3.5, 4, 3, 7),
      (24, 96, 12.0, 4.0, 0, 0, 0)]


@pytest.mark.parametrize("L,Nt,beta,U,team,inner,ns", CG)
def test_cg_slice_major_reaches_fp64_residual(L, Nt, beta, U, team, inner, ns):
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, operand_mode=4, team_ctas=team,
                               inner_ctas=inner, tile_slices=ns))
    E = oracle_E(L, Nt, beta)
    phi = synth.gaussian_field(11, Nt, V, beta / Nt * U, scale=0.5)
    chi = synth.complex_gaussian(12, Nt, V)
    x, st = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_MIXED)
    assert st.status == 0
    assert st.true_residual <= 1e-10
    assert st.reliable_updates >= 1
    res = chi - ops.apply_MMdag(E, phi, x.cpu().numpy())
    assert np.linalg.norm(res) / np.linalg.norm(chi) < 1.2e-10
    _, st64 = c.cg_solve(dev(phi), dev(chi), tol=1e-10, prec=hmc.PREC_FP64)
    assert st.iterations < 3 * st64.iterations + 20


def test_cg_slice_major_deterministic():
    L, Nt = 12, 64
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=8.0, U=3.8, operand_mode=4))
    phi = dev(synth.gaussian_field(3, Nt, V, 0.475, scale=0.5))
    chi = dev(synth.complex_gaussian(4, Nt, V))
    x1, s1 = c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    x2, s2 = c.cg_solve(phi, chi, tol=1e-10, prec=hmc.PREC_MIXED)
    assert s1.iterations == s2.iterations
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("L,Nt,beta,U,n_md", [(3, 8, 2.0, 2.0, 10), (6, 32, 4.0, 3.5, 3)])
def test_trajectory_slice_major_matches_oracle(L, Nt, beta, U, n_md):
    delta = beta / Nt
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, U=U, beta=beta, n_md=n_md, traj_length=0.3,
                               cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=4))
    E = oracle_E(L, Nt, beta)
    phi_np = synth.gaussian_field(5, Nt, V, delta * U, scale=0.5)
    phi = dev(phi_np)
    for traj in range(2):
        want = ohmc.trajectory(E, phi_np, delta, U, 0.3 / n_md, n_md, 77, traj, 0, tol=1e-12)
        out = c.trajectory(phi, 77, traj)
        assert out.status == 0
        assert out.max_true_residual <= 1e-10
        assert abs(out.dH - want["dH"]) < 1e-7
        assert bool(out.accept) == want["accept"]
        assert rel(phi.cpu().numpy(), want["phi"]) < 1e-8
        phi_np = want["phi"]


# uneven chains, slice-major tiles mixed with site-major and CUDA-core ones
BATCH = [(3, 8, 2.0, 4), (9, 16, 3.0, 4), (6, 16, 3.5, 3), (12, 16, 3.0, 4), (2, 5, 3.0, 4),
         (6, 8, 5.0, 1)]


def bparams(L, Nt, U, mode, **kw):
    return hmc.Params(L=L, Nt=Nt, U=U, beta=0.25 * Nt, n_md=3, traj_length=0.3,
                      cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=mode, **kw)


def test_batch_slice_major_matches_single_chains_and_oracle():
    b = hmc.Batch([bparams(*c) for c in BATCH])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = [synth.gaussian_field(20 + i, Nt, 2 * L * L, 0.25 * U, scale=0.5)
              for i, (L, Nt, U, _) in enumerate(BATCH)]
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    outs = b.trajectory(phi, 31, 0)
    for i, (L, Nt, U, mode) in enumerate(BATCH):
        single = hmc.Context(bparams(L, Nt, U, mode, team_ctas=1, inner_ctas=1))
        sphi = torch.from_numpy(fields[i]).to(DEV)
        o = single.trajectory(sphi, 31, 0, chain=i)
        assert outs[i].status == 0 and o.status == 0
        assert outs[i].dH == o.dH, (i, outs[i].dH, o.dH)     # same arithmetic, bitwise
        assert torch.equal(b.view(phi, i), sphi)
        p = bparams(L, Nt, U, mode)
        E = ops.transfer_matrix(lattice.hopping_matrix(L), p.delta)
        want = ohmc.trajectory(E, fields[i], p.delta, U, p.traj_length / p.n_md, p.n_md, 31, 0,
                               chain=i, tol=1e-12)
        assert outs[i].max_true_residual <= 1e-10
        assert abs(outs[i].dH - want["dH"]) < 1e-7
        assert bool(outs[i].accept) == want["accept"]


def test_apply_slice_major_split_k_deterministic():
    """Standalone applications split each tile's K over a cluster and sum
    the partials in rank order: repeated applications are bitwise equal
    (L = 24: 18 K chunks over 8 CTAs, ragged)."""
    L, Nt = 24, 96
    V = 2 * L * L
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=12.0, U=4.0, operand_mode=4))
    phi = dev(synth.gaussian_field(8, Nt, V, 0.5))
    psi = dev(synth.complex_gaussian(9, Nt, V), torch.complex64)
    a = c.apply_Mdag(phi, psi, prec=hmc.PREC_MIXED)
    b = c.apply_Mdag(phi, psi, prec=hmc.PREC_MIXED)
    assert torch.equal(a, b)


def test_batch_reuses_ctas_across_tile_widths():
    """More chains than CTAs, of four tile widths (W = 16, 32, 80, 176: ring
    depths 4, 4, 4, 2), so CTAs run several slice-major chains one after the
    other: every chain converges and matches its single-chain run bitwise."""
    n = 2 * torch.cuda.get_device_properties(0).multi_processor_count + 8
    Ls = [2, 3, 6, 9]
    chains = [(Ls[i % 4], 4 + (i % 3), 2.0 + 0.004 * i) for i in range(n)]

    def p(L, Nt, U, **kw):
        return hmc.Params(L=L, Nt=Nt, U=U, beta=0.125 * Nt, n_md=2, traj_length=0.2,
                          cg_tol=1e-10, precision=hmc.PREC_MIXED, operand_mode=4, **kw)
    b = hmc.Batch([p(*c) for c in chains])
    phi = torch.zeros(b.total, dtype=torch.float64, device=DEV)
    fields = [synth.gaussian_field(500 + i, Nt, 2 * L * L, 0.125 * U, scale=0.5)
              for i, (L, Nt, U) in enumerate(chains)]
    for i, f in enumerate(fields):
        b.view(phi, i).copy_(torch.from_numpy(f))
    outs = b.trajectory(phi, 3, 0)
    assert all(o.status == 0 for o in outs)
    assert all(o.max_true_residual <= 1e-10 for o in outs)
    for i in list(range(0, n, 37)) + [n - 1]:
        L, Nt, U = chains[i]
        single = hmc.Context(p(L, Nt, U, team_ctas=1, inner_ctas=1))
        sphi = torch.from_numpy(fields[i]).to(DEV)
        o = single.trajectory(sphi, 3, 0, chain=i)
        assert outs[i].dH == o.dH, (i, outs[i].dH, o.dH)
        assert torch.equal(b.view(phi, i), sphi)
