"""Zero-momentum single-particle correlator from one M^{-1} source
(hmc_correlator_k0) against the oracle's dense solve and, at phi = 0, the
closed form with Fermi factors.  Tolerances: FP64 CG to 1e-12 -> C(t) to
1e-10 relative (norm over t); mixed CG to 1e-10 (FP64 true residual) ->
1e-8."""
import numpy as np
import pytest
import torch

from oracle import lattice, observables as obs, operators as ops
from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("prec,tol,bound", [(hmc.PREC_FP64, 1e-12, 1e-10),
                                            (hmc.PREC_MIXED, 1e-10, 1e-8)])
@pytest.mark.parametrize("L,Nt,mu", [(2, 6, 0.0), (3, 8, 0.0), (6, 16, 0.5)])
def test_correlator_matches_oracle(L, Nt, mu, prec, tol, bound):
    beta, U = 0.125 * Nt, 3.0
    V = 2 * L * L
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U, mu=mu))
    E = ops.transfer_matrix(lattice.hopping_matrix(L), delta, delta * mu)
    phi = synth.gaussian_field(L * 13 + Nt, Nt, V, delta * U, scale=0.5)
    C, st = c.correlator_k0(torch.from_numpy(phi).to(DEV), tol=tol, prec=prec)
    assert st.status == 0
    want = obs.correlator_k0(E, phi)
    got = C.cpu().numpy()
    assert np.linalg.norm(got - want) <= bound * np.linalg.norm(want)


def test_free_correlator_closed_form():
    L, Nt, beta = 6, 32, 4.0
    delta = beta / Nt
    c = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=3.0))
    C, st = c.correlator_k0(torch.zeros((Nt, 2 * L * L), dtype=torch.float64, device=DEV),
                            tol=1e-12)
    t = np.arange(Nt)
    want = 0.5 * sum(np.exp(t * delta * e) / (1.0 + np.exp(beta * e)) for e in (3.0, -3.0))
    assert st.status == 0
    assert np.allclose(C.cpu().numpy(), want, rtol=1e-10, atol=1e-13)
