"""hmc_cg_solve_noalloc: the FP64 CG for callers that may not allocate device
memory (hosts whose device memory comes from a framework pool or a fixed
budget, plugins barred from growing the heap).  It must give the result of
hmc_cg_solve with HMC_PREC_FP64, call after call, while its scratch sits in
the library's static device array; on a stream under graph capture it must
refuse before enqueuing anything.  Collected last on purpose."""
import pytest
import torch

from paper_2210_06874_gb300 import hmc, synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("L,Nt,beta,U", [(3, 8, 2.0, 2.0), (6, 32, 4.0, 3.5), (5, 13, 1.6, 3.0)])
def test_noalloc_matches_cg_solve_twice(L, Nt, beta, U):
    V = 2 * L * L
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=beta, U=U))
    E = ctx.transfer_matrix().to(DEV)
    phi = torch.from_numpy(synth.gaussian_field(41, Nt, V, beta / Nt * U, scale=0.5)).to(DEV)
    chi = torch.from_numpy(synth.complex_gaussian(42, Nt, V)).to(DEV)
    want, st_want = ctx.cg_solve(phi, chi, tol=1e-12, prec=hmc.PREC_FP64)
    for _ in range(2):                       # two calls in a row share the scratch
        x = torch.full_like(chi, complex(float("nan"), 0.0))
        code, st = hmc.cg_solve_noalloc(E, L, Nt, phi, chi, x, 1e-12, 100000)
        torch.cuda.synchronize()
        assert code == hmc.HMC_OK, code
        assert st.status == hmc.HMC_OK
        assert st.true_residual < 1e-11
        assert abs(st.iterations - st_want.iterations) <= 1
        err = torch.linalg.vector_norm(x - want) / torch.linalg.vector_norm(want)
        assert err.item() < 1e-10


def test_noalloc_rejects_oversize():
    L, Nt = 24, 96                           # V * Nt = 110592 > 32768
    V = 2 * L * L
    E = torch.zeros((V, V), dtype=torch.float64, device=DEV)
    phi = torch.zeros((Nt, V), dtype=torch.float64, device=DEV)
    chi = torch.zeros((Nt, V), dtype=torch.complex128, device=DEV)
    x = torch.zeros_like(chi)
    code, _ = hmc.cg_solve_noalloc(E, L, Nt, phi, chi, x, 1e-10, 10)
    assert code == hmc.HMC_ERR_UNSUPPORTED


def test_noalloc_refuses_graph_capture():
    """The call synchronises and reads its result on the host, so it cannot
    be captured: under capture it returns HMC_ERR_UNSUPPORTED and leaves the
    capture valid (the work captured around it replays)."""
    L, Nt = 3, 8
    V = 2 * L * L
    ctx = hmc.Context(hmc.Params(L=L, Nt=Nt, beta=2.0, U=2.0))
    E = ctx.transfer_matrix().to(DEV)
    phi = torch.from_numpy(synth.gaussian_field(43, Nt, V, 0.5, scale=0.5)).to(DEV)
    chi = torch.from_numpy(synth.complex_gaussian(44, Nt, V)).to(DEV)
    x = torch.zeros_like(chi)
    code, _ = hmc.cg_solve_noalloc(E, L, Nt, phi, chi, x, 1e-12, 100000)   # set-up, uncaptured
    assert code == hmc.HMC_OK
    y = torch.zeros(4, device=DEV)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        y.add_(1.0)
        code, st = hmc.cg_solve_noalloc(E, L, Nt, phi, chi, x, 1e-12, 100000)
        y.add_(2.0)
    assert code == hmc.HMC_ERR_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, torch.full_like(y, 3.0))
