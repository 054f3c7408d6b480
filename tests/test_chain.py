"""Host logic of the chain driver (paper_2210_06874_gb300/chain.py) on CPU:
the JSON-lines log and checkpoint / resume.  The context is a stand-in that
runs the oracle's trajectory on a CPU tensor with the same call signature as
the library's Context.trajectory (the GPU chain itself is covered by the
-m gpu trajectory tests)."""
import io
import json
import types

import numpy as np
import torch

from oracle import hmc as ohmc, lattice, operators as ops
from paper_2210_06874_gb300 import chain


class OracleContext:
    def __init__(self, L=2, Nt=4, beta=1.0, U=2.0, n_md=4):
        self.delta = beta / Nt
        self.U, self.n_md = U, n_md
        self.E = ops.transfer_matrix(lattice.hopping_matrix(L), self.delta)

    def trajectory(self, phi, seed, traj, chain_id=0, allow_not_converged=False):
        out = ohmc.trajectory(self.E, phi.numpy(), self.delta, self.U, 1.0 / self.n_md,
                              self.n_md, seed, traj, chain_id, tol=1e-12)
        phi.copy_(torch.from_numpy(out["phi"]))
        return types.SimpleNamespace(dH=out["dH"], H0=out["H0"], H1=out["H1"], u=out["u"],
                                     accept=int(out["accept"]), cg_iterations=out["cg_iters"],
                                     cg_solves=out["cg_solves"], reliable_updates=0,
                                     max_true_residual=0.0, status=0)


def start():
    rng = np.random.default_rng(4)
    return torch.from_numpy(0.5 * rng.normal(0.0, np.sqrt(0.5), size=(4, 8)))


def test_log_lines_hold_every_field():
    ctx = OracleContext()
    phi = start()
    log = io.StringIO()
    recs = chain.run_chain(ctx, phi, 31, 0, 3, chain=2, log=log)
    lines = [json.loads(s) for s in log.getvalue().splitlines()]
    assert lines == recs and [r["traj"] for r in lines] == [0, 1, 2]
    for r in lines:
        assert r["chain"] == 2 and r["seconds"] >= 0.0
        assert set(chain.LOG_FIELDS) <= set(r)


def test_resume_repeats_the_uninterrupted_chain(tmp_path):
    ctx = OracleContext()
    whole = start()
    recs_whole = chain.run_chain(ctx, whole, 31, 0, 6)
    ck = str(tmp_path / "chain.npz")
    part = start()
    first = chain.run_chain(ctx, part, 31, 0, 3, checkpoint=ck, every=2)
    phi, seed, nxt, cid = chain.load_checkpoint(ck, "cpu")
    assert (seed, nxt, cid) == (31, 3, 0) and torch.equal(phi, part)
    second = chain.run_chain(ctx, phi, seed, nxt, 3, chain=cid)
    assert torch.equal(phi, whole)
    strip = [{k: v for k, v in r.items() if k != "seconds"} for r in first + second]
    assert strip == [{k: v for k, v in r.items() if k != "seconds"} for r in recs_whole]
