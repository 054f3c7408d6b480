"""Checkpoint / resume of a GPU chain through the C ABI: a chain stopped
after two trajectories, saved, reloaded into a fresh context and continued
ends bit-identical to the uninterrupted chain, with identical logs."""
import numpy as np
import pytest
import torch

from paper_2210_06874_gb300 import chain, hmc, synth

pytestmark = pytest.mark.gpu


def test_gpu_chain_resume_is_bit_identical(tmp_path):
    w = synth.WORKLOADS["l3_nt8"]

    def ctx():
        return hmc.Context(hmc.Params(L=w["L"], Nt=w["Nt"], kappa=w["kappa"], U=w["U"],
                                      beta=w["beta"], n_md=w["n_md"],
                                      traj_length=w["traj_length"], cg_tol=w["cg_tol"]))

    phi0 = np.ascontiguousarray(synth.start_field("l3_nt8") * 0.5)
    whole = torch.from_numpy(phi0).to("cuda:0")
    recs = chain.run_chain(ctx(), whole, w["seed"], 0, 4)
    part = torch.from_numpy(phi0).to("cuda:0")
    ck = str(tmp_path / "chain.npz")
    first = chain.run_chain(ctx(), part, w["seed"], 0, 2, checkpoint=ck)
    phi, seed, nxt, cid = chain.load_checkpoint(ck, "cuda:0")
    second = chain.run_chain(ctx(), phi, seed, nxt, 2, chain=cid)
    assert torch.equal(phi, whole)
    strip = [{k: v for k, v in r.items() if k != "seconds"} for r in first + second]
    assert strip == [{k: v for k, v in r.items() if k != "seconds"} for r in recs]
    assert all(r["status"] == 0 for r in recs)
