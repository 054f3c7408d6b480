"""Markov-chain driver over hmc_trajectory: a per-trajectory log in JSON
lines and checkpoint / resume.

The state of a chain is (phi, seed, chain id, index of the next trajectory).
Momenta, pseudofermion noise and the Metropolis uniform come from the
counter-based generator keyed by the seed, with the trajectory index and the
chain id in the counter, so a chain resumed from a checkpoint repeats the
uninterrupted chain bit for bit.
"""
import json
import os
import time

import numpy as np
import torch

LOG_FIELDS = ("dH", "H0", "H1", "u", "accept", "cg_iterations", "cg_solves",
              "reliable_updates", "max_true_residual", "status")


def save_checkpoint(path, phi, seed, next_traj, chain=0):
    """Write the chain state to `path` (.npz), atomically (a temporary file
    renamed over the target)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, phi=phi.detach().cpu().numpy(), seed=np.uint64(seed),
             next_traj=np.int64(next_traj), chain=np.int64(chain))
    os.replace(tmp, path)


def load_checkpoint(path, device):
    """(phi on `device`, seed, next_traj, chain) from save_checkpoint's file."""
    with np.load(path) as z:
        phi = torch.from_numpy(np.ascontiguousarray(z["phi"])).to(device)
        return phi, int(z["seed"]), int(z["next_traj"]), int(z["chain"])


def run_chain(ctx, phi, seed, first_traj, n_traj, chain=0, log=None, checkpoint=None,
              every=1, allow_not_converged=False):
    """Advance phi (in place) by n_traj trajectories with indices first_traj,
    first_traj + 1, ...  Each trajectory appends one JSON line to `log` (an
    open text file, or None): its index, the fields of hmc_traj_out and the
    host wall time in seconds.  With `checkpoint` (a path) the state is
    saved every `every` trajectories and after the last one.  Returns the
    trajectories' records."""
    records = []
    last = first_traj + n_traj - 1
    for k in range(first_traj, first_traj + n_traj):
        t0 = time.perf_counter()
        out = ctx.trajectory(phi, seed, k, chain, allow_not_converged=allow_not_converged)
        rec = {"traj": k, "chain": chain}
        rec.update({f: getattr(out, f) for f in LOG_FIELDS})
        rec["seconds"] = time.perf_counter() - t0
        records.append(rec)
        if log is not None:
            log.write(json.dumps(rec) + "\n")
            log.flush()
        if checkpoint is not None and ((k - first_traj + 1) % every == 0 or k == last):
            save_checkpoint(checkpoint, phi, seed, k + 1, chain)
    return records
