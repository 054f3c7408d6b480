"""bench.py's multi-GPU path is replicas only: every rank advances its own
chain (chain id = rank) and the whole-job rate is all ranks' units over the
slowest rank's time.  Checked with two gloo ranks on CPU."""
import os
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 1000.0 if rank == 0 else 2500.0        # rank 1 is the slow one
    rate, ms = bench.aggregate_rate(local_ms, 10, world, dist, torch.device("cpu"))
    # the Philox chain id of a replica is its rank: streams are disjoint
    from oracle import philox
    z = philox.momenta(123, 0, rank, 2, 3)
    zs = [torch.zeros(6, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(zs, torch.from_numpy(z.ravel()))
    q.put((rank, rate, ms, not torch.equal(zs[0], zs[1])))
    dist.destroy_process_group()


def test_replica_rate_two_ranks():
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms, distinct in res:
        assert ms == 2500.0                      # max over ranks
        assert abs(rate - 2 * 10 / 2.5) < 1e-12  # all ranks' units / slowest time
        assert distinct


def _chain_worker(rank, world, port, q):
    """One replica: the l3_nt8 chain of this rank (chain id = rank) advanced
    by two oracle trajectories, timed; the job's rate is reduced over ranks
    as bench.py does.  No collective touches the fields."""
    sys.path.insert(0, ROOT)
    import time
    import numpy as np
    import bench
    from oracle import hmc as ohmc, lattice, operators as ops
    from paper_2210_06874_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.WORKLOADS["l3_nt8"]
    delta = w["beta"] / w["Nt"]
    E = ops.transfer_matrix(lattice.hopping_matrix(w["L"]), delta * w["kappa"])
    phi = synth.start_field("l3_nt8")
    t0 = time.perf_counter()
    dHs = []
    for traj in range(2):
        r = ohmc.trajectory(E, phi, delta, w["U"], w["traj_length"] / w["n_md"], w["n_md"],
                            w["seed"], traj, rank, tol=w["cg_tol"], max_iter=100000)
        phi = r["phi"]
        dHs.append(r["dH"])
    ms = (time.perf_counter() - t0) * 1e3
    rate, ms_max = bench.aggregate_rate(ms, 2, world, dist, torch.device("cpu"))
    q.put((rank, float(np.sum(phi)), dHs, rate, ms, ms_max))
    dist.destroy_process_group()


def test_replica_chains_two_ranks():
    """Two gloo ranks each run their own chain: the chains differ (distinct
    Philox chain ids), every rank gets the same whole-job rate, which is 4
    trajectories over the slower rank's time."""
    port = 30500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_chain_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, d0, rate0, ms0, mx0), (r1, s1, d1, rate1, ms1, mx1) = res
    assert s0 != s1 and d0 != d1
    assert mx0 == mx1 == max(ms0, ms1)
    assert abs(rate0 - rate1) < 1e-9 and abs(rate0 - 4 / (mx0 * 1e-3)) < 1e-9
