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
