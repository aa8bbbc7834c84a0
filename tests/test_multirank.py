"""The N > 1 launch path on CPU: two gloo ranks run the benchmark's host-side multi-rank logic
(max over ranks of the timed region, whole-job rate of independent replicas, per-rank seeds)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, HERE)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    total_ms = 100.0 + 25.0 * rank                 # the slower rank sets the job's time
    tmax = bench.reduce_max(total_ms, dist, world, "cpu")
    rate = bench.whole_job_rate(world, 1000.0, 10, tmax)
    seeds = [bench.replica_seed(rank, k) for k in range(5)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (r, w, tmax, rate, gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_rate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, tmax, rate, gathered = res[rank]
        assert r == rank and w == world
        assert tmax == 125.0                              # max over ranks
        assert rate == world * 1000.0 * 10 / 0.125        # both replicas' work / slowest time
        # replicas draw different inputs
        assert set(gathered[0]).isdisjoint(gathered[1])
