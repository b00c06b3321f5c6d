"""Host logic of bench.py's multi-rank path on CPU (gloo, world size 2):
every rank advances its own replica (weak scaling, no collective on the data
path); the timed region is the slowest rank's, taken with a max-reduce."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2510_18688_gb300 import workloads as W
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    cfg, arr = W.sessile_droplet(64, seed=rank, radius=12.0)
    q.put((rank, t, float(cfg["theta_deg"]), float(arr["phi"].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] != out[1][2]  # each rank's replica is seeded by its rank


def test_whole_job_throughput_is_the_sum_over_ranks():
    import bench
    one = bench.whole_job_mlups(262144, 1, 100, 3.3)
    assert bench.whole_job_mlups(262144, 4, 100, 3.3) == pytest.approx(4 * one)
    assert bench.max_over_ranks(2.5, None) == 2.5
