"""bench.py's multi-rank path on CPU: two gloo ranks (replicas), the max over ranks of
the timed region and the whole-job throughput built from it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slow = bench.max_reduce(dist, 100.0 + 50.0 * rank, device="cpu")   # rank 1 is slower
    val = bench.whole_job_mpix_s(world, 10, 1920 * 1080, slow)
    q.put((rank, slow, val, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, val, env in out:
        assert slow == 150.0
        assert val == pytest.approx(2 * 10 * 1920 * 1080 / 0.150 / 1e6)
        assert env == (rank, world, 0)
