"""The benchmark's N-GPU logic on CPU ranks (gloo, world size 2).

bench.py runs one independent replica of the workload per rank (the path has
no exchange step), takes the slowest rank's time with one all-reduce and
reports the whole-job throughput; the reference arm runs on rank 0 only.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [1.5, 2.0][rank]
    t = bench.max_over_ranks(seconds, world, "cpu")
    v = bench.replica_value(world, 10 ** 9, 4, t)

    class A:
        steps, warmup = 1, 0
    ref = bench.run_reference(A()) if rank == 1 else "skipped"  # rank 1 must return at once
    q.put((rank, t, v, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, ref in res:
        assert t == 2.0                           # max over ranks
        assert v == pytest.approx(2 * 4 * 1e9 / 2.0 / 1e9)
    assert res[1][3] is None                      # reference arm: rank 1 does no work
