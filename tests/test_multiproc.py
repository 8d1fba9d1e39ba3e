"""Multi-rank logic on CPU ranks (gloo): the benchmark's N-GPU timing and the
distributed permute's plan and exchange.

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


def _dist_worker(rank, world, port, q):
    """One rank of the distributed permute: the library's plan, the oracle
    for the pack and unpack permutes (the CPU stand-in for the kernels) and
    a gloo all-to-all for the exchange."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1011_3583_gb300 import build, librearr
    build.build()
    orc = oracle.get()
    ok = []
    for e, dims, perm in ((4, [6 * world, 5, 2 * world], [2, 0, 1]), (2, [4 * world, 3, world, 2], [2, 3, 0, 1]),
                          (8, [2 * world, 3 * world], [1, 0]), (4, [2 * world, 3, 4], [0, 2, 1])):
        glob = synth.random_elements(7, int(np.prod(dims)), e)
        want = orc.permute(glob, e, dims, perm)
        plan = librearr.dist_permute_plan(e, dims, perm, world)
        sb = plan.slab_bytes
        mine = glob[rank * sb:(rank + 1) * sb]
        if plan.exchange:
            send = torch.from_numpy(orc.permute(mine, e, *plan.pack()))
            recv = torch.empty_like(send)
            dist.all_to_all_single(recv, send)
            out = orc.permute(recv.numpy(), e, *plan.unpack())
        else:
            out = orc.permute(mine, e, *plan.pack())
        ok.append(bool(np.array_equal(out, want[rank * sb:(rank + 1) * sb])))
    q.put((rank, ok))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_permute_on_gloo_ranks(world):
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_dist_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok in res:
        assert all(ok), (rank, ok)
