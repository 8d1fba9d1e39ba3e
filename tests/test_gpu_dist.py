"""Distributed permute (include/librearr_dist.h) on the GPU: P ranks emulated
on one device (every rank's pack and unpack run through the library; the
all-to-all is done by device copies of the pieces), and the torch.distributed
path (dist_permute) over NCCL with one rank.  Results must equal the oracle's
permute of the whole array, byte for byte."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build, librearr
    build.build()
    librearr.load()
    return librearr


def emulate(lr, glob, e, dims, perm, nranks):
    """Every rank's output slab (concatenated), from a device copy of glob."""
    import torch
    x = torch.from_numpy(glob).cuda()
    plan = lr.dist_permute_plan(e, dims, perm, nranks)
    sb, pb = plan.slab_bytes, plan.piece_bytes
    out = torch.full_like(x, 0x5A)
    if not plan.exchange:
        for r in range(nranks):
            lr.dist_permute_pack(out[r * sb:(r + 1) * sb], x[r * sb:(r + 1) * sb], plan, e)
    else:
        send, recv = torch.full_like(x, 0x11), torch.full_like(x, 0x22)
        for r in range(nranks):
            lr.dist_permute_pack(send[r * sb:(r + 1) * sb], x[r * sb:(r + 1) * sb], plan, e)
        torch.cuda.synchronize()
        for r in range(nranks):  # the all-to-all: piece r of every sender
            recv[r * sb:(r + 1) * sb] = torch.cat([send[j * sb + r * pb:j * sb + (r + 1) * pb] for j in range(nranks)])
        for r in range(nranks):
            lr.dist_permute_unpack(out[r * sb:(r + 1) * sb], recv[r * sb:(r + 1) * sb], plan, e)
    torch.cuda.synchronize()
    return out.cpu().numpy(), plan


CASES = [  # (elem_bytes, dims, perm, nranks)
    (4, [8, 6, 4], [2, 0, 1], 2),
    (4, [8, 6, 4], [0, 2, 1], 2),
    (8, [6, 6], [1, 0], 3),
    (2, [12, 5, 8, 3], [2, 0, 3, 1], 4),
    (1, [16, 4, 4, 2, 3], [2, 4, 0, 3, 1], 2),
    (12, [4, 9, 8], [2, 1, 0], 4),
    (4, [256, 96, 64], [2, 0, 1], 4),       # tiled planes
    (4, [1024, 1024], [1, 0], 8),           # 2-D transpose over 8 ranks
    (2, [64, 128, 256, 8], [0, 1, 3, 2], 4),  # the sharded axis stays: local only
    (8, [120, 40, 36], [1, 2, 0], 5),       # ragged tiles
    (16, [32, 3, 64], [2, 1, 0], 2),
]


@pytest.mark.parametrize("e,dims,perm,nranks", CASES)
def test_emulated_ranks_match_oracle(lr, e, dims, perm, nranks):
    orc = oracle.get()
    glob = synth.random_elements(sum(dims) + nranks, int(np.prod(dims)), e)
    got, plan = emulate(lr, glob, e, dims, perm, nranks)
    assert plan.exchange == (perm[0] != 0)
    assert np.array_equal(got, orc.permute(glob, e, dims, perm)), (e, dims, perm, nranks)


def test_table1_cube_over_4_ranks_sampled(lr):
    """512^3 fp32 (512 MiB) reversed over 4 emulated ranks: outputs sampled at
    the slab seams, the ends and at random positions."""
    orc = oracle.get()
    dims, perm, e, nranks = [512, 512, 512], [2, 1, 0], 4, 4
    n = 512 ** 3
    glob = synth.random_elements(99, n, e)
    got, plan = emulate(lr, glob, e, dims, perm, nranks)
    slab = n // nranks
    lin = np.unique(np.concatenate([np.arange(0, 64), np.arange(n - 64, n),
                                    *[np.arange(r * slab - 32, r * slab + 32) for r in range(1, nranks)],
                                    np.random.default_rng(3).integers(0, n, 8192)])).astype(np.int64)
    want = orc.permute_sample(glob, e, dims, perm, lin)
    got_s = got.reshape(-1, e)[lin].reshape(-1)
    assert np.array_equal(got_s, want)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_dist_permute_over_nccl_one_rank(lr):
    """dist_permute end to end through torch.distributed (NCCL, world size 1):
    pack, all_to_all_single and unpack on the current stream."""
    import torch
    import torch.distributed as dist
    import paper_1011_3583_gb300 as rr
    orc = oracle.get()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        for e, dims, perm in ((4, [64, 48, 32], [2, 0, 1]), (4, [64, 48, 32], [0, 2, 1]), (8, [300, 200], [1, 0])):
            glob = synth.random_elements(5, int(np.prod(dims)), e)
            x = torch.from_numpy(glob).cuda()
            y = torch.empty_like(x)
            plan = rr.dist_permute(y, x, e, dims, perm)
            torch.cuda.synchronize()
            assert plan.exchange == (perm[0] != 0)
            assert np.array_equal(y.cpu().numpy(), orc.permute(glob, e, dims, perm)), (e, dims, perm)
        with pytest.raises(ValueError):
            rr.dist_permute(torch.empty(16, dtype=torch.uint8), torch.empty(16, dtype=torch.uint8), 4, [2, 2], [1, 0])
    finally:
        dist.destroy_process_group()
