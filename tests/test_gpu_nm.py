"""N-to-M reorder (Sec. III.B base index and range) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, DevPool, sync, to_dev
from tests.oracle_pins import random_box

pytestmark = pytest.mark.gpu

ELEMS = (1, 2, 3, 4, 8, 12, 16)


@pytest.fixture(scope="module")
def lr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build, librearr
    build.build()
    librearr.load()
    return librearr


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


def check_nm(lr, orc, seed, e, dims, order, base, rng, src_off=0, dst_off=0):
    n = int(np.prod(dims))
    total = int(np.prod([rng[a] for a in order]))
    src = synth.random_elements(seed, n, e)
    s = to_dev(src, src_off)
    d = DevBuf(total * e, dst_off, fill=0x77)
    lr.reorder_nm(d.ptr, s.ptr, e, dims, order, base, rng)
    sync()
    want = orc.reorder_nm(src, e, dims, order, base, rng)
    got = d.download()
    assert np.array_equal(got, want), (dims, order, base, rng, e, src_off, dst_off)


def test_nm_random_boxes(lr, orc):
    g = synth.rng(55)
    for t in range(150):
        rank_in = int(g.integers(1, 8))
        dims, order, base, rng = random_box(g, rank_in, max_extent=40 if rank_in <= 3 else 9)
        e = ELEMS[t % len(ELEMS)]
        check_nm(lr, orc, 300 + t, e, dims, order, base, rng)


def test_nm_special_cases(lr, orc):
    # the full box with every axis kept is the permute
    check_nm(lr, orc, 1, 4, [33, 70, 65], [2, 0, 1], [0, 0, 0], [33, 70, 65])
    # rank-1 range copy ("specified range" access)
    check_nm(lr, orc, 2, 4, [100003], [0], [517], [90001])
    # the input's fastest axis dropped: no contiguous axis, each element gathered on its own
    check_nm(lr, orc, 3, 4, [40, 50, 60], [1, 0], [3, 7, 11], [30, 40, 0])
    # inner axis kept but sliced: short runs of the kept part
    check_nm(lr, orc, 4, 2, [64, 80, 96], [0, 1, 2], [5, 6, 7], [50, 60, 70])
    check_nm(lr, orc, 5, 8, [64, 80, 96], [2, 0, 1], [5, 6, 7], [50, 60, 80])
    # aligned sub-boxes take the vectorised tile path
    check_nm(lr, orc, 6, 4, [8, 256, 512], [2, 1], [3, 64, 128], [0, 128, 256])
    check_nm(lr, orc, 7, 1, [8, 256, 512], [2, 1], [3, 64, 128], [0, 128, 256])
    # unaligned pointers
    check_nm(lr, orc, 8, 4, [8, 256, 512], [2, 1], [3, 64, 128], [0, 128, 256], src_off=4, dst_off=8)
    check_nm(lr, orc, 9, 2, [30, 70, 90], [1, 2, 0], [1, 2, 3], [20, 60, 80], src_off=2, dst_off=6)
    # empty box: no launch
    before = lr.launch_count()
    lr.reorder_nm(0, 0, 4, [10, 10], [1, 0], [3, 4], [0, 5])
    assert lr.launch_count() == before


def test_nm_rejects_invalid(lr):
    fake_src, fake_dst = 1 << 40, 1 << 41
    bad = [([10, 10], [0, 0], [0, 0], [5, 5]),      # repeated axis
           ([10, 10], [0, 1], [6, 0], [5, 5]),      # range leaves the input
           ([10, 10], [1], [10, 0], [0, 5]),        # dropped axis base out of range
           ([10, 10], [2], [0, 0], [5, 5]),         # axis out of range
           ([10, 10], [0, 1, 0], [0, 0], [5, 5])]   # rank_out > rank_in
    for dims, order, base, rng in bad:
        with pytest.raises(lr.RearrError):
            lr.reorder_nm(fake_dst, fake_src, 4, dims, order, base, rng)


def test_nm_in_a_batch(lr, orc):
    import torch
    g = synth.rng(66)
    cases, bufs = [], []
    pool = DevPool()
    plan = lr.Plan()
    for t in range(40):
        dims, order, base, rng = random_box(g, int(g.integers(1, 6)), max_extent=24)
        e = ELEMS[t % len(ELEMS)]
        src = synth.random_elements(900 + t, int(np.prod(dims)), e)
        total = int(np.prod([rng[a] for a in order]))
        s, d = to_dev(src, 0, pool), DevBuf(total * e, fill=0, pool=pool)
        plan.add_reorder_nm(d.ptr, s.ptr, e, dims, order, base, rng)
        cases.append((src, e, dims, order, base, rng))
        bufs.append((s, d))
    plan.finalize()
    plan.run()
    sync()
    pool.check()
    for (src, e, dims, order, base, rng), (s, d) in zip(cases, bufs):
        assert np.array_equal(d.download(), orc.reorder_nm(src, e, dims, order, base, rng))
    plan.close()
