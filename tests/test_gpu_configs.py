"""The benchmark workloads at full size, compared with the oracle in full.

Every output byte of every full-size config is compared with the oracle's
loop nest: the 1024^2 fp32 transpose, all 6 orders of 512^3 fp32, all 24
orders of 64x128x256x64 at 2, 4 and 8 bytes, the 2^28 fp32 reorders, the
complex64 split, the 4096^2 image planes and the AoS/SoA records.  The oracle
is single-threaded C; independent oracle calls run on a few host threads at a
time (the ctypes call releases the interpreter lock) while the GPU runs the
next order.  Every output buffer is guarded (tests.gpu_util), so a write
outside it fails too.  A permute followed by its inverse, a reorder by the
inverse permutation and interlace followed by de-interlace are also checked
to give back the input.  The launch configuration is the one bench.py times
(single calls on one stream).
"""
import collections
import itertools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, sync, to_dev

pytestmark = pytest.mark.gpu

ORACLE_THREADS = max(1, min(6, (os.cpu_count() or 2) - 2))


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


def in_order(calls, window=ORACLE_THREADS):
    """Results of the callables in order, at most `window` running at once."""
    with ThreadPoolExecutor(max_workers=window) as ex:
        it = iter(calls)
        pending = collections.deque(ex.submit(f) for f in itertools.islice(it, window))
        while pending:
            r = pending.popleft().result()
            nxt = next(it, None)
            if nxt is not None:
                pending.append(ex.submit(nxt))
            yield r


def inverse(perm):
    inv = [0] * len(perm)
    for i, p in enumerate(perm):
        inv[p] = i
    return inv


def assert_same(got: np.ndarray, want: np.ndarray, what):
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{what}: {bad.size} bytes differ, first at byte {bad[0]}")


def permute_all_orders(lr, orc, dims, e, seed):
    import torch
    n = int(np.prod(dims))
    src_np = synth.random_elements(seed, n, e)
    src = to_dev(src_np)
    out = DevBuf(n * e)
    back = DevBuf(n * e)
    perms = [list(p) for p in itertools.permutations(range(len(dims)))]
    wants = in_order(lambda p=p: orc.permute(src_np, e, dims, p) for p in perms)
    for perm, want in zip(perms, wants):
        out.view.fill_(0xA5)
        lr.permute(out.ptr, src.ptr, e, dims, perm)
        sync()
        assert_same(out.download(), want, ("permute", dims, perm, e))
        del want
        lr.permute(back.ptr, out.ptr, e, [dims[p] for p in perm], inverse(perm))
        sync()
        back.check_guards()
        assert torch.equal(back.view, src.view), ("inverse round trip", dims, perm, e)


def test_config_transpose_1024(lr, orc):
    """1024 x 1024 fp32 transpose."""
    src_np = synth.random_elements(2024, 1024 * 1024, 4)
    src = to_dev(src_np)
    out = DevBuf(src_np.size, fill=0)
    lr.permute(out.ptr, src.ptr, 4, [1024, 1024], [1, 0])
    sync()
    assert_same(out.download(), orc.permute(src_np, 4, [1024, 1024], [1, 0]), "transpose 1024^2")


def test_config_rank3_512_cubed(lr, orc):
    permute_all_orders(lr, orc, [512, 512, 512], 4, seed=512)


@pytest.mark.parametrize("e", [2, 4, 8])
def test_config_rank4_all_orders(lr, orc, e):
    permute_all_orders(lr, orc, [64, 128, 256, 64], e, seed=64 + e)


@pytest.mark.parametrize("kind", ["random", "block4096"])
def test_config_reorder_2p28(lr, orc, kind):
    import torch
    n = 1 << 28
    src_np = synth.random_elements(28, n, 4)
    idx_np = (synth.random_permutation(29, n) if kind == "random"
              else synth.block_shuffled_permutation(30, n, 4096))
    with ThreadPoolExecutor(max_workers=1) as ex:
        want = ex.submit(orc.reorder, src_np, idx_np, 4)
        src, idx = to_dev(src_np), to_dev(idx_np)
        out = DevBuf(n * 4, fill=0x5A)
        lr.reorder(out.ptr, src.ptr, idx.ptr, n, 4)
        sync()
        assert_same(out.download(), want.result(), ("reorder 2^28", kind))
    # reorder by the inverse permutation restores the input everywhere
    inv_np = np.empty_like(idx_np)
    inv_np[idx_np] = np.arange(n, dtype=np.uint32)
    inv = to_dev(inv_np)
    back = DevBuf(n * 4)
    lr.reorder(back.ptr, out.ptr, inv.ptr, n, 4)
    sync()
    back.check_guards()
    assert torch.equal(back.view, src.view)


def interlace_both_ways(lr, orc, k, n, e, seed):
    """Interlace k planes and de-interlace an independent interlaced array,
    both compared with the oracle in full; then de-interlace the interlaced
    result and get the planes back."""
    import torch
    planes_np = [synth.random_elements(seed + j, n, e) for j in range(k)]
    arr_np = synth.random_elements(seed + 100, n * k, e)
    with ThreadPoolExecutor(max_workers=2) as ex:
        want_i = ex.submit(orc.interlace, planes_np, n, e)
        want_d = ex.submit(orc.deinterlace, arr_np, k, n, e)
        planes = [to_dev(p) for p in planes_np]
        inter = DevBuf(n * k * e, fill=0x33)
        lr.interlace(inter.ptr, [p.ptr for p in planes], n, e)
        sync()
        assert_same(inter.download(), want_i.result(), ("interlace", k, n, e))
        arr = to_dev(arr_np)
        outs = [DevBuf(n * e, fill=0x44) for _ in range(k)]
        lr.deinterlace([o.ptr for o in outs], arr.ptr, n, e)
        sync()
        for j, (o, w) in enumerate(zip(outs, want_d.result())):
            assert_same(o.download(), w, ("de-interlace", k, n, e, j))
    del arr, want_d
    for o in outs:
        o.view.fill_(0)
    lr.deinterlace([o.ptr for o in outs], inter.ptr, n, e)
    sync()
    for o, p in zip(outs, planes):
        o.check_guards()
        assert torch.equal(o.view, p.view), ("de-interlace round trip", k, n, e)


def test_config_complex_split_2p28(lr, orc):
    """complex64 of 2^28 elements <-> real and imaginary fp32 planes."""
    interlace_both_ways(lr, orc, 2, 1 << 28, 4, seed=64)


@pytest.mark.parametrize("k", [3, 4])
def test_config_image_planes_4096(lr, orc, k):
    """4096 x 4096 uint8 images, k planes."""
    interlace_both_ways(lr, orc, k, 4096 * 4096, 1, seed=70)


@pytest.mark.parametrize("k", [2, 3, 4, 8])
def test_config_aos_soa_2p26(lr, orc, k):
    interlace_both_ways(lr, orc, k, 1 << 26, 4, seed=80 + k)
