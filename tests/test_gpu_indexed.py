"""Scatter reorder and 64-bit index sequences on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, DevPool, sync, to_dev

pytestmark = pytest.mark.gpu


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


def run(lr, fn, src, idx, e, n, fill, offs=(0, 0, 0)):
    s, ix = to_dev(src, offs[0]), to_dev(idx, offs[2])
    d = DevBuf(n * e, offs[1], fill=fill)
    fn(d.ptr, s.ptr, ix.ptr, n, e)
    sync()
    return d.download()


@pytest.mark.parametrize("e", [1, 2, 3, 4, 8, 12, 16])
def test_scatter_permutation(lr, orc, e):
    for t, n in enumerate([1, 5, 1000, 65539, (1 << 18) + 7]):
        src = synth.random_elements(40 + t, n, e)
        p = synth.random_permutation(50 + t, n)
        got = run(lr, lr.scatter, src, p, e, n, fill=0)
        assert np.array_equal(got, orc.indexed(src, p, e, scatter=True)), (n, e)
        p64 = p.astype(np.uint64)
        got = run(lr, lr.scatter64, src, p64, e, n, fill=0)
        assert np.array_equal(got, orc.indexed(src, p64, e, scatter=True)), (n, e, "64")
        got = run(lr, lr.reorder64, src, p64, e, n, fill=0)
        assert np.array_equal(got, orc.indexed(src, p64, e, scatter=False)), (n, e, "gather64")


def test_scatter_unaligned(lr, orc):
    n = 5003
    for e, so, do, io in [(4, 4, 0, 4), (4, 0, 8, 0), (8, 8, 4, 8), (2, 2, 6, 12), (1, 1, 3, 4)]:
        src = synth.random_elements(e + so, n, e)
        p = synth.random_permutation(e + io, n)
        got = run(lr, lr.scatter, src, p, e, n, fill=0, offs=(so, do, io))
        assert np.array_equal(got, orc.indexed(src, p, e, scatter=True)), (e, so, do, io)


def test_scatter_repeats_are_valid(lr):
    """With repeated indices the written value is one of the colliding
    sources (which one is unspecified) and untouched positions keep theirs."""
    n, e = 70001, 4
    src = np.arange(n, dtype=np.uint32).view(np.uint8)     # tag = source position
    idx = synth.random_indices(9, n, n // 3)               # many collisions, a third targeted
    got = run(lr, lr.scatter, src, idx, e, n, fill=0xFF).view(np.uint32)
    targeted = np.zeros(n, bool)
    targeted[idx] = True
    assert np.all(got[~targeted] == 0xFFFFFFFF)
    # every targeted destination holds the tag of some i with idx[i] == destination
    ok = idx[got[targeted]] == np.flatnonzero(targeted)
    assert np.all(ok)


def test_gather64_with_repeats(lr, orc):
    for e in (1, 4, 8, 12):
        n = 33333
        src = synth.random_elements(60 + e, n, e)
        idx = synth.random_indices(61 + e, n, n).astype(np.uint64)
        got = run(lr, lr.reorder64, src, idx, e, n, fill=0)
        assert np.array_equal(got, orc.indexed(src, idx, e, scatter=False)), e


def test_scatter_in_a_batch(lr, orc):
    plan = lr.Plan()
    pool = DevPool()
    cases = []
    for t, (n, e) in enumerate([(1000, 4), (4099, 1), (77777, 8), (5, 16)]):
        src = synth.random_elements(70 + t, n, e)
        p = synth.random_permutation(80 + t, n)
        s, ix, d = to_dev(src, 0, pool), to_dev(p, 0, pool), DevBuf(n * e, fill=0, pool=pool)
        plan.add_scatter(d.ptr, s.ptr, ix.ptr, n, e)
        cases.append((src, p, e, s, ix, d))
    plan.finalize()
    plan.run()
    sync()
    pool.check()
    for src, p, e, s, ix, d in cases:
        assert np.array_equal(d.download(), orc.indexed(src, p, e, scatter=True))
    plan.close()


@pytest.mark.parametrize("e,kind", [(4, "perm"), (4, "block"), (4, "reverse"), (8, "perm"), (16, "perm")])
def test_scatter_large_sources(lr, orc, e, kind):
    """Scatters of 128 MiB or more (L2-resident passes, or the direct scatter
    when the indices are local)."""
    n = (128 << 20) // e + 4099
    if kind == "perm":
        idx = synth.random_permutation(17 + e, n)
    elif kind == "reverse":
        idx = np.arange(n - 1, -1, -1, dtype=np.uint32)
    else:
        m = n - n % 4096
        idx = np.concatenate([synth.block_shuffled_permutation(18, m, 4096), np.arange(m, n, dtype=np.uint32)])
    src = synth.random_elements(19 + e, n, e)
    got = run(lr, lr.scatter, src, idx, e, n, fill=0)
    assert np.array_equal(got, orc.indexed(src, idx, e, scatter=True)), (e, kind)


def test_scatter_large_repeats_are_valid(lr):
    n, e = (128 << 20) // 4 + 17, 4
    src = np.arange(n, dtype=np.uint32).view(np.uint8)
    idx = synth.random_indices(23, n, n // 2)
    got = run(lr, lr.scatter, src, idx, e, n, fill=0xFF).view(np.uint32)
    targeted = np.zeros(n, bool)
    targeted[idx] = True
    assert np.all(got[~targeted] == 0xFFFFFFFF)
    assert np.all(idx[got[targeted]] == np.flatnonzero(targeted))


@pytest.mark.parametrize("idx_bytes", [4, 8])
@pytest.mark.parametrize("off", [0, 4, 8])
def test_check_indices_counts_exactly(lr, idx_bytes, off):
    if idx_bytes == 8 and off % 8:
        pytest.skip("8-byte indices must be 8-byte aligned")
    g = np.random.default_rng(idx_bytes + off)
    for n in (1, 3, 1000, 65537, (1 << 20) + 5):
        bound = n
        dt = np.uint32 if idx_bytes == 4 else np.uint64
        idx = g.integers(0, n, size=n).astype(dt)
        k = int(g.integers(0, min(n, 50) + 1))
        pos = g.choice(n, size=k, replace=False) if k else np.array([], dtype=np.int64)
        big = (2 ** 32 + 7) if idx_bytes == 8 else (2 ** 32 - 1)
        idx[pos] = g.integers(n, big, size=k).astype(dt) if k else idx[pos]
        ix = to_dev(idx, off)
        assert lr.check_indices(ix.ptr, n, idx_bytes, bound) == int((idx.astype(np.uint64) >= bound).sum())


def test_reorder_checked(lr, orc):
    n, e = 100003, 4
    src = synth.random_elements(7, n, e)
    idx = synth.random_indices(8, n, n)
    got = run(lr, lr.reorder_checked, src, idx, e, n, fill=0x5A)
    assert np.array_equal(got, orc.reorder(src, idx, e))
    bad = idx.copy()
    bad[[0, 777, n - 1]] = [n, n + 5, 2 ** 32 - 1]
    with pytest.raises(lr.RearrError) as ex:
        run(lr, lr.reorder_checked, src, bad, e, n, fill=0x5A)
    assert ex.value.status == lr.ERANGE and "3 of" in str(ex.value)


def test_reorder_checked_leaves_dst_untouched(lr):
    n, e = 4096, 8
    src = synth.random_elements(9, n, e)
    idx = synth.random_indices(10, n, n)
    idx[100] = n
    s, ix = to_dev(src), to_dev(idx)
    d = DevBuf(n * e, 0, fill=0x33)
    with pytest.raises(lr.RearrError):
        lr.reorder_checked(d.ptr, s.ptr, ix.ptr, n, e)
    sync()
    assert np.all(d.download() == 0x33)


@pytest.mark.parametrize("e,kind,scatter", [(4, "perm", False), (4, "perm", True), (4, "repeat", False),
                                            (4, "block", False), (8, "perm", True), (16, "perm", False),
                                            (16, "repeat", False)])
def test_wide_indices_large_sources(lr, orc, e, kind, scatter):
    """64-bit index sequences over sources of 128 MiB or more (the bucketed
    passes read the 8-byte indices; the block-shuffled one keeps the direct
    path): the same bytes as the oracle."""
    n = (128 << 20) // e + 4099
    if kind == "perm":
        idx = synth.random_permutation(31 + e, n)
    elif kind == "repeat":
        idx = synth.random_indices(32 + e, n, n)
    else:
        m = n - n % 4096
        idx = np.concatenate([synth.block_shuffled_permutation(33, m, 4096), np.arange(m, n, dtype=np.uint32)])
    idx = idx.astype(np.uint64)
    src = synth.random_elements(34 + e, n, e)
    fn = lr.scatter64 if scatter else lr.reorder64
    got = run(lr, fn, src, idx, e, n, fill=0)
    assert np.array_equal(got, orc.indexed(src, idx, e, scatter=scatter)), (e, kind, scatter)
