"""Randomised parity against the oracle across every op class: permutes of
rank 1-6 and element sizes 1-16 at random alignments (every plan class:
copy, tile, cells, runs, strided), N-to-M boxes, the four index-sequence
forms, interlace / de-interlace with 1-12 planes, batched plans of mixed ops
and the host pipeline.  A fixed seed and a fixed number of draws."""
import collections

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, DevPool, sync, to_dev

pytestmark = pytest.mark.gpu

ELEMS = [1, 2, 3, 4, 6, 8, 12, 16]


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build
    build.build()
    import paper_1011_3583_gb300 as rr
    return rr


class Draws:
    def __init__(self, seed):
        self.g = np.random.default_rng(seed)

    def shape(self, rank, maxn=1 << 20):
        g = self.g
        while True:
            dims = [int(np.exp(g.uniform(0, np.log(200)))) for _ in range(rank)]
            if int(np.prod(dims)) <= maxn:
                return dims

    def permute(self):
        g = self.g
        e = int(g.choice(ELEMS))
        rank = int(g.integers(1, 7))
        dims = self.shape(rank)
        return e, dims, [int(x) for x in g.permutation(rank)]


def one_permute(rr, orc, d, it):
    e, dims, perm = d.permute()
    n = int(np.prod(dims))
    so = int(d.g.integers(0, 4)) * int(d.g.choice([1, e]))
    do = int(d.g.integers(0, 4)) * int(d.g.choice([1, e]))
    src = synth.random_elements(it, n, e)
    s, out = to_dev(src, so), DevBuf(n * e, do, fill=0xA5)
    rr.permute(out.ptr, s.ptr, e, dims, perm)
    sync()
    kind = rr.describe_permute(e, dims, perm, out.ptr, s.ptr)["kind"]
    ok = np.array_equal(out.download(), orc.permute(src, e, dims, perm))
    return "permute:" + kind, ok, (e, dims, perm, so, do)


def one_nm(rr, orc, d, it):
    g = d.g
    e = int(g.choice(ELEMS))
    rank = int(g.integers(1, 6))
    dims = d.shape(rank)
    base = [int(g.integers(0, x)) for x in dims]
    rng = [int(g.integers(1, x - b + 1)) for x, b in zip(dims, base)]
    order = [int(x) for x in g.permutation(rank)[:int(g.integers(1, rank + 1))]]
    n, tot = int(np.prod(dims)), int(np.prod([rng[a] for a in order]))
    src = synth.random_elements(it, n, e)
    s, out = to_dev(src), DevBuf(tot * e, 0, fill=0x11)
    rr.reorder_nm(out.ptr, s.ptr, e, dims, order, base, rng)
    sync()
    return "nm", np.array_equal(out.download(), orc.reorder_nm(src, e, dims, order, base, rng)), (e, dims, order, base, rng)


def one_indexed(rr, orc, d, it):
    g = d.g
    e = int(g.choice(ELEMS))
    n = int(g.integers(1, 300000))
    wide, scatter = bool(g.integers(0, 2)), bool(g.integers(0, 2))
    src = synth.random_elements(it, n, e)
    idx = synth.random_permutation(it, n).astype(np.uint64 if wide else np.uint32)
    s, ix, out = to_dev(src), to_dev(idx), DevBuf(n * e, 0, fill=0x22)
    fn = {(False, False): rr.reorder, (True, False): rr.reorder64, (False, True): rr.scatter,
          (True, True): rr.scatter64}[(wide, scatter)]
    fn(out.ptr, s.ptr, ix.ptr, n, e)
    sync()
    ok = np.array_equal(out.download(), orc.indexed(src, idx, e, scatter=scatter))
    return f"indexed:{'64' if wide else '32'}:{'scatter' if scatter else 'gather'}", ok, (e, n)


def one_interlace(rr, orc, d, it):
    g = d.g
    e = int(g.choice(ELEMS))
    k, n = int(g.integers(1, 13)), int(g.integers(1, 100000))
    off = 16 * int(g.integers(0, 2)) if g.integers(0, 2) else int(g.integers(0, 4))
    planes = [synth.random_elements(it + j, n, e) for j in range(k)]
    pd = [to_dev(p, off) for p in planes]
    iv = DevBuf(n * k * e, off, fill=0x33)
    rr.interlace(iv.ptr, [p.ptr for p in pd], n, e)
    sync()
    ok = np.array_equal(iv.download(), orc.interlace(planes, n, e))
    outs = [DevBuf(n * e, off, fill=0x44) for _ in range(k)]
    rr.deinterlace([o.ptr for o in outs], iv.ptr, n, e)
    sync()
    ok = ok and all(np.array_equal(o.download(), p) for o, p in zip(outs, planes))
    return "interlace", ok, (e, k, n, off)


def one_batch(rr, orc, d, it):
    g = d.g
    plan = rr.Plan()
    pool = DevPool()
    checks = []
    for j in range(int(g.integers(1, 40))):
        t = int(g.integers(0, 3))
        if t == 0:
            e, dims, perm = d.permute()
            n = int(np.prod(dims))
            src = synth.random_elements(it * 100 + j, n, e)
            s, out = to_dev(src, 0, pool), DevBuf(n * e, 0, fill=0, pool=pool)
            plan.add_permute(out.ptr, s.ptr, e, dims, perm)
            checks.append((out, orc.permute(src, e, dims, perm), s))
        elif t == 1:
            e, n = int(g.choice([1, 2, 4, 8])), int(g.integers(1, 100000))
            src, idx = synth.random_elements(it * 100 + j, n, e), synth.random_permutation(j, n)
            s, ix, out = to_dev(src, 0, pool), to_dev(idx, 0, pool), DevBuf(n * e, 0, fill=0, pool=pool)
            plan.add_reorder(out.ptr, s.ptr, ix.ptr, n, e)
            checks.append((out, orc.reorder(src, idx, e), (s, ix)))
        else:
            e, k, n = int(g.choice([1, 2, 4, 8])), int(g.integers(1, 9)), int(g.integers(1, 50000))
            planes = [synth.random_elements(it * 100 + j + q, n, e) for q in range(k)]
            pd = [to_dev(p, 0, pool) for p in planes]
            iv = DevBuf(n * k * e, 0, fill=0, pool=pool)
            plan.add_interlace(iv.ptr, [p.ptr for p in pd], n, e)
            checks.append((iv, orc.interlace(planes, n, e), pd))
    plan.finalize()
    plan.run()
    sync()
    pool.check()
    ok = all(np.array_equal(out.download(), want) for out, want, _ in checks)
    plan.close()
    return "batch", ok, (it, len(checks))


def one_pipeline(rr, orc, d, it):
    g = d.g
    form = int(g.integers(0, 3))
    if form == 0:
        e, dims, perm = d.permute()
        n = int(np.prod(dims))
        src = synth.random_elements(it, n, e)
        out = np.zeros(n * e, dtype=np.uint8)
        with rr.Pipeline(slot_bytes=2 * n * e + 4096, slots=3) as pipe:
            pipe.permute(out, src, e, dims, perm)
            pipe.sync()
        return "pipeline:permute", np.array_equal(out, orc.permute(src, e, dims, perm)), (e, dims, perm)
    if form == 1:
        e = int(g.choice(ELEMS))
        rank = int(g.integers(1, 5))
        dims = d.shape(rank)
        base = [int(g.integers(0, x)) for x in dims]
        rng = [int(g.integers(1, x - b + 1)) for x, b in zip(dims, base)]
        order = [int(x) for x in g.permutation(rank)[:int(g.integers(1, rank + 1))]]
        n, tot = int(np.prod(dims)), int(np.prod([rng[a] for a in order]))
        src = synth.random_elements(it, n, e)
        out = np.zeros(tot * e, dtype=np.uint8)
        with rr.Pipeline(slot_bytes=(n + tot) * e + 4096, slots=3) as pipe:
            pipe.reorder_nm(out, src, e, dims, order, base, rng)
            pipe.sync()
        return "pipeline:nm", np.array_equal(out, orc.reorder_nm(src, e, dims, order, base, rng)), (e, dims, order)
    e, n = int(g.choice(ELEMS)), int(g.integers(1, 200000))
    wide, scatter = bool(g.integers(0, 2)), bool(g.integers(0, 2))
    src = synth.random_elements(it, n, e)
    idx = synth.random_permutation(it, n).astype(np.uint64 if wide else np.uint32)
    out = np.zeros(n * e, dtype=np.uint8)
    with rr.Pipeline(slot_bytes=n * (2 * e + 8) + 4096, slots=3) as pipe:
        fn = {(False, False): pipe.reorder, (True, False): pipe.reorder64, (False, True): pipe.scatter,
              (True, True): pipe.scatter64}[(wide, scatter)]
        fn(out, src, idx, n, e)
        pipe.sync()
    return "pipeline:indexed", np.array_equal(out, orc.indexed(src, idx, e, scatter=scatter)), (e, n, wide, scatter)


@pytest.mark.parametrize("seed", [11, 12])
def test_random_ops_match_oracle(rr, seed):
    orc = oracle.get()
    d = Draws(seed)
    kinds = [one_permute, one_nm, one_indexed, one_interlace, one_batch, one_pipeline]
    stats, fails = collections.Counter(), []
    for it in range(1, 601):
        name, ok, what = kinds[int(d.g.integers(0, len(kinds)))](rr, orc, d, it)
        stats[name] += 1
        if not ok:
            fails.append((name, what))
    assert not fails, (dict(stats), fails[:5])
    assert all(stats[k] > 0 for k in ("nm", "interlace", "batch", "pipeline:permute", "pipeline:indexed"))
