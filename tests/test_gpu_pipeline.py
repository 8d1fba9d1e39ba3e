"""Host-buffer pipeline (include/librearr_pipeline.h) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from synth.stencils import fd_laplacian
from tests.gpu_util import HostBuf

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


def pinned(nbytes):
    import torch
    return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)


@pytest.mark.parametrize("host", ["pageable", "pinned"])
def test_mixed_ops_more_ops_than_slots(lr, orc, host):
    """Ten ops of different kinds and sizes through three slots: every output
    lands intact (slot reuse waits for the previous download)."""
    ops = []
    g = np.random.default_rng(3)
    for i in range(10):
        kind = ["permute", "reorder", "interlace", "deinterlace", "stencil"][i % 5]
        ops.append((kind, i, g))
    guarded = []

    def out_buf(nbytes):
        h = HostBuf(nbytes, offset=len(guarded) % 5)
        guarded.append(h)
        return h.body

    with lr.Pipeline(slot_bytes=8 << 20, slots=3) as pipe:
        checks = []
        for kind, i, _ in ops:
            seed = 100 + i
            if kind == "permute":
                dims, perm, e = [37, 64, 29], [2, 0, 1], 4
                src = synth.random_elements(seed, int(np.prod(dims)), e)
                dst = out_buf(src.size)
                if host == "pinned":
                    s_t, d_t = pinned(src.size), pinned(dst.size)
                    s_t.numpy()[:] = src
                    pipe.permute(d_t, s_t, e, dims, perm)
                    checks.append((lambda d_t=d_t: d_t.numpy().copy(), orc.permute(src, e, dims, perm)))
                else:
                    pipe.permute(dst, src, e, dims, perm)
                    checks.append((lambda dst=dst: dst, orc.permute(src, e, dims, perm)))
            elif kind == "reorder":
                n, e = 100003, 8
                src = synth.random_elements(seed, n, e)
                idx = synth.random_indices(seed, n, n)
                dst = out_buf(n * e)
                pipe.reorder(dst, src, idx, n, e)
                checks.append((lambda dst=dst: dst, orc.reorder(src, idx, e)))
            elif kind == "interlace":
                n, k, e = 50001, 3, 2
                planes = [synth.random_elements(seed + j, n, e) for j in range(k)]
                dst = out_buf(n * k * e)
                pipe.interlace(dst, planes, n, e)
                checks.append((lambda dst=dst: dst, orc.interlace(planes, n, e)))
            elif kind == "deinterlace":
                n, k, e = 40000, 4, 4
                src = synth.random_elements(seed, n * k, e)
                outs = [out_buf(n * e) for _ in range(k)]
                pipe.deinterlace(outs, src, n, e)
                want = orc.deinterlace(src, k, n, e)
                checks.append((lambda outs=outs: np.concatenate(outs), np.concatenate(want)))
            else:
                ny, nx = 300, 260
                grid = np.random.default_rng(seed).normal(size=(ny, nx)).astype(np.float32)
                taps = [(dy, dx, float(np.float32(w))) for dy, dx, w in fd_laplacian(2)]
                out = out_buf(ny * nx * 4).view(np.float32).reshape(ny, nx)
                pipe.stencil2d(out, grid, ny, nx, taps, 1)
                want = orc.stencil2d(grid, taps, 1)
                s = orc.stencil2d(np.abs(grid), [(a, b, abs(w)) for a, b, w in taps], 1)
                tol = (len(taps) + 1) * 2.0 ** -24 * s
                checks.append((lambda out=out, want=want, tol=tol: np.abs(out.astype(np.float64) - want) <= tol,
                               np.ones((ny, nx), dtype=bool)))
        pipe.sync()
        for h in guarded:
            h.check_guards()
        for i, (got, want) in enumerate(checks):
            assert np.array_equal(got(), want), ops[i][0]
        st = pipe.stats()
        assert st["ops"] == 10 and st["h2d_bytes"] > 0 and st["d2h_bytes"] > 0


def test_op_larger_than_a_slot_is_rejected(lr, orc):
    with lr.Pipeline(slot_bytes=1 << 20, slots=3) as pipe:
        big = np.zeros(1 << 20, dtype=np.uint8)
        out = np.zeros_like(big)
        with pytest.raises(lr.RearrError) as ex:
            pipe.permute(out, big, 1, [1024, 1024], [1, 0])  # 2 MiB of staging
        assert ex.value.status == lr.EINVAL
        # invalid arguments are rejected before anything is enqueued, and the
        # pipeline stays usable
        with pytest.raises(lr.RearrError):
            pipe.permute(out, big, 4, [16, 16], [0, 0])
        src = synth.random_elements(9, 256 * 128, 4)
        dst = np.zeros(src.size, dtype=np.uint8)
        pipe.permute(dst, src, 4, [256, 128], [1, 0])
        pipe.sync()
        assert np.array_equal(dst, orc.permute(src, 4, [256, 128], [1, 0]))
        assert pipe.stats()["ops"] == 1


def test_large_ops_stream_through(lr, orc):
    """Ops of 256 MiB each through three slots (the bench's e2e scale)."""
    import torch
    n = 1 << 26
    e = 4
    with lr.Pipeline(slot_bytes=2 * n * e + (1 << 20), slots=3) as pipe:
        src = pinned(n * e)
        src.numpy()[:] = synth.random_elements(1, n, e)
        dsts = [pinned(n * e) for _ in range(4)]
        dims, perms = [512, 256, 512], [[2, 1, 0], [1, 2, 0], [0, 2, 1], [2, 0, 1]]
        for d, p in zip(dsts, perms):
            pipe.permute(d, src, e, dims, p)
        pipe.sync()
        for d, p in zip(dsts, perms):
            lin = np.random.default_rng(sum(p)).integers(0, n, size=4096)
            want = orc.permute_sample(src.numpy(), e, dims, p, lin)
            got = d.numpy().view(np.uint32)[lin].view(np.uint8)
            assert np.array_equal(got, want), p
    del torch


def test_nm_scatter_and_wide_indices(lr, orc):
    """The N-to-M reorder, the scatter and the 64-bit index forms on host buffers."""
    with lr.Pipeline(slot_bytes=16 << 20, slots=3) as pipe:
        dims, order, base, rng = [40, 50, 60], [2, 0], [3, 7, 5], [30, 1, 50]
        src = synth.random_elements(1, int(np.prod(dims)), 4)
        guarded = [HostBuf(50 * 30 * 4, 3)] + [HostBuf(77777 * 8, j) for j in range(3)]
        out_nm = guarded[0].body
        pipe.reorder_nm(out_nm, src, 4, dims, order, base, rng)
        n, e = 77777, 8
        s2 = synth.random_elements(2, n, e)
        p = synth.random_permutation(3, n)
        outs = {k: h.body for k, h in zip(("scatter", "reorder64", "scatter64"), guarded[1:])}
        pipe.scatter(outs["scatter"], s2, p, n, e)
        pipe.reorder64(outs["reorder64"], s2, p.astype(np.uint64), n, e)
        pipe.scatter64(outs["scatter64"], s2, p.astype(np.uint64), n, e)
        pipe.sync()
        for h in guarded:
            h.check_guards()
        assert np.array_equal(out_nm, orc.reorder_nm(src, 4, dims, order, base, rng))
        assert np.array_equal(outs["scatter"], orc.indexed(s2, p, e, scatter=True))
        assert np.array_equal(outs["scatter64"], orc.indexed(s2, p, e, scatter=True))
        assert np.array_equal(outs["reorder64"], orc.reorder(s2, p, e))


def pinned_guarded(nbytes, off=0):
    """A page-locked buffer with guard bands before and after its body."""
    from tests.gpu_util import GUARD, guard_pattern
    t = pinned(GUARD + off + nbytes + GUARD)
    a = t.numpy()
    a[:GUARD + off] = guard_pattern(GUARD + off, 0)
    a[GUARD + off + nbytes:] = guard_pattern(GUARD, 1)
    return t, a[GUARD + off: GUARD + off + nbytes]


def guards_intact(t, nbytes, off=0):
    from tests.gpu_util import GUARD, guard_pattern
    a = t.numpy()
    return (np.array_equal(a[:GUARD + off], guard_pattern(GUARD + off, 0)) and
            np.array_equal(a[GUARD + off + nbytes:], guard_pattern(GUARD, 1)))


@pytest.mark.parametrize("mode", [1, 0])
def test_direct_ops_keep_submission_order(lr, orc, mode):
    """A chain through page-locked host buffers mixing ops that run directly on
    them (permutes planned as tiles and boxes, interlaces) and a staged op (a
    reorder): each op reads what the op before it wrote, so the
    results match the oracle's chain only if host memory sees the ops in
    submission order.  Mode 0 stages everything; both give the same bytes and
    no op writes outside its output."""
    e4, dims, perm = 4, [61, 47, 33], [2, 0, 1]
    n = int(np.prod(dims))
    src = synth.random_elements(71, n, e4)
    idx = synth.random_indices(72, n, n)
    bufs = {}
    for name, nb, off in (("src", n * e4, 0), ("a", n * e4, 4), ("b", n * e4, 0), ("c", n * e4, 8),
                          ("u8", 16 * 3 * 4099, 0), ("u8t", 16 * 3 * 4099, 1), ("il", 2 * n * e4, 0),
                          ("d0", n * e4, 0), ("d1", n * e4, 0)):
        bufs[name] = (pinned_guarded(nb, off), nb, off)
    body = {k: v[0][1] for k, v in bufs.items()}
    body["src"][:] = src
    img = synth.random_elements(73, 16 * 3 * 4099, 1)
    body["u8"][:] = img
    with lr.Pipeline(slot_bytes=8 << 20, slots=3) as pipe:
        pipe.set_direct(mode)
        t = {k: v[0][0] for k, v in bufs.items()}
        off = {k: v[2] for k, v in bufs.items()}
        from tests.gpu_util import GUARD

        def ptr(k):
            return t[k].data_ptr() + GUARD + off[k]

        pipe.permute(ptr("a"), ptr("src"), e4, dims, perm)                 # tile
        pipe.reorder(ptr("b"), ptr("a"), idx, n, e4)                       # staged, reads a
        pipe.permute(ptr("c"), ptr("b"), e4, [61, 47 * 33], [1, 0])        # reads b
        pipe.permute(ptr("u8t"), ptr("u8"), 1, [16, 3, 4099], [0, 2, 1])  # a box of 1-byte cells
        pipe.interlace(ptr("il"), [ptr("c"), ptr("a")], n, e4)             # reads c and a
        pipe.deinterlace([ptr("d0"), ptr("d1")], ptr("il"), n, e4)         # reads il
        pipe.sync()
        d = pipe.direct()
        # direct ops: the permutes whose plans stream, the interlace and the
        # de-interlace (the reorder is always staged)
        streaming = sum(lr.describe_permute(e, dm, pm, ptr(o), ptr(i))["kind"] in ("copy", "tile", "tile_cells",
                                                                                     "runs", "box")
                        for o, i, e, dm, pm in (("a", "src", e4, dims, perm), ("c", "b", e4, [61, 47 * 33], [1, 0]),
                                                ("u8t", "u8", 1, [16, 3, 4099], [0, 2, 1])))
        assert d["mode"] == mode
        assert d["direct_ops"] == (streaming + 2 if mode else 0), (d, streaming)
    a = orc.permute(src, e4, dims, perm)
    b = orc.reorder(a, idx, e4)
    c = orc.permute(b, e4, [61, 47 * 33], [1, 0])
    il = orc.interlace([c, a], n, e4)
    d0, d1 = orc.deinterlace(il, 2, n, e4)
    for k, want in (("a", a), ("b", b), ("c", c), ("il", il), ("d0", d0), ("d1", d1),
                    ("u8t", orc.permute(img, 1, [16, 3, 4099], [0, 2, 1]))):
        assert np.array_equal(body[k], want), k
    for k, (tb, nb, o) in bufs.items():
        assert guards_intact(tb[0], nb, o), k
