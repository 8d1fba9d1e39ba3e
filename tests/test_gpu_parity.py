"""GPU results of every librearr operation against the CPU oracle, bit for bit.

Sizes are small enough for the oracle to finish in seconds but span several
tiles with ragged tails; every call goes through the C ABI (ctypes binding).
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, DevPool, sync, to_dev

pytestmark = pytest.mark.gpu

ELEMS = (1, 2, 3, 4, 6, 8, 12, 16, 24, 40, 300)


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


def run_permute(lr, src_np, e, dims, perm, src_off=0, dst_off=0):
    n = int(np.prod(dims, dtype=np.int64))
    s = to_dev(src_np, src_off)
    d = DevBuf(n * e, dst_off, fill=0xA5)
    lr.permute(d.ptr, s.ptr, e, dims, perm)
    sync()
    return d.download()


def check_permute(lr, orc, seed, e, dims, perm, src_off=0, dst_off=0):
    n = int(np.prod(dims, dtype=np.int64))
    src = synth.random_elements(seed, n, e)
    got = run_permute(lr, src, e, dims, perm, src_off, dst_off)
    want = orc.permute(src, e, dims, perm)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"permute dims={dims} perm={perm} e={e} offs=({src_off},{dst_off}): "
                             f"{bad.size} bytes differ, first at byte {bad[0]}; "
                             f"plan={lr.describe_permute(e, dims, perm, 0, 0)}")


def test_permute_random_shapes(lr, orc):
    g = synth.rng(101)
    for t in range(160):
        rank = int(g.integers(1, 9))
        e = ELEMS[t % len(ELEMS)]
        budget = 400_000 // e
        dims = [int(g.integers(1, 80 if rank <= 3 else 12)) for _ in range(rank)]
        while int(np.prod(dims)) > budget:
            dims[int(np.argmax(dims))] //= 2
        perm = [int(v) for v in g.permutation(rank)]
        check_permute(lr, orc, 1000 + t, e, dims, perm)


@pytest.mark.parametrize("e", [1, 2, 4, 8, 16])
def test_permute_rank3_all_orders(lr, orc, e):
    dims = [67, 130, 129] if e <= 4 else [33, 70, 65]
    for perm in itertools.permutations(range(3)):
        check_permute(lr, orc, 77 + e, e, dims, list(perm))


@pytest.mark.parametrize("e", [1, 2, 4, 8])
def test_permute_rank4_all_orders(lr, orc, e):
    dims = [9, 33, 70, 17]
    for perm in itertools.permutations(range(4)):
        check_permute(lr, orc, 99 + e, e, dims, list(perm))


@pytest.mark.parametrize("e", [1, 2, 4, 8])
def test_permute_aligned_fast_paths(lr, orc, e):
    # power-of-two extents: 16-byte vectors on both sides, several tiles
    for dims, perm in [([256, 320], [1, 0]), ([16, 64, 96], [2, 0, 1]), ([8, 32, 16, 64], [3, 1, 0, 2]),
                       ([4, 96, 128], [0, 2, 1]), ([2, 3, 64, 128], [1, 0, 3, 2])]:
        check_permute(lr, orc, 5 + e, e, dims, perm)


@pytest.mark.parametrize("src_off,dst_off", [(1, 0), (0, 1), (2, 6), (4, 0), (0, 4), (8, 8), (12, 4), (3, 5)])
def test_permute_unaligned_pointers(lr, orc, src_off, dst_off):
    for e in (1, 2, 4, 8, 16):
        check_permute(lr, orc, 7 * e + src_off, e, [48, 136], [1, 0], src_off, dst_off)
        check_permute(lr, orc, 9 * e + dst_off, e, [5, 40, 24], [2, 1, 0], src_off, dst_off)


def test_permute_edge_cases(lr, orc):
    check_permute(lr, orc, 1, 4, [1], [0])
    check_permute(lr, orc, 2, 4, [1, 1, 1], [2, 0, 1])
    check_permute(lr, orc, 3, 8, [65537, 3], [1, 0])
    check_permute(lr, orc, 4, 1, [3, 65537], [1, 0])
    check_permute(lr, orc, 5, 4, [2, 3, 2, 3, 2, 3, 2, 3], [7, 6, 5, 4, 3, 2, 1, 0])
    check_permute(lr, orc, 6, 2, [3] * 8, [1, 0, 3, 2, 5, 4, 7, 6])
    check_permute(lr, orc, 7, 4, [1000, 1, 1, 3], [3, 2, 1, 0])
    check_permute(lr, orc, 8, 4, [7, 1024], [0, 1])          # identity -> copy
    check_permute(lr, orc, 9, 1, [3, 5, 1001], [1, 0, 2])    # unmoved inner run, 1001 B
    check_permute(lr, orc, 10, 4, [3, 5, 64], [1, 0, 2])     # runs of 256 B
    check_permute(lr, orc, 11, 2, [40, 3, 7], [1, 0, 2])     # short unmoved runs -> cells
    check_permute(lr, orc, 12, 5000, [3, 4], [1, 0])         # huge elements -> runs
    # zero elements: no launch, dst untouched
    before = lr.launch_count()
    lr.permute(0, 0, 4, [5, 0, 3], [2, 1, 0])
    assert lr.launch_count() == before


def test_permute_tagged_bijection(lr):
    """Tagged input: every output tag appears exactly once (catches stale or
    overwritten shared-memory tiles as duplicates)."""
    import torch
    for dims, perm in [([256, 256, 33], [2, 0, 1]), ([129, 67, 31], [1, 2, 0]), ([64, 64, 64, 16], [3, 2, 1, 0])]:
        n = int(np.prod(dims))
        src = synth.tagged_elements(n, 4)
        got = run_permute(lr, src, 4, dims, perm).view(np.uint32)
        assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32)), (dims, perm)


# ---------------------------------------------------------------------------
# reorder

@pytest.mark.parametrize("e", [1, 2, 3, 4, 8, 12, 16])
def test_reorder(lr, orc, e):
    for t, n in enumerate([1, 3, 4, 5, 1000, 65537, (1 << 18) + 3]):
        src = synth.random_elements(200 + t, n, e)
        for kind in ("perm", "repeat", "block"):
            if kind == "perm":
                idx = synth.random_permutation(300 + t, n)
            elif kind == "repeat":
                idx = synth.random_indices(400 + t, n, n)
            else:
                if n % 64:
                    continue
                idx = synth.block_shuffled_permutation(500 + t, n, 64)
            s, ix = to_dev(src), to_dev(idx)
            d = DevBuf(n * e, fill=0x5A)
            lr.reorder(d.ptr, s.ptr, ix.ptr, n, e)
            sync()
            assert np.array_equal(d.download(), orc.reorder(src, idx, e)), (n, e, kind)


def test_reorder_unaligned(lr, orc):
    n = 5003
    for e, so, do, io in [(4, 0, 0, 4), (4, 2, 0, 0), (8, 8, 4, 8), (2, 1, 3, 12), (16, 4, 8, 0), (1, 3, 1, 4)]:
        src = synth.random_elements(e + so, n, e)
        idx = synth.random_permutation(e + io, n)
        s, ix = to_dev(src, so), to_dev(idx, io)
        d = DevBuf(n * e, do)
        lr.reorder(d.ptr, s.ptr, ix.ptr, n, e)
        sync()
        assert np.array_equal(d.download(), orc.reorder(src, idx, e)), (e, so, do, io)


# ---------------------------------------------------------------------------
# interlace / de-interlace

def check_interlace(lr, orc, k, n, e, offs=None, seed=0):
    offs = offs or [0] * (k + 1)
    planes = [synth.random_elements(seed + 10 * j, n, e) for j in range(k)]
    pd = [to_dev(p, offs[j]) for j, p in enumerate(planes)]
    d = DevBuf(n * k * e, offs[k], fill=0x11)
    lr.interlace(d.ptr, [p.ptr for p in pd], n, e)
    sync()
    got = d.download()
    want = orc.interlace(planes, n, e)
    assert np.array_equal(got, want), ("interlace", k, n, e, offs)
    # de-interlace of an independent interlaced array
    arr = synth.random_elements(seed + 7, n * k, e)
    s = to_dev(arr, offs[k])
    outs = [DevBuf(n * e, offs[j], fill=0x22) for j in range(k)]
    lr.deinterlace([o.ptr for o in outs], s.ptr, n, e)
    sync()
    want = orc.deinterlace(arr, k, n, e)
    for j in range(k):
        assert np.array_equal(outs[j].download(), want[j]), ("deinterlace", k, n, e, offs, j)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7, 8, 9, 16])
def test_interlace(lr, orc, k):
    for e in (1, 2, 3, 4, 8, 16):
        for n in (1, 7, 1000, 4099, 65536 + 5):
            check_interlace(lr, orc, k, n, e, seed=k * 1000 + e * 10 + n % 7)


def test_interlace_many_planes_and_unaligned(lr, orc):
    check_interlace(lr, orc, 256, 37, 4, seed=1)
    check_interlace(lr, orc, 100, 513, 1, seed=2)
    for k in (2, 3, 4, 8):
        offs = [(4 * j + 4) % 16 for j in range(k + 1)]
        check_interlace(lr, orc, k, 3001, 4, offs, seed=3 + k)
        offs = [(j + 1) % 16 for j in range(k + 1)]
        check_interlace(lr, orc, k, 3001, 2, offs, seed=4 + k)


# ---------------------------------------------------------------------------
# batched execution

def make_op_buffers(op, offset=0, pool=None):
    """Device inputs (from the op's data seed) and zeroed outputs for one op
    spec, guarded, carved back to back from `pool` when one is given."""
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        n = int(np.prod(op["dims"]))
        src = synth.random_elements(op["data_seed"], n, e)
        return dict(src_np=src, src=to_dev(src, offset, pool), dst=DevBuf(n * e, offset, fill=0, pool=pool))
    if op["kind"] == "reorder":
        n = op["n"]
        src = synth.random_elements(op["data_seed"], n, e)
        idx = synth.random_permutation(op["data_seed"] ^ 1, n)
        return dict(src_np=src, idx_np=idx, src=to_dev(src, offset, pool), idx=to_dev(idx, 0, pool),
                    dst=DevBuf(n * e, offset, fill=0, pool=pool))
    k, n = op["k"], op["n"]
    if op["kind"] == "interlace":
        planes = [synth.random_elements(op["data_seed"] + j, n, e) for j in range(k)]
        return dict(planes_np=planes, planes=[to_dev(p, offset, pool) for p in planes],
                    dst=DevBuf(n * k * e, offset, fill=0, pool=pool))
    arr = synth.random_elements(op["data_seed"], n * k, e)
    return dict(src_np=arr, src=to_dev(arr, offset, pool),
                dsts=[DevBuf(n * e, offset, fill=0, pool=pool) for _ in range(k)])


def add_to_plan(plan, op, b):
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        plan.add_permute(b["dst"].ptr, b["src"].ptr, e, op["dims"], op["perm"])
    elif op["kind"] == "reorder":
        plan.add_reorder(b["dst"].ptr, b["src"].ptr, b["idx"].ptr, op["n"], e)
    elif op["kind"] == "interlace":
        plan.add_interlace(b["dst"].ptr, [p.ptr for p in b["planes"]], op["n"], e)
    else:
        plan.add_deinterlace([d.ptr for d in b["dsts"]], b["src"].ptr, op["n"], e)


def oracle_of(orc, op, b):
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        return [orc.permute(b["src_np"], e, op["dims"], op["perm"])]
    if op["kind"] == "reorder":
        return [orc.reorder(b["src_np"], b["idx_np"], e)]
    if op["kind"] == "interlace":
        return [orc.interlace(b["planes_np"], op["n"], e)]
    return orc.deinterlace(b["src_np"], op["k"], op["n"], e)


def outputs_of(op, b):
    if op["kind"] == "deinterlace":
        return [d.download() for d in b["dsts"]]
    return [b["dst"].download()]


def test_batch_mix_matches_oracle(lr, orc):
    ops = synth.batch_mix(seed=5, n_ops=160, hi_total=2 ** 15)
    pool = DevPool()
    bufs = [make_op_buffers(op, offset=(i % 3) * 4, pool=pool) for i, op in enumerate(ops)]
    plan = lr.Plan()
    for op, b in zip(ops, bufs):
        add_to_plan(plan, op, b)
    plan.finalize()
    for rep in range(2):  # the second replay must give the same bytes
        for b in bufs:
            for out in ([b["dst"]] if "dst" in b else b["dsts"]):
                out.view.fill_(0)
        plan.run()
        sync()
        pool.check()
        for i, (op, b) in enumerate(zip(ops, bufs)):
            want = oracle_of(orc, op, b)
            got = outputs_of(op, b)
            for w, gg in zip(want, got):
                assert np.array_equal(gg, w), (rep, i, op)
    plan.close()


def test_batch_rereads_inputs_on_replay(lr, orc):
    """A replay reads the buffers' current contents (the plan records pointers)."""
    op = dict(kind="permute", elem_bytes=4, dims=[37, 70, 5], perm=[2, 0, 1], data_seed=1)
    b = make_op_buffers(op)
    plan = lr.Plan()
    add_to_plan(plan, op, b)
    plan.finalize()
    plan.run()
    sync()
    assert np.array_equal(b["dst"].download(), orc.permute(b["src_np"], 4, op["dims"], op["perm"]))
    new = synth.random_elements(999, 37 * 70 * 5, 4)
    b["src"].upload(new)
    plan.run()
    sync()
    assert np.array_equal(b["dst"].download(), orc.permute(new, 4, op["dims"], op["perm"]))
    plan.close()


def test_batch_equals_single_calls(lr, orc):
    ops = synth.batch_mix(seed=9, n_ops=48, hi_total=2 ** 16)
    p1, p2 = DevPool(), DevPool()
    b1 = [make_op_buffers(op, pool=p1) for op in ops]
    b2 = [make_op_buffers(op, pool=p2) for op in ops]
    plan = lr.Plan()
    for op, b in zip(ops, b1):
        add_to_plan(plan, op, b)
    plan.finalize()
    plan.run()
    for op, b in zip(ops, b2):
        e = op["elem_bytes"]
        if op["kind"] == "permute":
            lr.permute(b["dst"].ptr, b["src"].ptr, e, op["dims"], op["perm"])
        elif op["kind"] == "reorder":
            lr.reorder(b["dst"].ptr, b["src"].ptr, b["idx"].ptr, op["n"], e)
        elif op["kind"] == "interlace":
            lr.interlace(b["dst"].ptr, [p.ptr for p in b["planes"]], op["n"], e)
        else:
            lr.deinterlace([d.ptr for d in b["dsts"]], b["src"].ptr, op["n"], e)
    sync()
    p1.check()
    p2.check()
    for op, x, y in zip(ops, b1, b2):
        for gx, gy in zip(outputs_of(op, x), outputs_of(op, y)):
            assert np.array_equal(gx, gy), op
    plan.close()


def test_batch_interlace_next_to_shared_memory_bodies(lr, orc):
    """Staged interlaces (k <= 4, 16-byte groups) alternating with runs and
    tile permutes: in one grab a CTA runs a staged interlace and then a body
    that fills shared memory (run offsets, tiles).  Every output must match."""
    ops = []
    for i in range(240):
        if i % 3 == 0:
            ops.append(dict(kind="interlace" if i % 2 else "deinterlace", elem_bytes=4, k=2 + i % 3,
                            n=1024 + 4 * (i % 7), data_seed=i))
        elif i % 3 == 1:
            ops.append(dict(kind="permute", elem_bytes=4, dims=[3 + i % 5, 9, 64], perm=[1, 0, 2], data_seed=i))
        else:
            ops.append(dict(kind="permute", elem_bytes=4, dims=[40, 33 + i % 4], perm=[1, 0], data_seed=i))
    pool = DevPool()
    bufs = [make_op_buffers(op, pool=pool) for op in ops]
    plan = lr.Plan()
    for op, b in zip(ops, bufs):
        add_to_plan(plan, op, b)
    plan.finalize()
    for rep in range(3):
        plan.run()
        sync()
        pool.check()
        for i, (op, b) in enumerate(zip(ops, bufs)):
            for w, g in zip(oracle_of(orc, op, b), outputs_of(op, b)):
                assert np.array_equal(g, w), (rep, i, op)
    plan.close()


def test_batch_many_planes(lr, orc):
    op = dict(kind="interlace", elem_bytes=4, k=12, n=333, data_seed=3)
    op2 = dict(kind="deinterlace", elem_bytes=2, k=9, n=1001, data_seed=4)
    pool = DevPool()
    b, b2 = make_op_buffers(op, pool=pool), make_op_buffers(op2, pool=pool)
    plan = lr.Plan()
    add_to_plan(plan, op, b)
    add_to_plan(plan, op2, b2)
    plan.finalize()
    plan.run()
    sync()
    pool.check()
    assert np.array_equal(outputs_of(op, b)[0], oracle_of(orc, op, b)[0])
    for g, w in zip(outputs_of(op2, b2), oracle_of(orc, op2, b2)):
        assert np.array_equal(g, w)
    plan.close()


# ---------------------------------------------------------------------------
# reorder of sources larger than the L2 (bucketed passes or direct gather,
# chosen on the device from the index locality)

def _l2_case(lr, orc, e, n, idx, seed):
    src = synth.random_elements(seed, n, e)
    s, ix = to_dev(src), to_dev(idx)
    d = DevBuf(n * e, 0, fill=0x3C)
    lr.reorder(d.ptr, s.ptr, ix.ptr, n, e)
    sync()
    got = d.download()
    want = orc.reorder(src, idx, e)
    assert np.array_equal(got, want), (e, n, seed)


@pytest.mark.parametrize("e,kind", [(4, "perm"), (4, "repeat"), (4, "skewed"), (4, "reverse"), (4, "block"),
                                    (8, "perm"), (16, "perm"), (16, "repeat")])
def test_reorder_large_sources(lr, orc, e, kind):
    n = (128 << 20) // e + 4099          # a little over 128 MiB, ragged last tile
    if kind == "perm":
        idx = synth.random_permutation(7 + e, n)
    elif kind == "repeat":
        idx = synth.random_indices(8 + e, n, n)
    elif kind == "skewed":
        idx = synth.random_indices(9, n, 1000)          # every index in one source chunk
    elif kind == "reverse":
        idx = np.arange(n - 1, -1, -1, dtype=np.uint32)
    else:
        m = n - n % 4096
        idx = np.concatenate([synth.block_shuffled_permutation(10, m, 4096),
                              np.arange(m, n, dtype=np.uint32)])
    _l2_case(lr, orc, e, n, idx, seed=e * 100 + len(kind))


@pytest.mark.parametrize("e,kind", [(4, "perm"), (8, "repeat"), (16, "perm")])
def test_reorder_large_sources_l2_scatter(lr, orc, tmp_path, e, kind):
    """The bucketed reorder with its last pass through ~16 MB destination
    chunks in the L2 (the form taken when CTA-sized destination chunks would
    need too many buckets), forced through the tuning table."""
    n = (128 << 20) // e + 4099
    idx = synth.random_permutation(17 + e, n) if kind == "perm" else synth.random_indices(18 + e, n, n)
    t = tmp_path / "l2_scatter.txt"
    t.write_text("reorder_smem_buckets 1\n")
    try:
        lr.tuning_load(str(t))
        _l2_case(lr, orc, e, n, idx, seed=e * 10 + 3)
    finally:
        lr.tuning_load(None)
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


def test_reorder_smem_scatter_chunk_edges(lr, orc):
    """Sources just over 128 MiB whose last 64 KB destination chunk holds one
    element, one tile, and one element short of a full chunk."""
    for e, extra in ((4, 1), (4, 4096), (8, (64 << 10) // 8 - 1), (16, 3)):
        n = (128 << 20) // e + extra
        _l2_case(lr, orc, e, n, synth.random_permutation(extra + e, n), seed=e + extra)


def test_every_tile_shape(lr, orc, tmp_path):
    """Each fast-tile shape (128/256/512-byte rows, 16 KB and 8 KB tiles),
    forced through the tuning table, gives the oracle's bytes on planes with
    ragged edges."""
    shapes = {1: [(128, 16384), (256, 16384)], 2: [(128, 16384), (256, 16384), (512, 16384), (128, 8192)],
              4: [(128, 16384), (256, 16384), (512, 16384), (128, 8192)], 8: [(128, 16384), (256, 16384), (512, 16384)],
              16: [(128, 16384), (256, 16384), (512, 16384)]}
    try:
        for e, cands in shapes.items():
            v = 16 // e
            dims = [5, 7 * 16 * v // 4 + 3 * v, 9 * 16 * v // 4 + v]   # multiples of the vector width, ragged
            for rowb, tb in cands:
                t = tmp_path / f"t{e}_{rowb}_{tb}.txt"
                # the planes are small: switch the thin-plane rule off so the tile runs
                t.write_text(f"rowb {e} 1 2147483647 1 2147483647 {rowb} {tb}\nthin_tile_bytes 1\nthin_tile_cells 1\n")
                lr.tuning_load(str(t))
                d = lr.describe_permute(e, dims, [0, 2, 1])
                assert d["kind"] == "tile" and d["tile_a"] * e == rowb and d["tile_a"] * d["tile_b"] * e == tb, d
                check_permute(lr, orc, 31 * e + rowb + tb, e, dims, [0, 2, 1])
    finally:
        lr.tuning_load(None)
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


THIN = [  # (dims, perm): transpose planes far smaller than a tile
    ([7, 122, 736, 2], [3, 2, 1, 0]),
    ([5, 3, 401, 2], [3, 1, 2, 0]),
    ([1000, 3, 2], [0, 2, 1]),
    ([2, 3, 4, 5, 6, 7], [5, 3, 1, 4, 2, 0]),
    ([3, 17, 2, 9], [1, 3, 0, 2]),
    ([13, 2, 3], [2, 1, 0]),
]


def _table_with(lr, tmp_path, name, extra):
    t = tmp_path / name
    t.write_text(open(lr.DEFAULT_TUNE_TABLE).read() + "\n" + extra + "\n")
    lr.tuning_load(str(t))


@pytest.fixture
def no_box(lr, tmp_path):
    """The committed table with boxes switched off: thin planes run strided."""
    _table_with(lr, tmp_path, "nobox.txt", "box_max_cell_bytes 0")
    yield
    lr.tuning_load(None)
    lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


@pytest.fixture
def all_thin(lr, tmp_path):
    """The committed table with every fast-tile plan counted thin and boxes on,
    so that any plane with long enough runs on both sides runs as boxes."""
    _table_with(lr, tmp_path, "allthin.txt", "thin_tile_bytes 1000000000\nthin_tile_cells 1000000000\n"
                                             "thin_l2_bytes 1000000000000\nbox_min_run_bytes 16\n"
                                             "box_max_cell_bytes 16")
    yield
    lr.tuning_load(None)
    lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


@pytest.mark.parametrize("e", [1, 2, 4, 8, 16])
def test_thin_planes(lr, orc, e):
    for t, (dims, perm) in enumerate(THIN):
        d = lr.describe_permute(e, dims, perm)
        # a thin plane runs as boxes or strided (as the table decides), unless
        # widening over its continuation axes turns it into a plane that
        # fills tiles
        widened = d["kind"] == "tile" and (d["wide_a"] >= 0 or d["wide_b"] >= 0)
        assert d["kind"] in ("box", "strided") or widened, (dims, perm, d)
        for off in (0, e if e < 16 else 0):  # aligned (16-byte stores) and unaligned destination
            check_permute(lr, orc, 300 + t, e, dims, perm, src_off=off, dst_off=off)


@pytest.mark.parametrize("e", [1, 2, 4, 8, 16])
def test_thin_planes_run_strided(lr, orc, e, no_box):
    for t, (dims, perm) in enumerate(THIN):
        d = lr.describe_permute(e, dims, perm)
        widened = d["kind"] == "tile" and (d["wide_a"] >= 0 or d["wide_b"] >= 0)
        assert d["kind"] == "strided" or widened, (dims, perm, d)
        for off in (0, e if e < 16 else 0):
            check_permute(lr, orc, 300 + t, e, dims, perm, src_off=off, dst_off=off)


def test_strided_tail_and_unit_edges(lr, orc, no_box):
    # cell counts around the unit size (256 threads x 16/E cells x 4 steps)
    for e, n_b in ((4, 1023), (4, 1024), (4, 1025), (1, 4097), (8, 511)):
        dims, perm = [n_b, 3, 2], [0, 2, 1]
        assert lr.describe_permute(e, dims, perm)["kind"] == "strided"
        check_permute(lr, orc, n_b, e, dims, perm)


# boxes of whole axes (thin planes): contiguous batches of whole planes, a
# partial axis with a ragged last range, short runs on one side, ranks 2-5
BOX = [  # (dims, perm)
    ([1000, 3, 2], [0, 2, 1]),
    ([64, 3, 5000], [0, 2, 1]),          # NCHW -> NHWC with 3 channels: partial axis, ragged end
    ([3, 20011], [1, 0]),                # one thin transpose, ragged partial axis
    ([20011, 5], [1, 0]),
    ([7, 122, 736, 2], [3, 2, 1, 0]),
    ([2, 10, 7, 74, 3], [4, 2, 1, 0, 3]),
    ([56, 5, 84, 3, 7], [2, 0, 4, 3, 1]),
    ([111, 2, 108, 81], [3, 2, 0, 1]),
    ([5, 2, 425, 25, 2], [0, 2, 3, 1, 4]),
    ([95, 14, 5, 58], [3, 0, 2, 1]),
    ([182, 4, 122], [1, 2, 0]),
    ([8, 234], [1, 0]),
    ([40, 5, 188, 24], [1, 3, 2, 0]),
]


@pytest.mark.parametrize("e", [1, 2, 4, 8, 16])
def test_box_planes(lr, orc, e, all_thin):
    n_box = 0
    for t, (dims, perm) in enumerate(BOX):
        d = lr.describe_permute(e, dims, perm)
        n_box += d["kind"] == "box"
        for so, do in ((0, 0), (e, 0), (0, e), (4 if e < 4 else 0, 8 if e < 8 else 0)):
            if e == 16 and (so or do):
                continue
            check_permute(lr, orc, 700 + t, e, dims, perm, src_off=so, dst_off=do)
    assert n_box >= len(BOX) // 2, n_box


def test_box_random_shapes(lr, orc, all_thin):
    """Random permutes of ranks 2-6 with every tile plan counted thin: boxes
    (and strided copies where a box's runs stay short) against the oracle."""
    g = synth.rng(404)
    kinds = {}
    for t in range(120):
        rank = int(g.integers(2, 7))
        e = ELEMS[t % len(ELEMS)]
        dims = [int(g.integers(1, 3000)) if g.random() < 0.25 else int(g.integers(1, 40)) for _ in range(rank)]
        while int(np.prod(dims)) * e > (2 << 20):
            dims[int(np.argmax(dims))] //= 2
        perm = [int(v) for v in g.permutation(rank)]
        k = lr.describe_permute(e, dims, perm)["kind"]
        kinds[k] = kinds.get(k, 0) + 1
        off = (0, 0) if t % 3 else (e % 16, (2 * e) % 16)
        check_permute(lr, orc, 4000 + t, e, dims, perm, src_off=off[0], dst_off=off[1])
    assert kinds.get("box", 0) >= 30, kinds


def _batch_of_thin_ops(lr, orc):
    ops = [dict(kind="permute", elem_bytes=[1, 2, 4, 8][i % 4], dims=dims, perm=perm, data_seed=i)
           for i, (dims, perm) in enumerate(THIN * 4)]
    ops += [dict(kind="permute", elem_bytes=[1, 2, 4, 8, 16][i % 5], dims=dims, perm=perm, data_seed=50 + i)
            for i, (dims, perm) in enumerate(BOX) if int(np.prod(dims)) <= 1 << 18]
    ops += [dict(kind="permute", elem_bytes=4, dims=[64, 96], perm=[1, 0], data_seed=99)]  # a tile op
    pool = DevPool()
    bufs = [make_op_buffers(op, offset=(i % 2) * 4, pool=pool) for i, op in enumerate(ops)]
    plan = lr.Plan()
    for op, b in zip(ops, bufs):
        add_to_plan(plan, op, b)
    plan.finalize()
    for rep in range(2):
        plan.run()
        sync()
        pool.check()
        for i, (op, b) in enumerate(zip(ops, bufs)):
            for w, g in zip(oracle_of(orc, op, b), outputs_of(op, b)):
                assert np.array_equal(g, w), (rep, i, op)
    plan.close()


def test_batch_with_box_ops(lr, orc, all_thin):
    _batch_of_thin_ops(lr, orc)


def test_batch_with_strided_ops(lr, orc, no_box):
    _batch_of_thin_ops(lr, orc)


def test_runs_in_input_order(lr, orc, tmp_path):
    """Short runs walked in input order (tuning knob runs_mirror_bytes) give
    the oracle's bytes: dense permutes whose innermost axis is unmoved, any
    element size, aligned and unaligned."""
    t = tmp_path / "mirror.txt"
    t.write_text(open(lr.DEFAULT_TUNE_TABLE).read() + "\nruns_mirror_bytes 4096\nruns_tile_max_bytes 1\n")
    cases = [([64, 128, 40, 64], [0, 2, 1, 3], 2), ([33, 17, 5, 64], [2, 1, 0, 3], 2), ([7, 9, 11, 32], [1, 2, 0, 3], 4),
             ([5, 300, 16], [1, 0, 2], 8), ([3, 4, 5, 6, 16], [4, 3, 1, 0, 2], 12), ([100, 3, 128], [1, 0, 2], 1)]
    try:
        lr.tuning_load(str(t))
        for i, (dims, perm, e) in enumerate(cases):
            perm = list(perm)
            if perm[-1] != len(dims) - 1:
                continue
            d = lr.describe_permute(e, dims, perm)
            assert d["kind"] == "runs", (dims, perm, d)
            for off in (0, 1 if e in (1, 12) else e):
                check_permute(lr, orc, 700 + i, e, dims, perm, src_off=off, dst_off=off)
    finally:
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


# ---------------------------------------------------------------------------
# widened planes: a short transpose plane spans several planes along the axis
# that continues its input rows (A) and/or its output runs (B)

WIDE = [  # (dims, perm, E, widened sides)
    ([16, 24, 40, 16], [3, 2, 1, 0], 4, "ab"),
    ([8, 5, 37, 32], [3, 2, 1, 0], 2, "ab"),      # ragged continuation extents
    ([32, 12, 10, 16], [2, 1, 3, 0], 4, "a"),
    ([16, 6, 10, 16], [2, 3, 1, 0], 4, "b"),
    ([64, 32, 48, 32], [3, 2, 1, 0], 1, "ab"),
    ([32, 9, 11, 32], [3, 2, 1, 0], 8, "ab"),
    ([16, 7, 13, 16], [3, 2, 1, 0], 16, "ab"),
    ([64, 33, 17, 64], [3, 2, 0, 1], 2, "a"),
    ([3, 64, 20, 64], [0, 3, 2, 1], 2, "a"),
    ([64, 6, 10, 64], [2, 3, 1, 0], 2, "b"),
    # A's extent not a multiple of a 16-byte chunk's elements: the store
    # phase splits every element's coordinate on its own
    ([9, 10, 11, 7], [3, 2, 1, 0], 4, "ab"),      # 4-byte loads (77-element rows)
    ([9, 10, 4, 7], [3, 2, 1, 0], 4, "ab"),       # 16-byte loads (28-element rows)
    ([5, 6, 13, 3], [3, 2, 1, 0], 2, "ab"),
    ([5, 6, 13, 3], [3, 2, 1, 0], 1, "ab"),
    ([5, 6, 13, 3], [3, 2, 1, 0], 8, "ab"),
    ([40, 3, 25, 5], [3, 1, 2, 0], 4, "a"),
]


def wide_sides(d):
    return ("a" if d["wide_a"] >= 0 else "") + ("b" if d["wide_b"] >= 0 else "")


@pytest.fixture
def no_thin_rule(lr, tmp_path):
    """The committed table with the thin-plane rule switched off, so that the
    small test planes run as (widened) tiles whatever its thresholds."""
    t = tmp_path / "no_thin.txt"
    t.write_text(open(lr.DEFAULT_TUNE_TABLE).read() + "\nthin_tile_bytes 1\nthin_tile_cells 1\n")
    lr.tuning_load(str(t))
    yield
    lr.tuning_load(None)
    lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


@pytest.mark.parametrize("case", range(len(WIDE)))
def test_widened_planes(lr, orc, case, no_thin_rule):
    dims, perm, e, sides = WIDE[case]
    d = lr.describe_permute(e, dims, perm)
    assert d["kind"] == "tile" and wide_sides(d) == sides, d
    check_permute(lr, orc, 800 + case, e, dims, perm)
    # an unaligned destination keeps the plane as it is (no widening)
    off = e if e < 16 else 4
    check_permute(lr, orc, 850 + case, e, dims, perm, dst_off=off)


def test_every_widened_tile_shape(lr, orc, tmp_path):
    """Each 16 KB and 32 KB shape forced on widened planes through the tuning
    table (rules for widened planes) gives the oracle's bytes."""
    cases = {1: ([48, 7, 9, 64], [3, 2, 1, 0]), 2: ([32, 7, 9, 64], [3, 2, 1, 0]), 4: ([16, 7, 9, 32], [3, 2, 1, 0]),
             8: ([16, 7, 9, 16], [3, 2, 1, 0]), 16: ([8, 7, 9, 8], [3, 2, 1, 0])}
    try:
        for e, (dims, perm) in cases.items():
            for rowb in (128, 256, 512):
                for tb in (16384, 32768):
                    if (e == 1 and rowb == 512) or (tb == 32768 and not (rowb in (128, 256) if e <= 2 else rowb in (256, 512))):
                        continue
                    t = tmp_path / f"w{e}_{rowb}_{tb}.txt"
                    t.write_text(f"rowb {e} 1 2147483647 1 2147483647 {rowb} {tb} 1\nthin_tile_bytes 1\nthin_tile_cells 1\n"
                                 "double_tile_min_bytes 1\n")
                    lr.tuning_load(str(t))
                    d = lr.describe_permute(e, dims, perm)
                    assert d["kind"] == "tile" and wide_sides(d) == "ab", d
                    assert d["tile_a"] * e == rowb and d["tile_a"] * d["tile_b"] * e == tb, d
                    check_permute(lr, orc, 31 * e + rowb + tb, e, dims, perm)
    finally:
        lr.tuning_load(None)
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)


def test_widened_planes_in_a_batch(lr, orc):
    """Widened planes (32 KB tiles in single calls) run in the batched kernel
    with the 16 KB tile of the same row length."""
    ops = [dict(kind="permute", elem_bytes=e, dims=dims, perm=perm, data_seed=900 + i)
           for i, (dims, perm, e, _) in enumerate(WIDE)]
    ops += [dict(kind="permute", elem_bytes=2, dims=[64, 16, 24, 64], perm=[3, 2, 1, 0], data_seed=999)]
    pool = DevPool()
    bufs = [make_op_buffers(op, offset=0, pool=pool) for op in ops]
    plan = lr.Plan()
    for op, b in zip(ops, bufs):
        add_to_plan(plan, op, b)
    plan.finalize()
    for rep in range(2):
        plan.run()
        sync()
        pool.check()
        for i, (op, b) in enumerate(zip(ops, bufs)):
            for w, g in zip(oracle_of(orc, op, b), outputs_of(op, b)):
                assert np.array_equal(g, w), (rep, i, op)
    plan.close()


# blocked runs: unmoved inner runs of 128 bytes up to 1 KB on a transpose
# plane, copied in blocks of cells (no shared memory)
BLOCKED = [  # (dims, perm, E)
    ([64, 128, 40, 64], [2, 1, 0, 3], 2),
    ([33, 17, 5, 64], [2, 1, 0, 3], 2),       # ragged blocks
    ([7, 9, 11, 32], [1, 2, 0, 3], 4),
    ([5, 300, 16], [1, 0, 2], 8),
    ([3, 4, 5, 6, 16], [4, 3, 1, 0, 2], 12),   # 12-byte elements, 4-byte words
    ([100, 3, 128], [1, 0, 2], 1),
    ([30, 20, 3, 96], [1, 0, 2, 3], 4),       # 1152-byte runs (3 x 96 x 4): the runs kernel
    ([40, 50, 7, 48], [2, 1, 0, 3], 4),       # 192-byte runs
]


@pytest.mark.parametrize("case", range(len(BLOCKED)))
def test_blocked_runs(lr, orc, case):
    dims, perm, e = BLOCKED[case]
    d = lr.describe_permute(e, dims, perm)
    for off in (0, 1 if e in (1, 12) else e):
        check_permute(lr, orc, 950 + case, e, dims, perm, src_off=off, dst_off=off)
    if perm[-1] == len(dims) - 1:  # an unmoved inner run: blocked below 1 KB, the runs kernel above
        assert d["kind"] == ("tile_cells" if 128 <= d["cell_bytes"] < 1024 else "runs"), d


def test_blocked_runs_in_a_batch(lr, orc):
    ops = [dict(kind="permute", elem_bytes=e, dims=dims, perm=perm, data_seed=960 + i)
           for i, (dims, perm, e) in enumerate(BLOCKED)]
    pool = DevPool()
    bufs = [make_op_buffers(op, offset=4 * (i % 2), pool=pool) for i, op in enumerate(ops)]
    plan = lr.Plan()
    for op, b in zip(ops, bufs):
        add_to_plan(plan, op, b)
    plan.finalize()
    plan.run()
    sync()
    pool.check()
    for i, (op, b) in enumerate(zip(ops, bufs)):
        for w, g in zip(oracle_of(orc, op, b), outputs_of(op, b)):
            assert np.array_equal(g, w), (i, op)
    plan.close()

