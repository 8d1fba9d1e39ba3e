"""Host-side checks of librearr that need no GPU.

* the shared library loads and exports every function include/librearr.h declares;
* argument validation returns REARR_EINVAL before any CUDA call;
* zero-size operations return REARR_OK and launch nothing;
* the plan compiler's canonical form (collapsed extents, strides, folded cell)
  describes the same permutation: a CPU interpretation of the collapsed plan
  reproduces the oracle's bytes (the oracle itself never collapses axes).
"""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import synth
from paper_1011_3583_gb300 import build as rbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lr():
    rbuild.build()
    from paper_1011_3583_gb300 import librearr
    librearr.load()
    return librearr


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rearr_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lr):
    names = declared_functions()
    assert len(names) >= 19, names
    L = ctypes.CDLL(lr.lib_path())
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_pipeline_rejects_invalid_before_cuda(lr):
    from paper_1011_3583_gb300 import librearr
    for slot_bytes, slots in ((1 << 20, 0), (1 << 20, 9), (0, 3)):
        with pytest.raises(librearr.RearrError) as ex:
            librearr.Pipeline(slot_bytes, slots)
        assert ex.value.status == librearr.EINVAL


def test_check_indices_validation(lr):
    from paper_1011_3583_gb300 import librearr
    for args in ((FAKE_SRC, 16, 3, 16), (None, 16, 4, 16), (FAKE_SRC + 4, 16, 8, 16)):
        with pytest.raises(librearr.RearrError) as ex:
            librearr.check_indices(*args)
        assert ex.value.status == librearr.EINVAL
    assert librearr.check_indices(None, 0, 4, 0) == 0


def test_thin_planes_classify(lr, tmp_path):
    from paper_1011_3583_gb300 import librearr
    # boxes on for every cell size
    t = tmp_path / "box16.txt"
    t.write_text(open(librearr.DEFAULT_TUNE_TABLE).read() + "\nbox_max_cell_bytes 16\nbox_min_run_bytes 16\n")
    librearr.tuning_load(str(t))
    # a thin plane runs as boxes of whole axes: (2 x 7) planes, the box also
    # spans the 122-axis whole and two indices of the 736-axis (16-byte input
    # runs, 1708 x 4 cells written in one run)
    d = librearr.describe_permute(4, [7, 122, 736, 2], [3, 2, 1, 0])
    assert d["kind"] == "box" and d["rank"] == 4, d
    assert (d["tile_a"], d["tile_b"], d["vec_in"], d["vec_out"], d["n_tiles"]) == (4, 1708, 16, 16, 368), d
    # a batch of whole 3 x 2 planes: 682 planes per box, contiguous on both sides
    d = librearr.describe_permute(4, [1000, 3, 2], [0, 2, 1])
    assert d["kind"] == "box" and (d["tile_a"], d["tile_b"], d["n_tiles"]) == (4092, 4092, 2), d
    # the same reversal with a plane that fills tiles stays tiled
    assert librearr.describe_permute(4, [512, 64, 64, 512], [3, 2, 1, 0])["kind"] == "tile"
    # unaligned destination: 4-byte stores
    assert librearr.describe_permute(4, [1000, 3, 2], [0, 2, 1], FAKE_DST + 4, FAKE_SRC)["vec_out"] == 4
    # ... a cells tile of 16-byte cells: one box
    d = lr.describe_permute(4, [8, 16, 4], [1, 0, 2], FAKE_DST, FAKE_SRC)
    assert d["cell_bytes"] == 16 and d["rank"] == 2 and d["kind"] == "box" and d["n_tiles"] == 1
    # boxes switched off (runs must reach more than a tile, or no cell size
    # allowed): strided copies
    for extra in ("box_min_run_bytes 1000000", "box_max_cell_bytes 0"):
        t = tmp_path / "nobox.txt"
        t.write_text(open(librearr.DEFAULT_TUNE_TABLE).read() + "\n" + extra + "\n")
        try:
            librearr.tuning_load(str(t))
            d = librearr.describe_permute(4, [7, 122, 736, 2], [3, 2, 1, 0])
            assert d["kind"] == "strided" and d["vec_out"] == 16 and d["rank"] == 4
            assert librearr.describe_permute(4, [1000, 3, 2], [0, 2, 1], FAKE_DST + 4, FAKE_SRC)["vec_out"] == 4
        finally:
            librearr.tuning_load(None)
            librearr.tuning_load(librearr.DEFAULT_TUNE_TABLE)
    # boxes for cells of at most box_max_cell_bytes
    t = tmp_path / "box2.txt"
    t.write_text(open(librearr.DEFAULT_TUNE_TABLE).read() + "\nbox_max_cell_bytes 2\nbox_min_run_bytes 16\n")
    try:
        librearr.tuning_load(str(t))
        assert librearr.describe_permute(2, [1000, 3, 2], [0, 2, 1])["kind"] == "box"
        assert librearr.describe_permute(4, [1000, 3, 2], [0, 2, 1])["kind"] == "strided"
    finally:
        librearr.tuning_load(None)
        librearr.tuning_load(librearr.DEFAULT_TUNE_TABLE)


def test_status_strings(lr):
    assert [lr.status_str(i) for i in range(7)] == [
        "REARR_OK", "REARR_EINVAL", "REARR_ENOMEM", "REARR_ECUDA", "REARR_ERANGE", "REARR_ETIMEDOUT", "REARR_EBUSY"]


def test_selftest_host(lr):
    lr.selftest_host()


FAKE_DST = 0x7F0000000000
FAKE_SRC = 0x7E0000000000


@pytest.mark.parametrize("dims,perm,e", [
    ([2, 3], [0, 0], 4),          # not a permutation
    ([2, 3], [0, 2], 4),          # out of range
    ([2, -1], [1, 0], 4),         # negative extent
    ([1] * 9, list(range(9)), 4),  # rank > 8
    ([2, 3], [1, 0], 0),          # elem_bytes == 0
])
def test_permute_rejects_invalid(lr, dims, perm, e):
    with pytest.raises(lr.RearrError) as ex:
        lr.permute(FAKE_DST, FAKE_SRC, e, dims, perm)
    assert ex.value.status == 1


def test_permute_rejects_null_and_overlap(lr):
    with pytest.raises(lr.RearrError):
        lr.permute(0, FAKE_SRC, 4, [4, 4], [1, 0])
    with pytest.raises(lr.RearrError):
        lr.permute(FAKE_SRC + 8, FAKE_SRC, 4, [4, 4], [1, 0])


def test_rank_zero_rejected(lr):
    with pytest.raises(lr.RearrError):
        lr.permute(FAKE_DST, FAKE_SRC, 4, [], [])


def test_zero_size_ops_are_noops(lr):
    before = lr.launch_count()
    lr.permute(0, 0, 4, [3, 0, 5], [2, 1, 0])
    lr.reorder(0, 0, 0, 0, 4)
    lr.interlace(0, [0, 0], 0, 4)
    lr.deinterlace([0, 0, 0], 0, 0, 4)
    assert lr.launch_count() == before


def test_other_ops_reject_invalid(lr):
    with pytest.raises(lr.RearrError):
        lr.reorder(FAKE_DST, FAKE_SRC, 0, 16, 4)          # NULL idx
    with pytest.raises(lr.RearrError):
        lr.reorder(FAKE_DST, FAKE_SRC, FAKE_SRC + 3, 16, 4)  # misaligned idx (and overlap)
    with pytest.raises(lr.RearrError):
        lr.reorder(FAKE_DST, FAKE_DST + 4, 0x100000, 16, 4)  # dst overlaps src
    with pytest.raises(lr.RearrError):
        lr.interlace(FAKE_DST, [], 16, 4)                   # k = 0
    with pytest.raises(lr.RearrError):
        lr.interlace(FAKE_DST, [FAKE_SRC] * 257, 16, 4)     # k > 256
    with pytest.raises(lr.RearrError):
        lr.interlace(FAKE_DST, [FAKE_SRC, 0], 16, 4)        # NULL plane
    with pytest.raises(lr.RearrError):
        lr.interlace(FAKE_DST, [FAKE_DST + 16, FAKE_SRC], 16, 4)  # plane inside dst
    with pytest.raises(lr.RearrError):
        lr.deinterlace([FAKE_DST, FAKE_DST + 8], FAKE_SRC, 16, 4)  # destination planes overlap
    with pytest.raises(lr.RearrError):
        lr.interlace(FAKE_DST, [FAKE_SRC, FAKE_SRC + 4096], 16, 0)


def test_plan_finalize_rules(lr):
    p = lr.Plan()
    p.add_permute(0, 0, 4, [0, 7], [1, 0])  # zero-size op is dropped
    assert p.stats() == (0, 0)
    with pytest.raises(lr.RearrError):
        p.add_permute(FAKE_DST, FAKE_SRC, 4, [2, 2], [0, 0])
    p.finalize()   # empty plan: nothing to upload, no CUDA call
    with pytest.raises(lr.RearrError) as ex:
        p.add_permute(FAKE_DST, FAKE_SRC, 4, [2, 2], [1, 0])
    assert ex.value.status == 6
    p.run()        # empty plan replays as a no-op
    p.close()


# --------------------------------------------------------------------------
# Canonical form of the plan compiler.

def test_describe_examples(lr):
    # identity and extent-1 axes collapse to a copy
    d = lr.describe_permute(4, [4, 1, 5, 6], [0, 1, 2, 3], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "copy"
    d = lr.describe_permute(4, [4, 1, 5, 6], [1, 0, 2, 3], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "copy"
    # 2-D transpose: a fast tile on the (A, B) plane
    d = lr.describe_permute(4, [1024, 1024], [1, 0], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "tile" and d["dims"] == [1024, 1024] and d["in_strides"] == [1, 1024]
    assert d["vec_in"] == 16 and d["vec_out"] == 16
    # 64x128x256x64 with (0,1,3,2) is a batch of 8192 transposes of 256 x 64
    d = lr.describe_permute(4, [64, 128, 256, 64], [0, 1, 3, 2], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "tile" and d["dims"] == [8192, 64, 256] and d["plane_a"] == 1
    # unmoved innermost axis folds into the cell (an op past the L2 bound of
    # the thin-plane rule, so that it stays a tile whatever the table says)
    d = lr.describe_permute(4, [2048, 2048, 4], [1, 0, 2], FAKE_DST, FAKE_SRC)
    assert d["cell_bytes"] == 16 and d["rank"] == 2 and d["kind"] == "tile"
    # ... and a plane of 8 x 16 such cells is too thin for tiles
    d = lr.describe_permute(4, [8, 16, 4], [1, 0, 2], FAKE_DST, FAKE_SRC)
    assert d["cell_bytes"] == 16 and d["rank"] == 2 and d["kind"] in ("strided", "box")
    # long unmoved runs are copied as runs
    d = lr.describe_permute(4, [8, 16, 512], [1, 0, 2], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "runs" and d["cell_bytes"] == 2048
    # element sizes that are not a power of two use multi-word cells
    d = lr.describe_permute(12, [33, 65], [1, 0], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "tile_cells" and d["word_bytes"] == 4
    # misaligned base pointers lower the access width
    d = lr.describe_permute(4, [64, 64], [1, 0], FAKE_DST + 2, FAKE_SRC)
    assert d["kind"] == "tile_cells" and d["word_bytes"] == 2
    d = lr.describe_permute(4, [64, 64], [1, 0], FAKE_DST + 4, FAKE_SRC)
    assert d["kind"] == "tile" and d["vec_out"] == 4 and d["vec_in"] == 16
    # ragged extents lower the vector widths, never the correctness
    d = lr.describe_permute(4, [3701, 4219], [1, 0], FAKE_DST, FAKE_SRC)
    assert d["kind"] == "tile" and d["vec_in"] == 4 and d["vec_out"] == 4


def interpret_plan(src_flat: np.ndarray, e: int, info: dict, total: int) -> np.ndarray:
    """Evaluate a collapsed plan on the CPU: output axis i advances the input by
    in_strides[i] cells of cell_bytes bytes; the output is row-major."""
    cell = info["cell_bytes"]
    if info["kind"] == "copy":
        return src_flat.copy()
    dims = info["dims"]
    strides = [s * cell for s in info["in_strides"]]
    view = np.lib.stride_tricks.as_strided(src_flat, shape=tuple(dims) + (cell,),
                                           strides=tuple(strides) + (1,), writeable=False)
    return np.ascontiguousarray(view).reshape(-1)


def test_collapsed_plan_equivalence(lr):
    orc = oracle.get()
    g = synth.rng(77)
    cases = []
    for rank in range(1, 9):
        for _ in range(12):
            dims = [int(g.integers(1, 5)) for _ in range(rank)]
            for _ in range(int(g.integers(0, rank))):
                dims[int(g.integers(0, rank))] = 1
            cases.append((dims, [int(v) for v in g.permutation(rank)]))
    for dims in ([2, 3, 4], [3, 1, 4, 1], [2, 2, 2, 2]):
        for perm in itertools.permutations(range(len(dims))):
            cases.append((list(dims), list(perm)))
    for ci, (dims, perm) in enumerate(cases):
        e = (1, 2, 3, 4, 8, 12, 16, 40)[ci % 8]
        n = int(np.prod(dims))
        src = synth.random_elements(9000 + ci, n, e)
        info = lr.describe_permute(e, dims, perm, FAKE_DST, FAKE_SRC)
        got = interpret_plan(src, e, info, n)
        want = orc.permute(src, e, dims, perm)
        assert np.array_equal(got, want), (dims, perm, e, info)
        # the canonical form never keeps an extent-1 axis and never an unmoved inner axis
        if info["kind"] in ("tile", "tile_cells"):
            assert all(d > 1 for d in info["dims"])
            assert info["in_strides"][-1] != 1


def test_reorder_nm_describe_routes_boxes(lr):
    """N-to-M boxes through the plan compiler, host only: a box that drops the
    input's fastest axis has no input-contiguous axis and, with one-word cells,
    is gathered cell by cell (strided); wider cells stay runs; a kept inner
    axis gives a tile or runs; the full box is the permute's plan."""
    d = lr.describe_reorder_nm(4, [1024, 1024, 256], [0, 1], [0, 0, 5], [1024, 1024, 1])
    assert d["kind"] == "strided" and d["word_bytes"] == 4 and d["vec_out"] == 16
    d = lr.describe_reorder_nm(2, [40, 50, 60], [1, 0], [3, 7, 11], [30, 40, 1])
    assert d["kind"] == "strided" and d["word_bytes"] == 2
    # 12-byte cells are no single word: runs
    assert lr.describe_reorder_nm(12, [40, 50, 60], [1, 0], [3, 7, 11], [30, 40, 1])["kind"] == "runs"
    # unaligned source for 4-byte cells: no 4-byte word, runs
    d = lr.describe_reorder_nm(4, [40, 50, 60], [1, 0], [3, 7, 11], [30, 40, 1], 0, FAKE_SRC + 2)
    assert d["kind"] == "runs"
    # inner axis kept: a transpose plane of the box
    assert lr.describe_reorder_nm(4, [8, 256, 512], [2, 1], [3, 64, 128], [1, 128, 256])["kind"] == "tile"
    # the full box in order (2, 0, 1) is the permute's plan
    full = lr.describe_reorder_nm(4, [33, 70, 65], [2, 0, 1], [0, 0, 0], [33, 70, 65])
    assert full == lr.describe_permute(4, [33, 70, 65], [2, 0, 1])
    with pytest.raises(lr.RearrError):
        lr.describe_reorder_nm(4, [10, 10], [0, 0], [0, 0], [5, 5])


def test_reorder_describe_paths(lr, tmp_path):
    """Which path an index-sequence op takes, host only: small sources and
    unaligned words run the direct kernel; large ones the bucketed passes
    with the shared-memory scatter, the L2 form (huge sources, or forced by
    the tuning table), or the scatter's linear form."""
    n = 1 << 28
    d = lr.describe_reorder(n, 4)
    assert d["form"] == "smem_scatter" and d["bucket_chunks"] == 64 and d["bucket_chunk_elems"] == 1 << 22
    assert d["dest_chunks"] == n >> 14 and d["dest_chunk_elems"] == 1 << 14   # 64 KB of fp32
    # scratch: s-, i- and v-arrays (12 bytes per element) plus the bucket
    # tables and the per-tile segment starts (65 x 2 bytes per 4096 indices)
    assert 12 * n < d["scratch_bytes"] < 12 * n + 20 * (64 * (n >> 14)) + 130 * (n >> 12) + (1 << 20)
    assert lr.describe_reorder(n, 4, idx_bytes=8) == d                       # 64-bit indices: same passes
    s = lr.describe_reorder(n, 4, scatter=True)
    assert s["form"] == "linear_scatter" and s["dest_chunks"] == 1
    assert lr.describe_reorder((128 << 20) // 4 - 1, 4)["form"] == "direct"  # below 128 MiB
    assert lr.describe_reorder(n, 4, src_addr=FAKE_SRC + 2)["form"] == "direct"  # 2-byte words
    assert lr.describe_reorder(n, 12)["form"] == "direct"                    # no 4/8/16-byte word
    for e, dchunk in ((8, 1 << 13), (16, 1 << 12)):
        d = lr.describe_reorder((256 << 20) // e, e)
        assert d["form"] == "smem_scatter" and d["dest_chunk_elems"] == dchunk
    huge = lr.describe_reorder(1 << 31, 4)                                   # 8 GB: too many buckets
    assert huge["form"] == "l2_scatter" and huge["bucket_chunks"] == 512 == huge["dest_chunks"]
    t = tmp_path / "l2.txt"
    t.write_text("reorder_smem_buckets 1\n")
    try:
        lr.tuning_load(str(t))
        assert lr.describe_reorder(n, 4)["form"] == "l2_scatter"
    finally:
        lr.tuning_load(None)
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)
    with pytest.raises(lr.RearrError) as ex:
        lr.describe_reorder(n, 4, idx_bytes=2)
    assert ex.value.status == lr.EINVAL
