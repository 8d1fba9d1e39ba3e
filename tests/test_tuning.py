"""The tuning table steers the plan compiler (host only)."""
import pytest


@pytest.fixture(scope="module")
def rr():
    from paper_1011_3583_gb300 import build
    build.build()
    import paper_1011_3583_gb300 as rr
    rr.load()
    return rr


def test_rowb_rule_changes_tile_shape(rr, tmp_path):
    dims, perm = [100, 64, 64], [0, 2, 1]           # E=4, DA=64, DB=64
    try:
        rr.tuning_load(None)
        assert rr.describe_permute(4, dims, perm)["tile_a"] == 64   # 256-byte rows by default
        t = tmp_path / "t.txt"
        t.write_text("# comment\nrowb 4 33 96 33 96 512   # tuned\nmin_grab 2\n")
        rr.tuning_load(str(t))
        d = rr.describe_permute(4, dims, perm)
        assert d["tile_a"] == 128 and d["tile_b"] == 32    # 512-byte rows
        assert rr.describe_permute(4, [100, 200, 64], perm)["tile_a"] == 64  # DB outside the rule
        assert rr.describe_permute(2, dims, perm)["tile_a"] != 256          # other element size
        with pytest.raises(rr.RearrError):
            rr.tuning_load(str(tmp_path / "missing.txt"))
        assert rr.describe_permute(4, dims, perm)["tile_a"] == 128          # previous table kept
    finally:
        rr.tuning_load(None)


def test_widening_rules_and_knobs(rr, tmp_path):
    """Keys of the table beyond the row length: 32 KB tiles, rules for widened
    planes (8th field), the widening threshold, the blocked-runs knobs and
    the vector-width cap."""
    rank4 = [64, 128, 256, 64]
    try:
        rr.tuning_load(None)
        d = rr.describe_permute(2, rank4, [3, 2, 1, 0])   # 128-byte sides: widened both ways by default
        assert d["kind"] == "tile" and d["wide_a"] == 1 and d["wide_b"] == 2
        t = tmp_path / "t.txt"
        t.write_text("rowb 2 1 100 1 100 256 16384 1\n"        # widened 2-byte planes of 64 x 64: 16 KB, 256-byte rows
                     "rowb 4 1 100 1 100 512 32768 0\n"        # plain 4-byte planes: 32 KB, 512-byte rows
                     "rowb 8 1 100 1 100 128 32768 0\n"        # no such 32 KB shape: ignored
                     "double_tile_min_bytes 1\n")              # 32 KB tiles for ops of any size
        rr.tuning_load(str(t))
        d = rr.describe_permute(2, rank4, [3, 2, 1, 0])
        assert (d["tile_a"], d["tile_b"]) == (128, 64)
        d = rr.describe_permute(4, [8, 64, 64], [0, 2, 1])  # a dense plane: never widened
        assert d["wide_a"] == d["wide_b"] == -1 and (d["tile_a"], d["tile_b"]) == (128, 64)
        t2 = tmp_path / "t2.txt"
        t2.write_text(t.read_text().replace("double_tile_min_bytes 1", "double_tile_min_bytes 1000000"))
        rr.tuning_load(str(t2))                              # a 128 KB op: the 16 KB tile of the same rows
        assert (rr.describe_permute(4, [8, 64, 64], [0, 2, 1])["tile_a"],
                rr.describe_permute(4, [8, 64, 64], [0, 2, 1])["tile_b"]) == (128, 32)
        rr.tuning_load(str(t))
        assert rr.describe_permute(8, [8, 64, 64], [0, 2, 1])["tile_a"] * rr.describe_permute(
            8, [8, 64, 64], [0, 2, 1])["tile_b"] * 8 == 16384
        t.write_text("wide_bytes 1\nruns_tile_max_bytes 1\ntile_vector_bytes 4\n")
        rr.tuning_load(str(t))
        d = rr.describe_permute(2, rank4, [3, 2, 1, 0])
        assert d["wide_a"] == d["wide_b"] == -1 and d["vec_in"] == 4 and d["vec_out"] == 4
        assert rr.describe_permute(2, rank4, [2, 1, 0, 3])["kind"] == "runs"
        t.write_text("runs_tile_max_bytes 1024\nruns_tile_cells 8\nruns_tile_side_bytes 2048\n")
        rr.tuning_load(str(t))
        d = rr.describe_permute(2, rank4, [2, 1, 0, 3])      # 128-byte runs: sides of 2048 / 128 = 16 cells
        assert d["kind"] == "tile_cells" and (d["tile_a"], d["tile_b"]) == (16, 16) and d["cell_bytes"] == 128
        d = rr.describe_permute(8, rank4, [2, 1, 0, 3])      # 512-byte runs: at least 8 cells a side
        assert d["kind"] == "tile_cells" and (d["tile_a"], d["tile_b"]) == (8, 8) and d["cell_bytes"] == 512
    finally:
        rr.tuning_load(None)
