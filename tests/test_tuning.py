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
