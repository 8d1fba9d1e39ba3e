"""Host-side checks of the 2-D stencil call (Sec. III.D) that need no GPU:
validation before any CUDA call, the tap-set classification that picks the
kernel body, the TMA staging rule and the tile count."""
import numpy as np
import pytest

from paper_1011_3583_gb300 import build as rbuild
from synth.stencils import fd_laplacian

FAKE_DST = 0x7F0000000000
FAKE_SRC = 0x7E0000000000


@pytest.fixture(scope="module")
def lr():
    rbuild.build()
    from paper_1011_3583_gb300 import librearr
    librearr.load()
    return librearr


def box(r, w=1.0):
    return [(dy, dx, w) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def cross(r, seed=0):
    g = np.random.default_rng(seed)
    return [(d, 0, float(g.normal())) for d in range(-r, r + 1)] + \
           [(0, d, float(g.normal())) for d in range(-r, r + 1) if d]


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_fd_laplacians_are_crosses(lr, order):
    d = lr.describe_stencil(4096, 4096, fd_laplacian(order))
    assert d["shape"] == "cross" and d["radius"] == order and d["n_unique"] == 4 * order + 1
    assert d["tma"] == 1
    assert d["n_tiles"] == (4096 // d["tile_y"]) * (4096 // d["tile_x"])


@pytest.mark.parametrize("r", range(1, 9))
def test_any_full_cross_is_a_cross(lr, r):
    assert lr.describe_stencil(100, 100, cross(r, r))["shape"] == "cross"


def test_box_family(lr):
    assert lr.describe_stencil(64, 64, box(1))["shape"] == "box"
    assert lr.describe_stencil(64, 64, box(2))["shape"] == "box"
    assert lr.describe_stencil(64, 64, box(3))["shape"] == "generic"     # 49 taps: no blocked body
    assert lr.describe_stencil(64, 64, box(1)[:-1])["shape"] == "generic"  # one tap missing


def test_partial_shapes_are_generic(lr):
    c = cross(2)
    assert lr.describe_stencil(64, 64, c[:-1])["shape"] == "generic"            # a cross arm missing
    assert lr.describe_stencil(64, 64, c + [(1, 1, 0.5)])["shape"] == "generic"  # off-axis tap
    assert lr.describe_stencil(64, 64, [(0, 0, 2.0)])["shape"] == "generic"      # radius 0
    d = lr.describe_stencil(64, 64, [(0, 5, 1.0), (-3, 0, 1.0)])
    assert d["shape"] == "generic" and d["radius"] == 5


def test_repeated_offsets_run_generic(lr):
    # each tap is one term of the sum (merging would change 0*inf + 1*inf)
    taps = fd_laplacian(2) + [(0, 0, 1.0), (2, 0, -0.5)]
    d = lr.describe_stencil(64, 64, taps)
    assert d["shape"] == "generic" and d["n_unique"] == 9 and d["radius"] == 2


def test_generic_body_by_tap_count(lr):
    taps = [(dy, dx, 1.0) for dy in range(-2, 3) for dx in range(-2, 3)]  # a 5x5 box minus a tap
    assert lr.describe_stencil(64, 64, taps[:24])["body"] == "generic_taps"
    d = lr.describe_stencil(64, 64, taps[:24] + [(3, 3, 1.0)])
    assert d["shape"] == "generic" and d["body"] == "generic_columns"
    assert lr.describe_stencil(64, 64, fd_laplacian(3))["body"] == "cross"
    assert lr.describe_stencil(64, 64, box(2))["body"] == "box"


def test_tma_rule(lr):
    taps = fd_laplacian(1)
    assert lr.describe_stencil(64, 64, taps)["tma"] == 1
    assert lr.describe_stencil(64, 66, taps)["tma"] == 0                          # row not 16-byte aligned
    assert lr.describe_stencil(64, 64, taps, 0, FAKE_DST, FAKE_SRC + 4)["tma"] == 0   # src misaligned
    assert lr.describe_stencil(64, 64, taps, 0, FAKE_DST + 8, FAKE_SRC)["tma"] == 0   # dst misaligned


def test_tiles_and_shared_memory(lr):
    d = lr.describe_stencil(257, 130, fd_laplacian(3))
    assert d["n_tiles"] == -(-257 // d["tile_y"]) * -(-130 // d["tile_x"])
    assert d["smem_bytes"] == (d["tile_y"] + 2 * 3) * (d["tile_x"] + 16) * 4
    assert lr.describe_stencil(0, 100, fd_laplacian(1))["n_tiles"] == 0


@pytest.mark.parametrize("args", [
    dict(taps=[]),                                      # no taps
    dict(taps=[(0, 0, 1.0)] * 65),                      # too many taps
    dict(taps=[(9, 0, 1.0)]),                           # beyond radius 8
    dict(taps=[(0, -9, 1.0)]),
    dict(boundary=2),                                   # unknown boundary
    dict(ny=-1),
])
def test_rejects_invalid(lr, args):
    a = dict(ny=16, nx=16, taps=[(0, 0, 1.0)], boundary=0)
    a.update(args)
    with pytest.raises(lr.RearrError) as ex:
        lr.stencil2d(FAKE_DST, FAKE_SRC, a["ny"], a["nx"], a["taps"], a["boundary"])
    assert ex.value.status == lr.EINVAL


def test_rejects_overlap_and_null(lr):
    with pytest.raises(lr.RearrError):
        lr.stencil2d(FAKE_SRC + 64, FAKE_SRC, 16, 16, [(0, 0, 1.0)])
    with pytest.raises(lr.RearrError):
        lr.stencil2d(None, FAKE_SRC, 16, 16, [(0, 0, 1.0)])


def test_empty_grid_launches_nothing(lr):
    n0 = lr.launch_count()
    lr.stencil2d(None, None, 0, 100, fd_laplacian(1))
    lr.stencil2d(None, None, 100, 0, fd_laplacian(1))
    assert lr.launch_count() == n0


def test_inject_wait_timeout_validation(lr):
    with pytest.raises(lr.RearrError):
        lr.inject_wait_timeout(-1)
    lr.inject_wait_timeout(0)
