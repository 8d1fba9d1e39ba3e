"""Generic 2-D stencil (Sec. III.D) on the GPU against the oracle.

Tolerance.  The kernel sums the ntaps products with fp32 fused multiply-adds
in its own order (the weights it receives are the float32 values the oracle
also receives).  With u = 2^-24 the standard bound for an FMA-accumulated dot
product of m terms is gamma_m = m u / (1 - m u); for m <= 64 this is below
(m + 1) u, so
    |kernel - exact| <= (ntaps + 1) * u * S,   S = sum_k |w_k| |src(y+dy_k, x+dx_k)|,
plus ntaps * 2^-149 for results that fall into the subnormal range.  S is computed by the oracle
itself, on |src| with |w|, under the same boundary.  The oracle accumulates in
double, whose own error (about ntaps * 2^-53 * S) is far below that bound.
Non-finite results (NaN, +-Inf inputs) must agree in kind.
"""
import numpy as np
import pytest

import oracle
from synth.stencils import fd_laplacian
from tests.gpu_util import DevBuf, sync, to_dev

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


def f32_taps(taps):
    """The weights as the kernel receives them (rounded to float32)."""
    return [(int(dy), int(dx), float(np.float32(w))) for dy, dx, w in taps]


def grid(seed, ny, nx):
    return np.random.default_rng(seed).normal(size=(ny, nx)).astype(np.float32)


def tolerance(orc, src, taps, boundary):
    s = orc.stencil2d(np.abs(src), [(dy, dx, abs(w)) for dy, dx, w in taps], boundary)
    return (len(taps) + 1) * 2.0 ** -24 * s + len(taps) * 2.0 ** -149


def assert_close(got, want, tol, what):
    got = got.astype(np.float64)
    fin = np.isfinite(want)
    assert np.array_equal(np.isnan(got), np.isnan(want)), what
    assert np.array_equal(got[np.isinf(want)], want[np.isinf(want)]), what
    err = np.abs(got[fin] - want[fin])
    bad = err > tol[fin]
    assert not bad.any(), (what, int(bad.sum()), float(err.max()), float(tol[fin][bad].min()))


def run(lr, src, taps, boundary, src_off=0, dst_off=0):
    ny, nx = src.shape
    s = to_dev(src, src_off)
    d = DevBuf(ny * nx * 4, dst_off, fill=0x7F)
    lr.stencil2d(d.ptr, s.ptr, ny, nx, taps, boundary)
    sync()
    return d.download().view(np.float32).reshape(ny, nx)


def check(lr, orc, src, taps, boundary, src_off=0, dst_off=0):
    taps = f32_taps(taps)
    got = run(lr, src, taps, boundary, src_off, dst_off)
    want = orc.stencil2d(src, taps, boundary)
    assert_close(got, want, tolerance(orc, src, taps, boundary), (src.shape, len(taps), boundary, src_off, dst_off))


def random_cross(seed, r):
    g = np.random.default_rng(seed)
    return [(d, 0, float(g.normal())) for d in range(-r, r + 1)] + \
           [(0, d, float(g.normal())) for d in range(-r, r + 1) if d]


def random_box(seed, r):
    g = np.random.default_rng(seed)
    return [(dy, dx, float(g.normal())) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]


def random_taps(seed, k, r):
    g = np.random.default_rng(seed)
    return [(int(g.integers(-r, r + 1)), int(g.integers(-r, r + 1)), float(g.normal())) for _ in range(k)]


# Shapes: single tile, exact tiles, ragged tails in x and y, single rows and
# columns, rows that are and are not 16-byte multiples (TMA and plain staging).
SHAPES = [(1, 1), (1, 4), (1, 1000), (5, 1), (3, 7), (128, 64), (129, 65), (257, 196), (300, 203), (700, 1024)]


@pytest.mark.parametrize("order", [1, 2, 3, 4])
@pytest.mark.parametrize("boundary", [0, 1])
def test_fd_orders(lr, orc, order, boundary):
    for i, (ny, nx) in enumerate(SHAPES):
        check(lr, orc, grid(100 * order + i, ny, nx), fd_laplacian(order), boundary)


@pytest.mark.parametrize("r", range(1, 9))
def test_every_cross_radius(lr, orc, r):
    for boundary in (0, 1):
        for ny, nx in ((259, 200), (131, 77)):
            check(lr, orc, grid(r, ny, nx), random_cross(r, r), boundary)


@pytest.mark.parametrize("r", [1, 2])
def test_boxes(lr, orc, r):
    for boundary in (0, 1):
        for ny, nx in SHAPES:
            check(lr, orc, grid(7 * r, ny, nx), random_box(r, r), boundary)


def test_generic_tap_sets(lr, orc):
    g = np.random.default_rng(5)
    for t in range(24):
        r = int(g.integers(0, 9))
        k = int(g.integers(1, 65))
        taps = random_taps(1000 + t, k, r)  # repeated offsets allowed: each is a term
        ny, nx = SHAPES[t % len(SHAPES)]
        d = lr.describe_stencil(ny, nx, f32_taps(taps))
        assert d["shape"] in ("generic", "cross", "box")
        check(lr, orc, grid(t, ny, nx), taps, t % 2)


@pytest.mark.parametrize("r", range(0, 9))
def test_both_generic_bodies_every_radius(lr, orc, r):
    for k, body in ((11, "generic_taps"), (40, "generic_columns")):
        taps = random_taps(50 + r + k, k, r)
        taps[0] = (r, -r, 0.5)  # reach the radius
        assert lr.describe_stencil(259, 200, f32_taps(taps))["body"] == body
        for boundary in (0, 1):
            check(lr, orc, grid(r + k, 259, 200), taps, boundary)
            check(lr, orc, grid(r + k, 131, 77), taps, boundary)


def test_max_taps_and_radius(lr, orc):
    taps = random_taps(77, 64, 8) + []
    taps[0] = (8, -8, 0.25)
    taps[1] = (-8, 8, -0.5)
    check(lr, orc, grid(3, 300, 300), taps, 0)
    check(lr, orc, grid(3, 300, 300), taps, 1)


@pytest.mark.parametrize("src_off,dst_off", [(4, 0), (0, 4), (8, 12)])
def test_unaligned_pointers_use_plain_staging(lr, orc, src_off, dst_off):
    src = grid(9, 200, 256)
    d = lr.describe_stencil(200, 256, fd_laplacian(2), 0, 0x1000 + dst_off, 0x100000000 + src_off)
    assert d["tma"] == 0
    check(lr, orc, src, fd_laplacian(2), 1, src_off, dst_off)
    check(lr, orc, src, random_taps(4, 20, 3), 0, src_off, dst_off)


def test_special_values(lr, orc):
    src = grid(11, 150, 200)
    g = np.random.default_rng(12)
    pos = g.integers(0, 150 * 200, size=12)
    flat = src.reshape(-1)
    flat[pos[:4]] = np.nan
    flat[pos[4:8]] = np.inf
    flat[pos[8:10]] = -np.inf
    flat[pos[10:]] = -0.0
    for taps in (fd_laplacian(1), fd_laplacian(4), random_box(3, 2), random_taps(8, 30, 5) + [(0, 0, 0.0)]):
        for boundary in (0, 1):
            check(lr, orc, src, taps, boundary)


def test_duplicate_offsets(lr, orc):
    taps = fd_laplacian(2) + [(0, 0, 0.75), (1, 0, -0.125), (0, -2, 2.0)]
    assert lr.describe_stencil(100, 100, f32_taps(taps))["shape"] == "generic"
    check(lr, orc, grid(21, 190, 120), taps, 0)
    check(lr, orc, grid(21, 190, 120), taps, 1)


def test_constant_field(lr, orc):
    # Laplacian of a constant grid is 0 inside; with the clamped boundary it is
    # 0 everywhere (every read sees the same value).
    src = np.full((300, 260), 3.0, dtype=np.float32)
    got = run(lr, src, f32_taps(fd_laplacian(3)), 1)
    tol = tolerance(orc, src, f32_taps(fd_laplacian(3)), 1)
    assert np.all(np.abs(got) <= tol)


def test_no_wait_timed_out(lr):
    assert lr.wait_timeouts() == 0


def test_launches_counted(lr):
    src = grid(1, 64, 64)
    n0 = lr.launch_count()
    run(lr, src, fd_laplacian(1), 0)
    assert lr.launch_count() == n0 + 1


def band_oracle(orc, src, taps, boundary, rows):
    """Oracle rows of a large grid: each output row y from the band of input
    rows y - r .. y + r (cut at the grid's edges, which are the band's edges
    there), so the band's boundary handling matches the grid's."""
    ny = src.shape[0]
    r = max(max(abs(dy), abs(dx)) for dy, dx, _ in taps)
    out, tol = [], []
    for y in rows:
        lo, hi = max(0, y - r), min(ny, y + r + 1)
        band = np.ascontiguousarray(src[lo:hi])
        out.append(orc.stencil2d(band, taps, boundary)[y - lo])
        tol.append(tolerance(orc, band, taps, boundary)[y - lo])
    return np.array(out), np.array(tol)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_table4_grid_4096(lr, orc, order):
    """The 4096 x 4096 float grid of Table 4, orders I-IV, every output."""
    import torch
    src = grid(4096 + order, 4096, 4096)
    taps = f32_taps(fd_laplacian(order))
    s = to_dev(src)
    d = DevBuf(src.nbytes)
    for boundary in (0, 1):
        lr.stencil2d(d.ptr, s.ptr, 4096, 4096, taps, boundary)
        sync()
        got = d.download().view(np.float32).reshape(4096, 4096)
        assert_close(got, orc.stencil2d(src, taps, boundary), tolerance(orc, src, taps, boundary),
                     ("4096", order, boundary))


@pytest.mark.parametrize("order", [1, 4])
def test_large_grid_sampled_rows(lr, orc, order):
    """A 16384 x 16384 grid (1 GiB each way), rows sampled at the edges, at
    tile seams and at random."""
    import torch
    ny = nx = 16384
    gen = torch.Generator(device="cuda").manual_seed(order)
    s = torch.randn((ny, nx), device="cuda", generator=gen, dtype=torch.float32)
    dbuf = DevBuf(ny * nx * 4)
    d = dbuf.view.view(torch.float32).view(ny, nx)
    taps = f32_taps(fd_laplacian(order))
    rows = sorted(set([0, 1, 2, 3, 4, 127, 128, 129, 255, 256, ny - 129, ny - 128, ny - 5, ny - 1] +
                      list(np.random.default_rng(order).integers(0, ny, size=16))))
    for boundary in (0, 1):
        lr.stencil2d(dbuf.ptr, s, ny, nx, taps, boundary)
        sync()
        dbuf.check_guards()
        # only the input rows the sampled outputs read travel to the host
        need = sorted({min(max(y + k, 0), ny - 1) for y in rows for k in range(-order, order + 1)})
        src = np.zeros((ny, nx), dtype=np.float32)
        src[need] = s[need].cpu().numpy()
        want, tol = band_oracle(orc, src, taps, boundary, rows)
        got = d[rows].cpu().numpy()
        assert_close(got, want, tol, ("16384", order, boundary))


def test_injected_wait_timeout_is_reported(lr, orc):
    """A TMA barrier that never completes (16 bytes more expected than the
    copy delivers): the bounded waits run out, the CTA counts a timeout and
    skips its outputs, and the context stays usable for the next call."""
    src = grid(2, 64, 64)
    d = lr.describe_stencil(64, 64, f32_taps(fd_laplacian(1)))
    assert d["n_tiles"] == 1 and d["tma"] == 1
    before = lr.wait_timeouts()
    lr.inject_wait_timeout(1)
    got = run(lr, src, f32_taps(fd_laplacian(1)), 0)
    assert lr.wait_timeouts() == before + 1
    assert np.all(got.view(np.uint32) == 0x7F7F7F7F)  # outputs skipped
    check(lr, orc, src, fd_laplacian(1), 0)            # the next launch is normal
    assert lr.wait_timeouts() == before + 1
