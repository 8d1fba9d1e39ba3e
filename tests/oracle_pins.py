"""Checks that pin the CPU oracle to facts outside itself.

Each ``pin_*`` function takes an oracle instance and returns a list of failure
messages (empty when the pin holds).  ``test_oracle.py`` runs them against the
committed oracle (all must hold) and against copies of the oracle with a
planted mistake (at least one must fail for every planted mistake).

The facts used, none of which re-types the oracle's own formula:
  * brute-force SCATTER enumeration (input index -> output position), the
    opposite direction to the oracle's gather loop nest;
  * numpy's transpose / fancy indexing / stack / reshape as library routines;
  * textbook special cases: the 2-D matrix transpose B[c][r] = A[r][c], the
    identity order "[0 1 2] = memcpy" (arXiv:1011.3583 Table 1), the complex
    number split into real and imaginary planes (Sec. III.C);
  * invariants: a permute followed by its inverse is the identity, a double
    transpose is the identity, interlace then de-interlace restores the
    planes, the output of a permute is a bijection of the input elements.
"""
from __future__ import annotations

import itertools
from typing import List

import numpy as np

import synth

ELEM_SIZES = (1, 2, 3, 4, 6, 8, 12, 16)


def _void(e: int) -> np.dtype:
    return np.dtype((np.void, e))


def _as_elems(flat: np.ndarray, e: int, dims) -> np.ndarray:
    return flat.view(_void(e)).reshape(dims)


def _inverse(perm):
    inv = [0] * len(perm)
    for i, p in enumerate(perm):
        inv[p] = i
    return inv


def scatter_permute(src_flat: np.ndarray, e: int, dims, perm) -> np.ndarray:
    """Brute force in the other direction: walk every INPUT multi-index x and
    place its element at the output multi-index (x[perm[0]], ..., x[perm[r-1]])."""
    rank = len(dims)
    od = [dims[p] for p in perm]
    total = int(np.prod(dims, dtype=np.int64)) if rank else 0
    out = np.zeros(total * e, dtype=np.uint8)
    in_lin = 0
    for x in itertools.product(*[range(d) for d in dims]):
        y = [x[perm[i]] for i in range(rank)]
        pos = 0
        for i in range(rank):
            pos = pos * od[i] + y[i]
        out[pos * e:(pos + 1) * e] = src_flat[in_lin * e:(in_lin + 1) * e]
        in_lin += 1
    return out


def pin_bruteforce_small(orc) -> List[str]:
    """Every perm of rank 1..4 on small extents (incl. 1 and 0), rank 5 on all
    perms of a 2x1x3x2x2 box, and ranks 6..8 on sampled perms; elem sizes vary."""
    fails = []
    g = synth.rng(11)
    cases = []
    shapes = {1: [(5,), (1,), (0,)], 2: [(3, 4), (1, 5), (4, 1)], 3: [(2, 3, 4), (3, 1, 2)],
              4: [(2, 3, 2, 3), (1, 2, 1, 3)], 5: [(2, 1, 3, 2, 2)]}
    for rank, shs in shapes.items():
        for sh in shs:
            for perm in itertools.permutations(range(rank)):
                cases.append((list(sh), list(perm)))
    for rank in (6, 7, 8):
        for _ in range(6):
            sh = [int(g.integers(1, 3)) for _ in range(rank)]
            sh[int(g.integers(0, rank))] = 3
            cases.append((sh, [int(v) for v in g.permutation(rank)]))
    for ci, (dims, perm) in enumerate(cases):
        e = ELEM_SIZES[ci % len(ELEM_SIZES)]
        n = int(np.prod(dims, dtype=np.int64))
        src = synth.random_elements(1000 + ci, n, e, special=False)
        got = orc.permute(src, e, dims, perm)
        want = scatter_permute(src, e, dims, perm)
        if not np.array_equal(got, want):
            fails.append(f"brute force dims={dims} perm={perm} e={e}")
    return fails


def pin_numpy_transpose(orc) -> List[str]:
    """numpy.transpose(...).copy() as an independent library routine."""
    fails = []
    g = synth.rng(12)
    for t in range(40):
        rank = int(g.integers(1, 9))
        dims = [int(g.integers(1, 6)) for _ in range(rank)]
        while int(np.prod(dims)) > 20000:
            dims[int(np.argmax(dims))] -= 1
        perm = [int(v) for v in g.permutation(rank)]
        e = ELEM_SIZES[t % len(ELEM_SIZES)]
        n = int(np.prod(dims, dtype=np.int64))
        src = synth.random_elements(2000 + t, n, e)
        want = np.ascontiguousarray(_as_elems(src, e, dims).transpose(perm)).reshape(-1).view(np.uint8)
        got = orc.permute(src, e, dims, perm)
        if not np.array_equal(got, want):
            fails.append(f"numpy transpose dims={dims} perm={perm} e={e}")
    return fails


def pin_matrix_transpose(orc) -> List[str]:
    """2-D perm (1, 0) is the matrix transpose B[c][r] = A[r][c]."""
    fails = []
    for (r, c, e) in [(2, 3, 4), (5, 7, 1), (1, 9, 2), (16, 3, 8), (33, 65, 4)]:
        src = synth.random_elements(r * 100 + c, r * c, e, special=False)
        A = src.reshape(r, c, e)
        got = orc.permute(src, e, [r, c], [1, 0]).reshape(c, r, e)
        ok = all(np.array_equal(got[j, i], A[i, j]) for i in range(r) for j in range(c))
        if not ok:
            fails.append(f"matrix transpose {r}x{c} e={e}")
    # A worked example by hand: [[0 1 2] [3 4 5]] -> [[0 3] [1 4] [2 5]].
    src = np.arange(6, dtype=np.uint32)
    got = orc.permute(src, 4, [2, 3], [1, 0]).view(np.uint32)
    if got.tolist() != [0, 3, 1, 4, 2, 5]:
        fails.append("hand-worked 2x3 transpose")
    return fails


def pin_identity_is_memcpy(orc) -> List[str]:
    """The identity order is a plain copy ("[0 1 2] memcpy", Table 1)."""
    fails = []
    for dims in ([4, 5, 6], [7], [2, 3, 4, 5, 1, 2], [3, 3, 3, 3, 3, 3, 3, 2]):
        for e in (1, 4, 12):
            n = int(np.prod(dims))
            src = synth.random_elements(n + e, n, e)
            got = orc.permute(src, e, dims, list(range(len(dims))))
            if not np.array_equal(got, src):
                fails.append(f"identity dims={dims} e={e}")
    return fails


def pin_inverse_roundtrip(orc) -> List[str]:
    """permute(permute(x, p), p^-1) == x and a double transpose is the identity."""
    fails = []
    g = synth.rng(13)
    for t in range(30):
        rank = int(g.integers(2, 9))
        dims = [int(g.integers(1, 5)) for _ in range(rank)]
        perm = [int(v) for v in g.permutation(rank)]
        e = ELEM_SIZES[t % len(ELEM_SIZES)]
        n = int(np.prod(dims))
        src = synth.random_elements(3000 + t, n, e)
        mid = orc.permute(src, e, dims, perm)
        back = orc.permute(mid, e, [dims[p] for p in perm], _inverse(perm))
        if not np.array_equal(back, src):
            fails.append(f"inverse roundtrip dims={dims} perm={perm}")
    for (r, c) in [(3, 5), (64, 31)]:
        src = synth.random_elements(r + c, r * c, 4)
        tt = orc.permute(orc.permute(src, 4, [r, c], [1, 0]), 4, [c, r], [1, 0])
        if not np.array_equal(tt, src):
            fails.append(f"double transpose {r}x{c}")
    return fails


def pin_bijection(orc) -> List[str]:
    """On tagged inputs (element i holds i) the output tags are a permutation
    of 0..n-1, and each lands where the output multi-index says."""
    fails = []
    g = synth.rng(14)
    for t in range(20):
        rank = int(g.integers(2, 7))
        dims = [int(g.integers(1, 7)) for _ in range(rank)]
        perm = [int(v) for v in g.permutation(rank)]
        n = int(np.prod(dims))
        src = synth.tagged_elements(n, 4)
        out = orc.permute(src, 4, dims, perm).view(np.uint32)
        if not np.array_equal(np.sort(out), np.arange(n, dtype=np.uint32)):
            fails.append(f"bijection dims={dims} perm={perm}")
            continue
        # tag -> input multi-index; its output coordinates must be x[perm].
        xs = np.stack(np.unravel_index(out.astype(np.int64), dims), axis=-1)
        ys = np.stack(np.unravel_index(np.arange(n), [dims[p] for p in perm]), axis=-1)
        if not np.array_equal(xs[:, perm], ys):
            fails.append(f"tag placement dims={dims} perm={perm}")
    return fails


def pin_paper_rank3_orders(orc) -> List[str]:
    """The six orders of the paper's 3-D permute list (Sec. III.B) on a
    non-cubic box: all distinct results except the identity, which is memcpy."""
    fails = []
    dims = [2, 3, 5]
    src = synth.tagged_elements(30, 4)
    seen = set()
    for perm in itertools.permutations(range(3)):
        out = orc.permute(src, 4, dims, list(perm))
        want = np.ascontiguousarray(src.view(np.uint32).reshape(dims).transpose(perm)).reshape(-1)
        if not np.array_equal(out.view(np.uint32), want):
            fails.append(f"rank-3 order {perm}")
        seen.add(out.tobytes())
    if len(seen) != 6:
        fails.append("rank-3 orders not all distinct")
    return fails


def pin_sample_matches_full(orc) -> List[str]:
    """The pointwise evaluation equals the full permute at every index."""
    fails = []
    g = synth.rng(15)
    for t in range(10):
        rank = int(g.integers(1, 9))
        dims = [int(g.integers(1, 5)) for _ in range(rank)]
        perm = [int(v) for v in g.permutation(rank)]
        e = ELEM_SIZES[t % len(ELEM_SIZES)]
        n = int(np.prod(dims))
        src = synth.random_elements(4000 + t, n, e)
        full = orc.permute(src, e, dims, perm)
        lin = np.arange(n, dtype=np.int64)[::-1].copy()
        samp = orc.permute_sample(src, e, dims, perm, lin)
        if not np.array_equal(samp, full.reshape(n, e)[lin].reshape(-1)):
            fails.append(f"sample dims={dims} perm={perm}")
        # numpy pins the pointwise evaluation directly too
        want = np.ascontiguousarray(_as_elems(src, e, dims).transpose(perm)).reshape(-1)
        if not np.array_equal(samp.view(_void(e)), want[lin]):
            fails.append(f"sample vs numpy dims={dims} perm={perm}")
    return fails


def pin_reorder(orc) -> List[str]:
    """Gather dst[i] = src[idx[i]] against numpy fancy indexing, with repeats,
    the identity sequence and a permutation followed by its inverse."""
    fails = []
    for t, (n, e) in enumerate([(1, 4), (7, 1), (100, 2), (257, 8), (1000, 12), (4096, 4)]):
        src = synth.random_elements(5000 + t, n, e)
        se = src.view(_void(e))
        idx = synth.random_indices(5100 + t, n, n)
        if not np.array_equal(orc.reorder(src, idx, e).view(_void(e)), se[idx.astype(np.int64)]):
            fails.append(f"reorder fancy-index n={n} e={e}")
        ident = np.arange(n, dtype=np.uint32)
        if not np.array_equal(orc.reorder(src, ident, e), src):
            fails.append(f"reorder identity n={n}")
        p = synth.random_permutation(5200 + t, n)
        inv = np.empty_like(p)
        inv[p] = np.arange(n, dtype=np.uint32)
        if not np.array_equal(orc.reorder(orc.reorder(src, p, e), inv, e), src):
            fails.append(f"reorder inverse n={n}")
    # The pointwise evaluation agrees with numpy fancy indexing at sampled positions.
    for t, (n, e) in enumerate([(1, 4), (999, 3), (4096, 8)]):
        src = synth.random_elements(5300 + t, n, e)
        idx = synth.random_indices(5400 + t, n, n)
        pos = synth.random_indices(5500 + t, min(n, 257), n).astype(np.int64)
        want = src.view(_void(e))[idx.astype(np.int64)[pos]]
        if not np.array_equal(orc.reorder_sample(src, idx, e, pos).view(_void(e)), want):
            fails.append(f"reorder sample n={n} e={e}")
    # A hand-worked example: src = [10 20 30 40], idx = [3 0 0 2] -> [40 10 10 30].
    got = orc.reorder(np.array([10, 20, 30, 40], np.uint32), np.array([3, 0, 0, 2], np.uint32), 4)
    if got.view(np.uint32).tolist() != [40, 10, 10, 30]:
        fails.append("hand-worked gather")
    return fails


def pin_interlace(orc) -> List[str]:
    """Interlace = numpy stack on a new innermost axis; de-interlace =
    reshape(n, k) columns; both directions restore each other; k = 1 is a copy;
    the complex split example of Sec. III.C."""
    fails = []
    for t, (k, n, e) in enumerate([(2, 5, 4), (3, 17, 1), (4, 33, 2), (8, 9, 8), (1, 10, 4),
                                   (5, 3, 3), (9, 7, 16), (3, 1, 4)]):
        planes = [synth.random_elements(6000 + 10 * t + j, n, e) for j in range(k)]
        got = orc.interlace(planes, n, e)
        want = np.stack([p.view(_void(e)) for p in planes], axis=-1).reshape(-1)
        if not np.array_equal(got.view(_void(e)), want):
            fails.append(f"interlace k={k} n={n} e={e}")
        back = orc.deinterlace(got, k, n, e)
        if not all(np.array_equal(b, p) for b, p in zip(back, planes)):
            fails.append(f"interlace roundtrip k={k} n={n} e={e}")
        arr = synth.random_elements(6500 + t, n * k, e)
        parts = orc.deinterlace(arr, k, n, e)
        cols = arr.view(_void(e)).reshape(n, k)
        if not all(np.array_equal(parts[j].view(_void(e)), cols[:, j]) for j in range(k)):
            fails.append(f"deinterlace columns k={k} n={n} e={e}")
        if not np.array_equal(orc.interlace(parts, n, e), arr):
            fails.append(f"deinterlace roundtrip k={k} n={n} e={e}")
    # complex64 -> real / imaginary planes (the paper's example of Sec. III.C)
    z = (np.arange(6) + 1j * (100 + np.arange(6))).astype(np.complex64)
    re, im = orc.deinterlace(z.view(np.uint8), 2, 6, 4)
    if not (np.array_equal(re.view(np.float32), z.real) and np.array_equal(im.view(np.float32), z.imag)):
        fails.append("complex split")
    return fails


def pin_rejects_invalid(orc) -> List[str]:
    """Invalid arguments are refused rather than computed."""
    from oracle import OracleError
    fails = []
    bad = [([2, 3], [0, 0]), ([2, 3], [0, 2]), ([2, -1], [1, 0]), ([1] * 9, list(range(9)))]
    for dims, perm in bad:
        try:
            orc.permute(np.zeros(64, np.uint8), 1, dims, perm)
            fails.append(f"accepted dims={dims} perm={perm}")
        except OracleError:
            pass
    try:
        orc.reorder(np.zeros(4, np.uint32), np.array([0, 4, 1, 2], np.uint32), 4)
        fails.append("accepted out-of-range index")
    except OracleError:
        pass
    return fails


def pin_worked_examples(orc) -> List[str]:
    """Hand-worked examples of each operation (tests/golden/worked_examples.json)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_examples.json")
    with open(path) as f:
        ex = json.load(f)
    fails = []
    for c in ex["permute"]:
        got = orc.permute(np.array(c["src"], np.uint32), 4, c["dims"], c["perm"]).view(np.uint32)
        if got.tolist() != c["dst"]:
            fails.append(f"worked permute {c['dims']} {c['perm']}")
    for c in ex["reorder"]:
        got = orc.reorder(np.array(c["src"], np.uint32), np.array(c["idx"], np.uint32), 4)
        if got.view(np.uint32).tolist() != c["dst"]:
            fails.append("worked reorder")
    for c in ex["interlace"]:
        planes = [np.array(p, np.uint32) for p in c["planes"]]
        n = len(c["planes"][0])
        got = orc.interlace(planes, n, 4).view(np.uint32)
        if got.tolist() != c["dst"]:
            fails.append("worked interlace")
        back = orc.deinterlace(np.array(c["dst"], np.uint32), len(planes), n, 4)
        if [b.view(np.uint32).tolist() for b in back] != c["planes"]:
            fails.append("worked de-interlace")
    return fails


def random_box(g, rank_in, max_extent=6):
    """A random N-to-M request: dims, order (kept axes in output order), base, range."""
    dims = [int(g.integers(1, max_extent + 1)) for _ in range(rank_in)]
    rank_out = int(g.integers(1, rank_in + 1))
    order = [int(v) for v in g.permutation(rank_in)[:rank_out]]
    base, rng = [], []
    for a in range(rank_in):
        if a in order:
            b = int(g.integers(0, dims[a]))
            base.append(b)
            rng.append(int(g.integers(0 if dims[a] > 1 and g.random() < 0.05 else 1, dims[a] - b + 1)))
        else:
            base.append(int(g.integers(0, dims[a])))
            rng.append(0)
    return dims, order, base, rng


def nm_numpy(src_flat, e, dims, order, base, rng):
    """numpy slicing: ints for dropped axes, slices for kept ones, then the kept
    axes (in input order) transposed into the requested output order."""
    a = src_flat.view(_void(e)).reshape(dims)
    key, kept = [], []
    for ax in range(len(dims)):
        if ax in order:
            key.append(slice(base[ax], base[ax] + rng[ax]))
            kept.append(ax)
        else:
            key.append(base[ax])
    sub = a[tuple(key)]
    return np.ascontiguousarray(sub.transpose([kept.index(ax) for ax in order])).reshape(-1)


def pin_reorder_nm(orc) -> List[str]:
    """N-to-M reorder (Sec. III.B) against numpy slicing + transpose, against a
    scatter-side brute force, and its special cases: full box = permute, and a
    rank-1 box = a contiguous range copy (the access of a specified range of
    Sec. III.A)."""
    fails = []
    g = synth.rng(21)
    for t in range(60):
        rank_in = int(g.integers(1, 7))
        dims, order, base, rng = random_box(g, rank_in)
        e = ELEM_SIZES[t % len(ELEM_SIZES)]
        n = int(np.prod(dims))
        src = synth.random_elements(7000 + t, n, e)
        got = orc.reorder_nm(src, e, dims, order, base, rng)
        want = nm_numpy(src, e, dims, order, base, rng)
        if not np.array_equal(got.view(_void(e)), want):
            fails.append(f"nm numpy dims={dims} order={order} base={base} range={rng}")
            continue
        # scatter-side brute force: walk the input box, place each element
        od = [rng[a] for a in order]
        out = np.zeros(int(np.prod(od)) * e, dtype=np.uint8) if od else np.zeros(0, np.uint8)
        boxes = [range(base[a], base[a] + rng[a]) if a in order else [base[a]] for a in range(rank_in)]
        for x in itertools.product(*boxes):
            pos = 0
            for i, a in enumerate(order):
                pos = pos * od[i] + (x[a] - base[a])
            lin = int(np.ravel_multi_index(x, dims))
            out[pos * e:(pos + 1) * e] = src[lin * e:(lin + 1) * e]
        if not np.array_equal(got, out):
            fails.append(f"nm brute force dims={dims} order={order}")
    for t in range(10):  # full box with all axes kept is the permute
        rank = int(g.integers(1, 6))
        dims = [int(g.integers(1, 6)) for _ in range(rank)]
        perm = [int(v) for v in g.permutation(rank)]
        src = synth.random_elements(7500 + t, int(np.prod(dims)), 4)
        if not np.array_equal(orc.reorder_nm(src, 4, dims, perm, [0] * rank, dims), orc.permute(src, 4, dims, perm)):
            fails.append(f"nm full box != permute dims={dims} perm={perm}")
    src = np.arange(100, dtype=np.uint32)
    if orc.reorder_nm(src, 4, [100], [0], [17], [40]).view(np.uint32).tolist() != list(range(17, 57)):
        fails.append("nm range copy")
    return fails


def pin_indexed(orc) -> List[str]:
    """Scatter and 64-bit indices: a scatter by p equals a gather by p^-1;
    numpy fancy assignment out[p] = src (unique indices); 64-bit indices give
    the 32-bit results; the gather form equals oracle_reorder; a hand-worked
    scatter."""
    fails = []
    for t, (n, e) in enumerate([(1, 4), (9, 1), (1000, 3), (4097, 8), (700, 16)]):
        src = synth.random_elements(8000 + t, n, e)
        p = synth.random_permutation(8100 + t, n)
        inv = np.empty_like(p)
        inv[p] = np.arange(n, dtype=np.uint32)
        sc = orc.indexed(src, p, e, scatter=True)
        if not np.array_equal(sc, orc.indexed(src, inv, e, scatter=False)):
            fails.append(f"scatter != gather by inverse n={n}")
        want = np.zeros(n, _void(e))
        want[p.astype(np.int64)] = src.view(_void(e))
        if not np.array_equal(sc.view(_void(e)), want):
            fails.append(f"scatter vs numpy n={n}")
        if not np.array_equal(orc.indexed(src, p.astype(np.uint64), e, scatter=True), sc):
            fails.append(f"scatter64 != scatter32 n={n}")
        g32 = orc.indexed(src, p, e, scatter=False)
        if not np.array_equal(orc.indexed(src, p.astype(np.uint64), e, scatter=False), g32) or \
                not np.array_equal(g32, orc.reorder(src, p, e)):
            fails.append(f"gather64 / gather32 / reorder disagree n={n}")
    got = orc.indexed(np.array([10, 20, 30], np.uint32), np.array([2, 0, 1], np.uint32), 4, scatter=True)
    if got.view(np.uint32).tolist() != [20, 30, 10]:
        fails.append("hand-worked scatter")
    return fails


def pin_stencil2d(orc) -> List[str]:
    """2-D stencil (Sec. III.D) against scipy.ndimage.correlate (a library
    routine, both boundary modes), exactness of the finite-difference
    Laplacians on low-degree polynomials, single-tap shifts and linearity."""
    from scipy import ndimage
    from synth.stencils import fd_laplacian
    fails = []
    g = synth.rng(31)
    for t in range(12):
        ny, nx = int(g.integers(1, 40)), int(g.integers(1, 50))
        R = int(g.integers(0, 5))
        k = int(g.integers(1, 12))
        taps = [(int(g.integers(-R, R + 1)), int(g.integers(-R, R + 1)), float(g.normal())) for _ in range(k)]
        src = g.normal(size=(ny, nx)).astype(np.float32)
        ker = np.zeros((2 * R + 1, 2 * R + 1))
        for dy, dx, w in taps:
            ker[dy + R, dx + R] += w
        for boundary, mode in ((0, "constant"), (1, "nearest")):
            got = orc.stencil2d(src, taps, boundary)
            want = ndimage.correlate(src.astype(np.float64), ker, mode=mode, cval=0.0)
            if not np.allclose(got, want, rtol=1e-12, atol=1e-12):
                fails.append(f"stencil vs scipy {ny}x{nx} R={R} boundary={boundary}")
    yy, xx = np.mgrid[0:24, 0:24].astype(np.float64)
    for order in (1, 2, 3, 4):
        taps = fd_laplacian(order)
        # Laplacian of x^4 + y^2 is 12 x^2 + 2: exact for accuracy >= 4; order
        # 1 (accuracy 2) is exact on degree 3: use x^3 + y^2 (6 x + 2) there.
        f = (xx ** 3 + yy ** 2) if order == 1 else (xx ** 4 + yy ** 2)
        lap = (6 * xx + 2) if order == 1 else (12 * xx ** 2 + 2)
        got = orc.stencil2d(f.astype(np.float32), taps, 0)
        r = order
        inner = (slice(r, 24 - r), slice(r, 24 - r))
        if not np.allclose(got[inner], lap[inner], rtol=0, atol=1e-7):
            fails.append(f"FD Laplacian order {order} not exact on its polynomial")
    src = g.normal(size=(17, 23)).astype(np.float32)
    for dy, dx in ((0, 0), (2, -3), (-1, 4)):
        for boundary in (0, 1):
            got = orc.stencil2d(src, [(dy, dx, 1.0)], boundary)
            want = np.zeros((17, 23))
            for y in range(17):
                for x in range(23):
                    yy2, xx2 = y + dy, x + dx
                    if 0 <= yy2 < 17 and 0 <= xx2 < 23:
                        want[y, x] = src[yy2, xx2]
                    elif boundary == 1:
                        want[y, x] = src[min(max(yy2, 0), 16), min(max(xx2, 0), 22)]
            if not np.array_equal(got, want):
                fails.append(f"shift ({dy},{dx}) boundary {boundary}")
    a = g.normal(size=(15, 19)).astype(np.float32)
    b = g.normal(size=(15, 19)).astype(np.float32)
    taps = fd_laplacian(2)
    lhs = orc.stencil2d((2 * a + b).astype(np.float32), taps, 1)
    rhs = 2 * orc.stencil2d(a, taps, 1) + orc.stencil2d(b, taps, 1)
    if not np.allclose(lhs, rhs, rtol=1e-5, atol=1e-5):
        fails.append("stencil linearity")
    return fails


ALL_PINS = [pin_worked_examples, pin_reorder_nm, pin_indexed, pin_stencil2d, pin_bruteforce_small, pin_numpy_transpose, pin_matrix_transpose,
            pin_identity_is_memcpy, pin_inverse_roundtrip, pin_bijection,
            pin_paper_rank3_orders, pin_sample_matches_full, pin_reorder, pin_interlace,
            pin_rejects_invalid]


def run_all(orc) -> List[str]:
    fails = []
    for pin in ALL_PINS:
        try:
            fails += pin(orc)
        except Exception as ex:  # a crash of a mutant counts as a caught mistake
            fails.append(f"{pin.__name__} raised {type(ex).__name__}: {ex}")
    return fails
