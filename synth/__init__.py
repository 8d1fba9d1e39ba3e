"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Everything here draws random numbers or random shapes; none of it computes a
rearrangement.  All streams come from numpy's PCG64 generator (O'Neill 2014)
seeded with an explicit integer, so every input can be re-created from its seed.

The workloads mirror the paper's (arXiv:1011.3583 Tables 1-3): dense arrays of
random 32-bit patterns (fp32 implied there), rank-3/4 shapes, index sequences
and k-plane interlaces.  The paper used no public dataset, so nothing here
stands in for one.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

# Bit patterns that a kernel doing float arithmetic on the payload would alter:
# quiet/signalling NaNs with payloads, negative zero, denormals, infinities.
SPECIAL_F32 = np.array([0x7FC00001, 0x7F800001, 0xFFC12345, 0x7FBFFFFF, 0x80000000,
                        0x00000001, 0x807FFFFF, 0x7F800000, 0xFF800000], dtype=np.uint32)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_bytes(seed: int, nbytes: int) -> np.ndarray:
    """nbytes uniformly random bytes (uint8)."""
    if nbytes == 0:
        return np.empty(0, dtype=np.uint8)
    return np.frombuffer(rng(seed).bytes(nbytes), dtype=np.uint8).copy()


def random_elements(seed: int, count: int, elem_bytes: int, special: bool = True) -> np.ndarray:
    """count elements of elem_bytes random bytes each, as flat uint8.

    With ``special`` set, a few 4-byte slots are overwritten with the NaN / -0 /
    denormal patterns of SPECIAL_F32, so that a kernel that moved the payload
    through float registers would be caught.
    """
    b = random_bytes(seed, count * elem_bytes)
    if special and b.size >= 4 * len(SPECIAL_F32) * 8:
        words = b[: (b.size // 4) * 4].view(np.uint32)
        pos = rng(seed ^ 0x5EC1A1).choice(words.size, size=len(SPECIAL_F32), replace=False)
        words[pos] = SPECIAL_F32
    return b


def tagged_elements(count: int, elem_bytes: int) -> np.ndarray:
    """Element i holds the little-endian tag i (truncated to elem_bytes bytes).

    With elem_bytes >= 4 and count < 2**32 every tag is distinct, which turns a
    result into a check that the output is a bijection of the input elements.
    """
    out = np.zeros((count, elem_bytes), dtype=np.uint8)
    tags = np.arange(count, dtype=np.uint64)
    for b in range(min(elem_bytes, 8)):
        out[:, b] = ((tags >> np.uint64(8 * b)) & np.uint64(0xFF)).astype(np.uint8)
    return out.reshape(-1)


def random_permutation(seed: int, n: int) -> np.ndarray:
    """Uniform random permutation of 0..n-1 as uint32 (numpy's shuffle)."""
    p = np.arange(n, dtype=np.uint32)
    rng(seed).shuffle(p)
    return p


def block_shuffled_permutation(seed: int, n: int, block: int) -> np.ndarray:
    """Permutation that keeps runs of ``block`` consecutive indices together and
    shuffles the order of the n/block runs (n must be a multiple of block)."""
    assert n % block == 0
    nb = n // block
    order = random_permutation(seed, nb).astype(np.uint64)
    idx = (order[:, None] * np.uint64(block) + np.arange(block, dtype=np.uint64)[None, :])
    return idx.reshape(-1).astype(np.uint32)


def random_indices(seed: int, n: int, high: int) -> np.ndarray:
    """n uniform indices in [0, high) (repeats allowed) as uint32."""
    return rng(seed).integers(0, high, size=n, dtype=np.uint32)


def log_uniform_extent(g: np.random.Generator, lo: int = 1, hi: int = 512) -> int:
    """An integer extent drawn log-uniform in [lo, hi]."""
    v = math.exp(g.uniform(math.log(lo), math.log(hi + 1)))
    return int(min(hi, max(lo, math.floor(v))))


def random_shape(g: np.random.Generator, rank: int, lo_total: int, hi_total: int,
                 lo: int = 1, hi: int = 512) -> List[int]:
    """Extents drawn log-uniform in [lo, hi], resampled until the element total
    lies in [lo_total, hi_total]."""
    while True:
        dims = [log_uniform_extent(g, lo, hi) for _ in range(rank)]
        t = int(np.prod(dims, dtype=np.int64))
        if lo_total <= t <= hi_total:
            return dims


ELEM_CHOICES = (1, 2, 4, 8)


def batch_mix(seed: int, n_ops: int, lo_total: int = 2 ** 8, hi_total: int = 2 ** 22) -> List[Dict]:
    """The uneven batched mix: n_ops independent op specs.

    Kinds are equiprobable among permute (rank 2-5, uniform random perm),
    reorder (uniform random permutation of n) and interlace with k in {2,3,4}
    (interlace or de-interlace with equal odds).  elem_bytes is uniform in
    {1,2,4,8}; every axis extent is log-uniform in [1,512]; each op's element
    total is resampled into [lo_total, hi_total].  Specs hold shapes and seeds
    only; buffers are drawn from ``data_seed`` when needed.
    """
    g = rng(seed)
    ops: List[Dict] = []
    for i in range(n_ops):
        kind = int(g.integers(0, 3))
        e = int(ELEM_CHOICES[int(g.integers(0, len(ELEM_CHOICES)))])
        data_seed = int(g.integers(0, 2 ** 62))
        if kind == 0:
            rank = int(g.integers(2, 6))
            dims = random_shape(g, rank, lo_total, hi_total)
            perm = [int(x) for x in g.permutation(rank)]
            ops.append(dict(kind="permute", elem_bytes=e, dims=dims, perm=perm, data_seed=data_seed))
        elif kind == 1:
            rank = int(g.integers(2, 6))
            n = int(np.prod(random_shape(g, rank, lo_total, hi_total), dtype=np.int64))
            ops.append(dict(kind="reorder", elem_bytes=e, n=n, data_seed=data_seed))
        else:
            k = int(g.integers(2, 5))
            rank = int(g.integers(2, 6))
            total = int(np.prod(random_shape(g, rank, lo_total * k, hi_total), dtype=np.int64))
            n = max(1, total // k)
            direction = "interlace" if int(g.integers(0, 2)) == 0 else "deinterlace"
            ops.append(dict(kind=direction, elem_bytes=e, k=k, n=n, data_seed=data_seed))
    return ops


def op_bytes(op: Dict) -> int:
    """Algorithmic bytes (read + write) of one op spec, index reads included."""
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        n = int(np.prod(op["dims"], dtype=np.int64))
        return 2 * n * e
    if op["kind"] == "reorder":
        return 2 * op["n"] * e + 4 * op["n"]
    return 2 * op["n"] * op["k"] * e


def large_permute(g: np.random.Generator, lo_bytes: int = 256 << 20, hi_bytes: int = 1 << 30) -> Dict:
    """A large rank-3/4 fp32 permute with a uniform random perm whose payload
    lies in [lo_bytes, hi_bytes]; extents are multiples of 16 in [16, 2048]."""
    while True:
        rank = int(g.integers(3, 5))
        dims = [16 * int(g.integers(1, 129)) for _ in range(rank)]
        nbytes = 4 * int(np.prod(dims, dtype=np.int64))
        if lo_bytes <= nbytes <= hi_bytes:
            perm = [int(x) for x in g.permutation(rank)]
            return dict(kind="permute", elem_bytes=4, dims=dims, perm=perm,
                        data_seed=int(g.integers(0, 2 ** 62)))


def poisson_arrivals(seed: int, rate_per_s: float, count: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    gaps = rng(seed).exponential(1.0 / rate_per_s, size=count)
    return np.cumsum(gaps)
