"""Randomised parity of the large index-sequence forms against the oracle.
Sources of 128-170 MiB take the bucketed passes: element sizes 4/8/16,
32- and 64-bit indices, gathers and scatters, random permutations, repeats,
indices confined to a few source chunks, half-local sequences, and both
scatter forms of the gather (CTA-sized destination chunks in shared memory,
or ~16 MB chunks in the L2, forced through the tuning table).  A fixed seed
and a fixed number of draws."""
import numpy as np
import pytest

import oracle
import synth
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


def indices(g, seed, n, kind):
    if kind == "perm":
        return synth.random_permutation(seed, n)
    if kind == "repeat":
        return synth.random_indices(seed, n, n)
    if kind == "few_chunks":  # every index inside one eighth of the source (one or two chunks)
        lo = int(g.integers(0, max(1, n - (n >> 3))))
        return (lo + synth.random_indices(seed, n, min(n - lo, n >> 3))).astype(np.uint32)
    # half-local: a block-shuffled permutation whose entries at a random half
    # of the positions are shuffled among themselves (still a permutation)
    m = n - n % 4096
    p = np.concatenate([synth.block_shuffled_permutation(seed, m, 4096), np.arange(m, n, dtype=np.uint32)])
    a = np.unique(synth.random_indices(seed + 1, n // 2, n))
    p[a] = p[a][synth.random_permutation(seed + 2, a.size)]
    return p


@pytest.mark.parametrize("seed", [1, 2])
def test_large_reorders_match_oracle(lr, tmp_path, seed):
    orc = oracle.get()
    g = np.random.default_rng(100 + seed)
    l2_table = tmp_path / "l2.txt"
    l2_table.write_text("reorder_smem_buckets 1\n")
    fails = []
    try:
        for draw in range(8):
            e = int(g.choice([4, 8, 16]))
            n = int(g.integers((128 << 20) // e, (170 << 20) // e))
            wide, scatter = bool(g.integers(0, 2)), bool(g.integers(0, 2))
            kind = str(g.choice(["perm", "repeat", "few_chunks", "half_local"] if not scatter else
                                ["perm", "half_local"]))  # a scatter's result is unique for permutations
            force_l2 = bool(g.integers(0, 4) == 0)
            idx = indices(g, 1000 * seed + draw, n, kind)
            if wide:
                idx = idx.astype(np.uint64)
            src = synth.random_elements(2000 * seed + draw, n, e)
            lr.tuning_load(str(l2_table) if force_l2 else lr.DEFAULT_TUNE_TABLE)
            s, ix = to_dev(src), to_dev(idx)
            d = DevBuf(n * e, 0, fill=0x6B)
            fn = {(False, False): lr.reorder, (True, False): lr.reorder64, (False, True): lr.scatter,
                  (True, True): lr.scatter64}[(wide, scatter)]
            fn(d.ptr, s.ptr, ix.ptr, n, e)
            sync()
            if not np.array_equal(d.download(), orc.indexed(src, idx, e, scatter=scatter)):
                fails.append((e, n, wide, scatter, kind, force_l2))
            del s, ix, d
    finally:
        lr.tuning_load(None)
        lr.tuning_load(lr.DEFAULT_TUNE_TABLE)
    assert not fails, fails
