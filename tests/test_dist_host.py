"""Distributed permute (include/librearr_dist.h): the host plan, checked
without a GPU.  The plan's pack and unpack permutes are applied by the oracle
on every rank's slab, the all-to-all is done by slicing, and the ranks'
output slabs together must equal the oracle's permute of the whole array."""
import numpy as np
import pytest

import oracle
import synth
from paper_1011_3583_gb300 import build as rbuild


@pytest.fixture(scope="module")
def lr():
    rbuild.build()
    from paper_1011_3583_gb300 import librearr
    librearr.load()
    return librearr


def simulate(lr, orc, e, dims, perm, nranks, seed):
    """Every rank's output slab, computed with the plan and the oracle."""
    n = int(np.prod(dims))
    glob = synth.random_elements(seed, n, e)
    plan = lr.dist_permute_plan(e, dims, perm, nranks)
    slab = plan.slab_bytes
    assert slab * nranks == n * e
    ins = [glob[r * slab:(r + 1) * slab] for r in range(nranks)]
    if not plan.exchange:
        return glob, plan, [orc.permute(x, e, *plan.pack()) for x in ins]
    sends = [orc.permute(x, e, *plan.pack()) for x in ins]
    pb = plan.piece_bytes
    recvs = [np.concatenate([sends[j][r * pb:(r + 1) * pb] for j in range(nranks)]) for r in range(nranks)]
    return glob, plan, [orc.permute(x, e, *plan.unpack()) for x in recvs]


CASES = [  # (elem_bytes, dims, perm, nranks)
    (4, [8, 6, 4], [2, 0, 1], 2),
    (4, [8, 6, 4], [0, 2, 1], 2),      # sharded axis stays slowest: no exchange
    (4, [8, 6, 4], [1, 2, 0], 2),
    (8, [6, 6], [1, 0], 3),            # 2-D transpose over 3 ranks
    (2, [12, 5, 8, 3], [3, 2, 1, 0], 1),
    (2, [12, 5, 8, 3], [2, 0, 3, 1], 4),
    (1, [16, 4, 4, 2, 3], [2, 4, 0, 3, 1], 2),
    (12, [4, 9, 8], [2, 1, 0], 4),
    (4, [64], [0], 8),                 # rank 1
    (16, [6, 2, 3, 2, 2, 2, 3], [6, 0, 1, 2, 3, 4, 5], 3),
]


@pytest.mark.parametrize("e,dims,perm,nranks", CASES)
def test_plan_reproduces_the_global_permute(lr, e, dims, perm, nranks):
    orc = oracle.get()
    glob, plan, outs = simulate(lr, orc, e, dims, perm, nranks, seed=sum(dims) + nranks)
    assert plan.exchange == (perm[0] != 0)
    assert np.array_equal(np.concatenate(outs), orc.permute(glob, e, dims, perm))


def test_random_plans(lr):
    orc = oracle.get()
    g = np.random.default_rng(4)
    for t in range(60):
        rank = int(g.integers(1, 7))
        nranks = int(g.integers(1, 6))
        perm = [int(x) for x in g.permutation(rank)]
        dims = [int(g.integers(1, 5)) for _ in range(rank)]
        dims[0] *= nranks
        dims[perm[0]] = dims[perm[0]] if dims[perm[0]] % nranks == 0 else dims[perm[0]] * nranks
        e = int(g.choice([1, 2, 4, 8, 3]))
        glob, plan, outs = simulate(lr, orc, e, dims, perm, nranks, seed=t)
        assert np.array_equal(np.concatenate(outs), orc.permute(glob, e, dims, perm)), (e, dims, perm, nranks)


def test_plan_shapes(lr):
    p = lr.dist_permute_plan(4, [8, 6, 4], [2, 0, 1], 2)
    assert (p.nranks, p.exchange, p.slab_bytes, p.piece_bytes) == (2, 1, 384, 192)
    # pack: axis 2 split into (2 ranks, 2 rows), destination rank first
    assert p.pack() == ([4, 6, 2, 2], [2, 3, 0, 1])
    # unpack: the source rank goes in front of output axis 1 (input axis 0)
    assert p.unpack() == ([2, 2, 4, 6], [1, 0, 2, 3])


@pytest.mark.parametrize("args", [
    (0, [8, 4], [1, 0], 2),            # elem_bytes 0
    (4, [8, 4], [1, 0], 0),            # no ranks
    (4, [8, 3], [1, 0], 2),            # output rows not a multiple of the ranks
    (4, [9, 4], [1, 0], 2),            # input rows not a multiple of the ranks
    (4, [8, 4], [1, 1], 2),            # not a permutation
    (4, [8, 0], [1, 0], 2),            # empty axis
    (4, [2] * 8, list(range(8)), 2),   # rank + 1 axes would exceed the maximum
])
def test_plan_rejects(lr, args):
    with pytest.raises(lr.RearrError) as ex:
        lr.dist_permute_plan(*args)
    assert ex.value.status == lr.EINVAL


def test_unpack_needs_an_exchange_plan(lr):
    p = lr.dist_permute_plan(4, [8, 4], [0, 1], 2)
    assert p.exchange == 0
    with pytest.raises(lr.RearrError):
        lr.dist_permute_unpack(0x1000, 0x2000, p, 4)
