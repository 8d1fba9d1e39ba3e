"""rearr_batch_noalloc, the batched entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc (a serving process whose
device memory is all reserved for its own pool, or a latency-critical path that
cannot take the synchronisation an allocation may cause).  It runs a plan from
a fixed work-list buffer compiled into the library instead of the buffer that
rearr_plan_finalize allocates.  These tests check, through the C ABI, that it
gives exactly the bytes the regular rearr_plan_finalize + rearr_batch path
gives, and the oracle's, on two calls in a row (the fixed buffer keeps the
previous call's contents, so the second call must not depend on them), with
every buffer guarded against writes outside it, and that a plan too large for
the buffer is refused before any work is issued.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import DevBuf, DevPool, sync
from tests.test_gpu_parity import add_to_plan, make_op_buffers, oracle_of, outputs_of

# The fixed work-list buffer holds about 1280 ops (the documented capacity).
DOCUMENTED_CAPACITY_OPS = 1280

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build, librearr
    build.build()
    librearr.load()
    return librearr


def fresh_outputs(op, b, pool):
    """Second set of zeroed, guarded output buffers for an op (inputs shared)."""
    c = dict(b)
    if op["kind"] == "deinterlace":
        c["dsts"] = [DevBuf(d.nbytes, d.offset, fill=0, pool=pool) for d in b["dsts"]]
    else:
        c["dst"] = DevBuf(b["dst"].nbytes, b["dst"].offset, fill=0, pool=pool)
    return c


def clear(op, b, value):
    for out in (b["dsts"] if op["kind"] == "deinterlace" else [b["dst"]]):
        out.view.fill_(value)


def test_noalloc_matches_batch_on_two_calls(lr):
    ops = synth.batch_mix(seed=21, n_ops=96, hi_total=2 ** 15)
    ops += [dict(kind="interlace", elem_bytes=4, k=12, n=333, data_seed=5),
            dict(kind="deinterlace", elem_bytes=2, k=9, n=1001, data_seed=6)]
    orc = oracle.get()
    pool = DevPool()
    ref = [make_op_buffers(op, offset=(i % 3) * 4, pool=pool) for i, op in enumerate(ops)]
    mine = [fresh_outputs(op, b, pool) for op, b in zip(ops, ref)]

    regular = lr.Plan()
    for op, b in zip(ops, ref):
        add_to_plan(regular, op, b)
    regular.finalize()
    regular.run()

    noalloc = lr.Plan()
    for op, b in zip(ops, mine):
        add_to_plan(noalloc, op, b)
    for call, fill in enumerate((0x00, 0xC3)):
        for op, b in zip(ops, mine):
            clear(op, b, fill)
        noalloc.run_noalloc()
        sync()
        pool.check()
        for i, (op, x, y) in enumerate(zip(ops, ref, mine)):
            for want, got, exact in zip(outputs_of(op, x), outputs_of(op, y), oracle_of(orc, op, x)):
                assert np.array_equal(got, want), (call, i, op)
                assert np.array_equal(got, exact), ("oracle", call, i, op)
    regular.close()
    noalloc.close()


def test_noalloc_refuses_a_plan_larger_than_its_buffer(lr):
    """Four times the documented capacity of small permutes is refused before
    anything is issued.  Every op names the same real 64-byte buffers, so even
    a plan that was wrongly accepted would only rewrite them."""
    src, dst = DevBuf(64, fill=1), DevBuf(64, fill=0)
    plan = lr.Plan()
    for i in range(4 * DOCUMENTED_CAPACITY_OPS):
        plan.add_permute(dst.ptr, src.ptr, 4, [4, 4], [1, 0])
    before = lr.launch_count()
    with pytest.raises(lr.RearrError) as ex:
        plan.run_noalloc()
    assert ex.value.status == lr.EINVAL and "fixed" in str(ex.value)
    assert lr.launch_count() == before
    plan.close()
