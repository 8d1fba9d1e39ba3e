"""The serving loop on the GPU: every request's result is the same alone (a
single call) and in the mix (served with others, batched on several streams),
admission waits for memory under the budget, and host-injected completion
delays surface as REARR_ETIMEDOUT without touching the GPU."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import guard_pattern, sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1011_3583_gb300 import build
    build.build()
    import paper_1011_3583_gb300 as rr
    return rr


def op_inputs(op):
    """Host input buffers of an op spec, from its data seed."""
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        return [synth.random_elements(op["data_seed"], int(np.prod(op["dims"])), e)]
    if op["kind"] == "reorder":
        return [synth.random_elements(op["data_seed"], op["n"], e),
                synth.random_permutation(op["data_seed"] ^ 1, op["n"]).view(np.uint8)]
    if op["kind"] == "interlace":
        return [synth.random_elements(op["data_seed"] + j, op["n"], e) for j in range(op["k"])]
    return [synth.random_elements(op["data_seed"], op["n"] * op["k"], e)]


def oracle_outputs(op, ins):
    orc = oracle.get()
    e = op["elem_bytes"]
    if op["kind"] == "permute":
        return [orc.permute(ins[0], e, op["dims"], op["perm"])]
    if op["kind"] == "reorder":
        return [orc.reorder(ins[0], ins[1].view(np.uint32), e)]
    if op["kind"] == "interlace":
        return [orc.interlace(ins, op["n"], e)]
    return orc.deinterlace(ins[0], op["k"], op["n"], e)


def upload(rr, ptr, host):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(host).view(np.uint8)).cuda()
    rr.memcpy_d2d(ptr, t, t.numel())
    sync()


def download(rr, ptr, nbytes):
    import torch
    t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    rr.memcpy_d2d(t, ptr, nbytes)
    sync()
    return t.cpu().numpy()


SENTINEL = dict(kind="permute", elem_bytes=1, dims=[256], perm=[0])


def serve_all(rr, srv, ops):
    """Reserve, fill and submit every op, then wait for all; returns outputs.

    A sentinel reservation (256 bytes in, 256 out, filled with a seeded
    pattern and never submitted) is made before the first request and after
    every request.  The slab is first-fit and nothing is released until the
    end, so every request's buffers lie between sentinel buffers; a write
    outside a request's own buffers changes a sentinel and fails the test."""
    sentinels = []

    def sentinel():
        t = srv.reserve(SENTINEL)
        ins, outs = srv.buffers(t)
        pat = guard_pattern(256, 2 + len(sentinels))
        for p in ins + outs:
            upload(rr, p, pat)
        sentinels.append((t, ins + outs, pat))

    tickets, wants = [], []
    sentinel()
    for op in ops:
        ins = op_inputs(op)
        t = srv.reserve(op)
        in_ptrs, _ = srv.buffers(t)
        for p, h in zip(in_ptrs, ins):
            upload(rr, p, h)
        sentinel()
        tickets.append(t)
        wants.append(oracle_outputs(op, ins))
    for t in tickets:  # submitted back to back, so the ready queue builds up
        srv.submit(t)
    outs = []
    for t, w in zip(tickets, wants):
        srv.wait(t, timeout_us=30_000_000)
        _, out_ptrs = srv.buffers(t)
        outs.append([download(rr, p, x.size) for p, x in zip(out_ptrs, w)])
        assert srv.latency(t) > 0
        srv.release(t)
    for t, ptrs, pat in sentinels:
        for p in ptrs:
            assert np.array_equal(download(rr, p, 256), pat), "a write landed outside a request's buffers"
        srv.release(t)
    return outs, wants


@pytest.mark.parametrize("batching", [True, False])
def test_each_result_same_alone_and_in_the_mix(rr, batching):
    ops = synth.batch_mix(seed=31, n_ops=120, hi_total=2 ** 14)
    srv = rr.Server(budget_bytes=512 << 20, n_streams=3, max_batch_ops=64, batching=batching)
    outs, wants = serve_all(rr, srv, ops)
    for i, (o, w) in enumerate(zip(outs, wants)):
        for got, want in zip(o, w):
            assert np.array_equal(got, want), (i, ops[i])
    st = srv.stats()
    # every request and every sentinel (one more than the requests) was released
    assert st["completed"] == len(ops) and st["released"] == 2 * len(ops) + 1 and st["slab_used"] == 0
    if batching:
        assert st["launches"] < len(ops)      # some requests went out together
    srv.close()


@pytest.mark.parametrize("batching", [True, False])
def test_wide_interlaces_and_large_gathers_served(rr, batching):
    """Interlaces with 5-8 planes (16-byte group path in single calls, the
    generic body in batched launches) and reorders of several batched work
    units, served together: every result matches the oracle."""
    ops = []
    for i, k in enumerate((5, 6, 7, 8, 6, 8)):
        ops.append(dict(kind="interlace" if i % 2 == 0 else "deinterlace", elem_bytes=[4, 8, 2, 1][i % 4], k=k,
                        n=4096 + 16 * i, data_seed=500 + i))
    ops += [dict(kind="reorder", elem_bytes=e, n=n, data_seed=600 + n) for e, n in ((4, 10000), (8, 70001), (1, 33))]
    srv = rr.Server(budget_bytes=256 << 20, n_streams=2, max_batch_ops=16, batching=batching)
    outs, wants = serve_all(rr, srv, ops)
    for i, (o, w) in enumerate(zip(outs, wants)):
        for got, want in zip(o, w):
            assert np.array_equal(got, want), (i, ops[i])
    srv.close()


def test_admission_waits_for_memory(rr):
    e, n = 4, (3 << 20) // 4                      # 3 MiB in + 3 MiB out per request
    op = dict(kind="permute", elem_bytes=e, dims=[n // 1024, 1024], perm=[1, 0])
    srv = rr.Server(budget_bytes=8 << 20, n_streams=2)
    big = dict(kind="permute", elem_bytes=4, dims=[4096, 1024], perm=[1, 0])   # 32 MiB > budget
    with pytest.raises(rr.RearrError) as ex:
        srv.reserve(big)
    assert ex.value.status == 2                   # REARR_ENOMEM
    t1 = srv.reserve(op)
    with pytest.raises(rr.RearrError) as ex:
        srv.reserve(op, timeout_us=0)             # no room until t1 is released
    assert ex.value.status == 5                   # REARR_ETIMEDOUT
    got = {}

    def second():
        got["t"] = srv.reserve(op, timeout_us=20_000_000)

    th = threading.Thread(target=second)
    th.start()
    time.sleep(0.2)
    assert "t" not in got                         # still waiting for memory
    srv.submit(t1)
    srv.wait(t1)
    srv.release(t1)                               # frees 6 MiB: the waiter is admitted
    th.join(timeout=20)
    assert "t" in got
    srv.release(got["t"])
    srv.close()


def test_injected_completion_delay_times_out_then_completes(rr):
    srv = rr.Server(budget_bytes=64 << 20, n_streams=2)
    srv.inject_completion_delay(400_000)          # completions hidden for 0.4 s (host side)
    op = dict(kind="permute", elem_bytes=4, dims=[64, 64], perm=[1, 0])
    t = srv.reserve(op)
    srv.submit(t)
    with pytest.raises(rr.RearrError) as ex:
        srv.wait(t, timeout_us=20_000)
    assert ex.value.status == 5                   # REARR_ETIMEDOUT
    assert not srv.poll(t)
    with pytest.raises(rr.RearrError) as ex:
        srv.release(t)                            # still in flight
    assert ex.value.status == 6                   # REARR_EBUSY
    srv.wait(t, timeout_us=5_000_000)
    assert srv.latency(t) >= 0.4
    srv.release(t)
    srv.close()


def test_trace_driver(rr):
    import torch
    ops = synth.batch_mix(seed=41, n_ops=300, hi_total=2 ** 16)
    templates = []
    keep = []
    for o in ops:
        row = [None] * 4
        if o["kind"] == "reorder":
            p = torch.randperm(o["n"], device="cuda", dtype=torch.int64).to(torch.int32)
            keep.append(p)
            row[1] = p
        templates += row
    arrivals = synth.poisson_arrivals(5, rate_per_s=20000.0, count=len(ops))
    for batching in (True, False):
        srv = rr.Server(budget_bytes=1 << 30, n_streams=3, batching=batching)
        lat, wall = srv.run_trace(ops, arrivals, templates, timeout_us=60_000_000)
        assert len(lat) == len(ops) and min(lat) > 0 and wall > 0
        st = srv.stats()
        assert st["completed"] == len(ops) and st["slab_used"] == 0
        srv.close()


def test_lone_requests_run_as_single_ops(rr):
    """A request that is alone in the ready queue goes out as its single-op
    kernel (one launch per request when each waits for the previous), with the
    oracle's result."""
    ops = synth.batch_mix(seed=32, n_ops=12, hi_total=2 ** 14)
    srv = rr.Server(budget_bytes=256 << 20, n_streams=2, max_batch_ops=64, batching=True)
    for i, op in enumerate(ops):
        ins = op_inputs(op)
        t = srv.reserve(op)
        in_ptrs, _ = srv.buffers(t)
        for p, h in zip(in_ptrs, ins):
            upload(rr, p, h)
        srv.submit(t)
        srv.wait(t, timeout_us=30_000_000)
        _, out_ptrs = srv.buffers(t)
        for p, want in zip(out_ptrs, oracle_outputs(op, ins)):
            assert np.array_equal(download(rr, p, want.size), want), (i, op)
        srv.release(t)
    assert srv.stats()["launches"] == len(ops)
    srv.close()
