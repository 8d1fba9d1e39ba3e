"""Autotuner of librearr's tuning table (run on the target GPU).

    python -m paper_1011_3583_gb300.autotune --out paper_1011_3583_gb300/tuning/gb300.txt

It measures, with CUDA events and the library's own kernels only:

* for every fully vectorised fast-tile class -- element size E in
  {1, 2, 4, 8, 16} x input-fastest extent DA x output-fastest extent DB, each
  extent in one of five buckets -- the tile shape (staged row length of 128,
  256 or 512 bytes; 16 KB tiles, or 8 KB half tiles for 2- and 4-byte
  elements) that moves a representative permute of that class fastest.  The representative case is a [nb, DB, DA] tensor permuted
  to [nb, DA, DB], nb chosen so that each call moves about 256 MiB;
* the batched kernel's work grab (tiles taken per atomicAdd) on the 4096-op
  uneven mix, with the tile rules just measured;
* the thin-plane threshold (average cells per tile below which a permute runs
  as an element-wise strided copy) on the permutes of the whole mix, batched
  and as single calls (the sum of both times is minimised);
* the longest run (128, 256 or 512 bytes) that is faster walked in input
  order than in output order.

The result is a text table read by rearr_tuning_load (see tuning.cpp).
"""
from __future__ import annotations

import argparse
import os
import statistics
import tempfile
import time

import numpy as np

# (lo, hi, representative) extent buckets; representatives are multiples of 16
BUCKETS = [(1, 48, 32), (49, 96, 64), (97, 192, 128), (193, 384, 256), (385, 2 ** 31 - 1, 1024)]
ELEMS = (1, 2, 4, 8, 16)
TARGET_BYTES = 256 << 20


def _time(torch, fn, stream, reps=10, warmup=2):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    return statistics.median(ts)


def _write(path, lines):
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def tune_rowb(rr, torch, stream, tmpdir, log):
    rules = []
    buf_a = torch.empty(TARGET_BYTES + (1 << 20), dtype=torch.uint8, device="cuda").random_()
    buf_b = torch.empty_like(buf_a)
    for E in ELEMS:
        # (staged row bytes, tile payload bytes); 2- and 4-byte elements also
        # have an 8 KB half tile for planes too small to fill 16 KB
        cands = [(128, 16384), (256, 16384)] + ([] if E == 1 else [(512, 16384)])
        if E in (2, 4):
            cands.append((128, 8192))
        for (alo, ahi, DA) in BUCKETS:
            for (blo, bhi, DB) in BUCKETS:
                nb = max(1, TARGET_BYTES // (DA * DB * E))
                dims, perm = [nb, DB, DA], [0, 2, 1]
                best = None
                for rowb, tbytes in cands:
                    table = os.path.join(tmpdir, "cand.txt")
                    _write(table, [f"rowb {E} {alo} {ahi} {blo} {bhi} {rowb} {tbytes}"])
                    rr.tuning_load(table)
                    d = rr.describe_permute(E, dims, perm, buf_b.data_ptr(), buf_a.data_ptr())
                    if d["kind"] != "tile" or d["tile_a"] * E != rowb or d["tile_a"] * d["tile_b"] * E != tbytes:
                        continue  # not a fully vectorised tile: the table does not apply
                    t = _time(torch, lambda: rr.permute(buf_b, buf_a, E, dims, perm, stream), stream)
                    gbs = 2 * nb * DA * DB * E / t / 1e9
                    log(f"E={E:2d} DA={DA:5d} DB={DB:5d} rowb={rowb:3d} tile={tbytes:5d}: {gbs:8.1f} GB/s")
                    if best is None or gbs > best[2]:
                        best = (rowb, tbytes, gbs)
                if best:
                    rules.append(f"rowb {E} {alo} {ahi} {blo} {bhi} {best[0]} {best[1]}   # {best[2]:.0f} GB/s")
    rr.tuning_load(None)
    return rules


def tune_grab(rr, torch, stream, tmpdir, log, base_lines, n_ops=4096):
    import bench  # the mix's buffers and plan helpers
    import synth
    ops = synth.batch_mix(seed=1, n_ops=n_ops)
    pool, bufs = bench.batch_buffers(torch, ops, torch.device("cuda"))
    nbytes = sum(synth.op_bytes(o) for o in ops)
    best = None
    for g in (1, 2, 4, 8, 16, 32):
        table = os.path.join(tmpdir, "grab.txt")
        _write(table, base_lines + [f"min_grab {g}", f"max_grab {g}"])
        rr.tuning_load(table)
        plan = rr.Plan()
        for o, p in zip(ops, bufs):
            bench.add_to_plan(plan, o, p)
        plan.finalize(stream)
        t = _time(torch, lambda: plan.run(stream), stream)
        plan.close()
        log(f"grab={g:2d}: {nbytes / t / 1e9:8.1f} GB/s  {n_ops / t:10.0f} ops/s")
        if best is None or t < best[1]:
            best = (g, t)
    rr.tuning_load(None)
    del pool
    return [f"min_grab {best[0]}", f"max_grab {best[0]}   # {nbytes / best[1] / 1e9:.0f} GB/s on the mix"]


def tune_thin(rr, torch, stream, tmpdir, log, base_lines):
    import bench
    import synth
    ops = [o for o in synth.batch_mix(seed=1, n_ops=4096) if o["kind"] == "permute"]
    pool, bufs = bench.batch_buffers(torch, ops, torch.device("cuda"))
    best = None
    for cells in (256, 512, 1024, 2048, 4096):
        table = os.path.join(tmpdir, "thin.txt")
        _write(table, base_lines + [f"thin_tile_cells {cells}"])
        rr.tuning_load(table)
        plan = rr.Plan()
        for o, p in zip(ops, bufs):
            bench.add_to_plan(plan, o, p)
        plan.finalize(stream)
        tb = _time(torch, lambda: plan.run(stream), stream)
        plan.close()

        def plain():
            for o, p in zip(ops, bufs):
                rr.permute(p[1], p[0], o["elem_bytes"], o["dims"], o["perm"], stream)
        tp = _time(torch, plain, stream, reps=3)
        log(f"thin_tile_cells={cells:5d}: batched {tb * 1e3:7.3f} ms  single calls {tp * 1e3:7.3f} ms")
        if best is None or tb + tp < best[1]:
            best = (cells, tb + tp)
    rr.tuning_load(None)
    del pool
    return [f"thin_tile_cells {best[0]}"]


def tune_runs_order(rr, torch, stream, tmpdir, log, base_lines):
    """Largest run length (128, 256, 512 B) for which walking runs in input
    order beats output order on a 1 GiB-class permute with that run length."""
    best = 1
    for e in (2, 4, 8):  # runs of 64 elements: 128, 256, 512 bytes
        dims, perm = [64, 128, 256, 64], [2, 1, 0, 3]
        n = int(np.prod(dims))
        a = torch.empty(n * e, dtype=torch.uint8, device="cuda").random_()
        b = torch.empty_like(a)
        times = []
        for mirror in (1, 64 * e):
            table = os.path.join(tmpdir, "runs.txt")
            _write(table, base_lines + [f"runs_mirror_bytes {mirror}"])
            rr.tuning_load(table)
            times.append(_time(torch, lambda: rr.permute(b, a, e, dims, perm, stream), stream))
        log(f"runs of {64 * e:3d} B: output order {2 * n * e / times[0] / 1e9:7.1f} GB/s, "
            f"input order {2 * n * e / times[1] / 1e9:7.1f} GB/s")
        if times[1] < times[0]:
            best = 64 * e
        del a, b
    rr.tuning_load(None)
    return [f"runs_mirror_bytes {best}"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    import torch
    os.environ.pop("REARR_TUNE_TABLE", None)
    from paper_1011_3583_gb300 import build
    build.build()
    import paper_1011_3583_gb300 as rr
    rr.load()
    rr.tuning_load(None)
    stream = torch.cuda.Stream()
    log_lines = []

    def log(s):
        print(s, flush=True)
        log_lines.append("# " + s)

    t0 = time.time()
    with tempfile.TemporaryDirectory() as tmp:
        rules = tune_rowb(rr, torch, stream, tmp, log)
        base = [r.split("#")[0] for r in rules]
        grab = tune_grab(rr, torch, stream, tmp, log, base)
        thin = tune_thin(rr, torch, stream, tmp, log, base + [g.split("#")[0] for g in grab])
        runs = tune_runs_order(rr, torch, stream, tmp, log, base)
    head = [f"# librearr tuning table for {torch.cuda.get_device_name()} "
            f"(paper_1011_3583_gb300/autotune.py, {time.time() - t0:.0f} s)"]
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    _write(args.out, head + grab + thin + runs + rules + log_lines)
    print(f"wrote {args.out}: {len(rules)} tile rules")


if __name__ == "__main__":
    np.seterr(all="ignore")
    main()
