"""Autotuner of librearr's tuning table (run on the target GPU).

    python -m paper_1011_3583_gb300.autotune --out paper_1011_3583_gb300/tuning/gb300.txt

It measures, with CUDA events and the library's own kernels only:

* for every fully vectorised fast-tile class -- element size E in
  {1, 2, 4, 8, 16} x input-fastest extent DA x output-fastest extent DB, each
  extent in one of five buckets, x whether the plane is widened over the axes
  that continue it -- the tile shape (staged rows of 128, 256 or 512 bytes;
  16 KB tiles, 32 KB double tiles, and for 2- and 4-byte elements on planes
  that are not widened 8 KB half tiles) that moves the class's
  representative permutes fastest in total.  The synthetic representatives
  move about 256 MiB each: a plane that is not widened is measured both dense
  (a [nb, DB, DA] tensor to [nb, DA, DB]: rows of a tile are contiguous on
  both sides) and, when its sides are long enough not to be widened,
  far-strided ([DB, nb, DA] to [DA, nb, DB]); a widened plane is measured as
  the rank-4 reversal [DB, n1, n2, DA] to [DA, n2, n1, DB], whose input rows
  and output runs continue over n2 and n1.  The permutes of the workloads the
  table serves (every order of 512^3 fp32 and of 64x128x256x64 at 2, 4 and 8
  bytes) are added to the representatives of the class they fall in;
* the vector width of the fast tiles: the widest the alignment allows (16
  bytes) against accesses of at most 4 bytes, on a few classes;
* the blocked copy of unmoved inner runs of 128-512 bytes (bytes per block
  side, and the longest run length for which it beats the runs kernel);
* the batched kernel's work grab (tiles taken per atomicAdd) on the 4096-op
  uneven mix, with the tile rules just measured;
* the thin-plane threshold (average cells per tile below which a permute runs
  as staged boxes of whole axes or an element-wise strided copy), then the
  largest cell size that runs as boxes and the shortest box run worth it, on
  the permutes of the whole mix, batched and as single calls (the sum of both
  times is minimised);
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


def _double_ok(E, rowb):
    return rowb in (128, 256) if E <= 2 else rowb in (256, 512)


def _representatives(E, DA, DB, wide):
    """(dims, perm) cases of a class, each moving about TARGET_BYTES."""
    nb = max(1, TARGET_BYTES // (DA * DB * E))
    if wide:
        n1 = max(1, int(round(nb ** 0.5)))
        n2 = max(1, nb // n1)
        return [([DB, n1, n2, DA], [3, 2, 1, 0])]
    return [([nb, DB, DA], [0, 2, 1]), ([DB, nb, DA], [2, 1, 0])]


def _bucket(x):
    for i, (lo, hi, _) in enumerate(BUCKETS):
        if lo <= x <= hi:
            return i
    return len(BUCKETS) - 1


def _workload_cases(rr):
    """The fast-tile permutes of the workloads this table serves (every order
    of 512^3 fp32 and of 64x128x256x64 at 2, 4 and 8 bytes), keyed by their
    tuning class (E, DA bucket, DB bucket, widened) under the default rules."""
    import itertools
    cases = {}
    shapes = [([512, 512, 512], 4)] + [([64, 128, 256, 64], e) for e in (2, 4, 8)]
    for dims, E in shapes:
        for perm in itertools.permutations(range(len(dims))):
            d = rr.describe_permute(E, dims, list(perm))
            if d["kind"] != "tile" or d["vec_in"] != 16:
                continue
            DA, DB = d["dims"][d["plane_a"]], d["dims"][d["rank"] - 1]
            wide = int(d["wide_a"] >= 0 or d["wide_b"] >= 0)
            cases.setdefault((E, _bucket(DA), _bucket(DB), wide), []).append((list(dims), list(perm)))
    return cases


def tune_rowb(rr, torch, stream, tmpdir, log):
    """Per class: the shape with the least total time over the class's
    synthetic representatives and the workload permutes that fall in it."""
    rules = []
    rr.tuning_load(None)
    workload = _workload_cases(rr)
    big = max(int(np.prod(d)) * 8 for d in ([512, 512, 512], [64, 128, 256, 64]))
    buf_a = torch.empty(max(TARGET_BYTES + (1 << 20), big), dtype=torch.uint8, device="cuda").random_()
    buf_b = torch.empty_like(buf_a)
    for E in ELEMS:
        for wide in (0, 1):
            cands = [(128, 16384), (256, 16384)] + ([] if E == 1 else [(512, 16384)])
            cands += [(r, 32768) for r in (128, 256, 512) if _double_ok(E, r)]
            if E in (2, 4) and not wide:
                cands.append((128, 8192))
            for ia, (alo, ahi, DA) in enumerate(BUCKETS):
                for ib, (blo, bhi, DB) in enumerate(BUCKETS):
                    reps = _representatives(E, DA, DB, wide) + workload.get((E, ia, ib, wide), [])
                    best = None
                    for rowb, tbytes in cands:
                        table = os.path.join(tmpdir, "cand.txt")
                        _write(table, [f"rowb {E} {alo} {ahi} {blo} {bhi} {rowb} {tbytes} {wide}"])
                        rr.tuning_load(table)
                        total, ok = 0.0, 0
                        for dims, perm in reps:
                            if int(np.prod(dims)) * E > buf_a.numel():
                                continue
                            d = rr.describe_permute(E, dims, perm, buf_b.data_ptr(), buf_a.data_ptr())
                            widened = d["kind"] == "tile" and (d["wide_a"] >= 0 or d["wide_b"] >= 0)
                            if (d["kind"] != "tile" or widened != bool(wide) or d["tile_a"] * E != rowb
                                    or d["tile_a"] * d["tile_b"] * E != tbytes):
                                continue  # the rule does not apply to this case
                            total += _time(torch, lambda: rr.permute(buf_b, buf_a, E, dims, perm, stream), stream,
                                           reps=20)
                            ok += 1
                        if ok == 0:
                            continue
                        log(f"E={E:2d} DA={DA:5d} DB={DB:5d} wide={wide} rowb={rowb:3d} tile={tbytes:5d}: "
                            f"{total * 1e3:8.3f} ms over {ok} case(s)")
                        if best is None or (ok, -total) > (best[3], -best[2]):
                            best = (rowb, tbytes, total, ok)
                    if best:
                        rules.append(f"rowb {E} {alo} {ahi} {blo} {bhi} {best[0]} {best[1]} {wide}   "
                                     f"# {best[2] * 1e3:.3f} ms over {best[3]} case(s)")
    rr.tuning_load(None)
    return rules


def tune_vector(rr, torch, stream, tmpdir, log, base_lines):
    """The fast tile's widest access (16 bytes) against at most 4 bytes."""
    a = torch.empty(TARGET_BYTES, dtype=torch.uint8, device="cuda").random_()
    b = torch.empty_like(a)
    cases = [(E, dims, perm) for E in (1, 2, 4, 8)
             for dims, perm in (([64, 128, 256, 64], [3, 2, 1, 0]), ([512, 512, 256], [2, 1, 0]))]
    totals = {}
    for cap in (16, 4):
        table = os.path.join(tmpdir, "vec.txt")
        _write(table, base_lines + [f"tile_vector_bytes {cap}"])
        rr.tuning_load(table)
        t = 0.0
        for E, dims, perm in cases:
            dims = list(dims)
            while int(np.prod(dims)) * E > a.numel():
                dims[0] //= 2
            t1 = _time(torch, lambda: rr.permute(b, a, E, dims, perm, stream), stream)
            log(f"tile_vector_bytes={cap:2d} E={E} dims={dims} perm={perm}: "
                f"{2 * int(np.prod(dims)) * E / t1 / 1e9:8.1f} GB/s")
            t += t1
        totals[cap] = t
    rr.tuning_load(None)
    best = min(totals, key=totals.get)
    return [f"tile_vector_bytes {best}   # 16: {totals[16] * 1e3:.3f} ms, 4: {totals[4] * 1e3:.3f} ms on "
            f"{len(cases)} permutes"]


def tune_runs_blocks(rr, torch, stream, tmpdir, log, base_lines):
    """Blocked runs against the runs kernel, per run length (64 elements of
    2, 4 and 8 bytes), and the block size in cells."""
    orders = ([2, 1, 0, 3], [1, 2, 0, 3], [0, 2, 1, 3], [2, 0, 1, 3])
    dims = [64, 128, 256, 64]
    n = int(np.prod(dims))
    a = torch.empty(n * 8, dtype=torch.uint8, device="cuda").random_()
    b = torch.empty_like(a)
    times = {}
    blocks = ("runs_tile_side_bytes 1024", "runs_tile_side_bytes 2048", "runs_tile_side_bytes 4096")
    for setting in ("runs_tile_max_bytes 1",) + blocks:
        table = os.path.join(tmpdir, "blk.txt")
        _write(table, base_lines + ["runs_tile_max_bytes 4096", "runs_tile_cells 8", setting] if "side" in setting
               else base_lines + [setting])
        rr.tuning_load(table)
        for e in (2, 4, 8):
            t = sum(_time(torch, lambda: rr.permute(b, a, e, dims, p, stream), stream) for p in orders)
            times[(setting, e)] = t
            log(f"{setting:24s} runs of {64 * e:3d} B: {len(orders) * 2 * n * e / t / 1e9:8.1f} GB/s")
    rr.tuning_load(None)
    best_block = min(blocks, key=lambda s: sum(times[(s, e)] for e in (2, 4, 8)))
    limit = 1
    for e in (2, 4, 8):
        if times[(best_block, e)] < times[("runs_tile_max_bytes 1", e)]:
            limit = 64 * e + 1
        else:
            break
    return ["runs_tile_cells 8", best_block, f"runs_tile_max_bytes {limit}"]


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


def _mix_permutes(torch):
    import bench
    import synth
    ops = [o for o in synth.batch_mix(seed=1, n_ops=4096) if o["kind"] == "permute"]
    pool, bufs = bench.batch_buffers(torch, ops, torch.device("cuda"))
    return ops, pool, bufs


def _time_mix(rr, torch, stream, table, ops, bufs):
    """(batched replay, one call per op) times of the mix's permutes under a table."""
    import bench
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
    return tb, tp


def tune_thin(rr, torch, stream, tmpdir, log, base_lines):
    ops, pool, bufs = _mix_permutes(torch)
    best = None
    for cells in (256, 512, 1024, 2048, 4096, 8192, 16384):
        table = os.path.join(tmpdir, "thin.txt")
        _write(table, base_lines + [f"thin_tile_cells {cells}"])
        tb, tp = _time_mix(rr, torch, stream, table, ops, bufs)
        log(f"thin_tile_cells={cells:5d}: batched {tb * 1e3:7.3f} ms  single calls {tp * 1e3:7.3f} ms")
        if best is None or tb + tp < best[1]:
            best = (cells, tb + tp)
    rr.tuning_load(None)
    del pool
    return [f"thin_tile_cells {best[0]}"]


def tune_box(rr, torch, stream, tmpdir, log, base_lines):
    """Thin planes as staged boxes: the largest cell size that runs as boxes
    (0: none) and the shortest run for which a box beats the strided copy,
    on the mix's permutes (batched plus single calls)."""
    ops, pool, bufs = _mix_permutes(torch)
    best = None
    for cell in (0, 1, 2, 4, 16):
        for min_run in ((16,) if cell == 0 else (16, 64)):
            table = os.path.join(tmpdir, "box.txt")
            _write(table, base_lines + [f"box_max_cell_bytes {cell}", f"box_min_run_bytes {min_run}"])
            tb, tp = _time_mix(rr, torch, stream, table, ops, bufs)
            log(f"box_max_cell_bytes={cell:2d} box_min_run_bytes={min_run:3d}: batched {tb * 1e3:7.3f} ms  "
                f"single calls {tp * 1e3:7.3f} ms")
            if best is None or tb + tp < best[2]:
                best = (cell, min_run, tb + tp)
    rr.tuning_load(None)
    del pool
    return [f"box_max_cell_bytes {best[0]}", f"box_min_run_bytes {best[1]}"]


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
        vec = tune_vector(rr, torch, stream, tmp, log, base)
        base += [v.split("#")[0] for v in vec]
        blocks = tune_runs_blocks(rr, torch, stream, tmp, log, base)
        base += blocks
        grab = tune_grab(rr, torch, stream, tmp, log, base)
        base += [g.split("#")[0] for g in grab]
        thin = tune_thin(rr, torch, stream, tmp, log, base)
        box = tune_box(rr, torch, stream, tmp, log, base + thin)
        runs = tune_runs_order(rr, torch, stream, tmp, log, base + ["runs_tile_max_bytes 1"])
    head = [f"# librearr tuning table for {torch.cuda.get_device_name()} "
            f"(paper_1011_3583_gb300/autotune.py, {time.time() - t0:.0f} s)"]
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    _write(args.out, head + grab + thin + box + runs + blocks + vec + rules + log_lines)
    print(f"wrote {args.out}: {len(rules)} tile rules")


if __name__ == "__main__":
    np.seterr(all="ignore")
    main()
