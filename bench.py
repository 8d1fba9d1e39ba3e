"""Benchmark of librearr on the generic-permute workload.

One step = one pass over the workload, one library call (one kernel) per op,
all on one stream, inputs resident in HBM:
  * the 6 axis orders of a 512 x 512 x 512 fp32 tensor (512 MiB),
  * the 24 axis orders of a 64 x 128 x 256 x 64 tensor at 2, 4 and 8 bytes per
    element (256 MiB, 512 MiB, 1 GiB),
  * a reorder of 2^28 fp32 elements by a uniform random permutation and by a
    permutation of 65536 shuffled blocks of 4096 elements.
Inputs are seeded random bit patterns (numpy PCG64), every op reads at least
256 MiB, so every operand is larger than the 129 MB L2 and no flush is needed.

Throughput is effective GB/s = (bytes read + bytes written) / time, GB = 1e9,
index reads of the reorders included.  The roofline denominators are a
cudaMemcpyAsync device-to-device copy measured in the same run and the
copy bandwidth recorded in MEASURED_PEAKS.json (a STREAM-style copy measured on
the same GPU model).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs the whole workload on its own GPU (independent
replicas, no collective on the data path); the value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "permute GB/s (R+W) as % of GB300 D2D memcpy; batched ops/s & p99 vs plain"
WORKLOAD = "generic permute: 6 orders of 512^3 fp32, 24 orders of 64x128x256x64 at 2/4/8 B, reorder 2^28 fp32 (random, 4096-block)"
MIB = 1 << 20


def workload_ops():
    """The op list of one step (shapes only)."""
    import itertools
    ops = []
    for perm in itertools.permutations(range(3)):
        ops.append(dict(kind="permute", elem_bytes=4, dims=[512, 512, 512], perm=list(perm)))
    for e in (2, 4, 8):
        for perm in itertools.permutations(range(4)):
            ops.append(dict(kind="permute", elem_bytes=e, dims=[64, 128, 256, 64], perm=list(perm)))
    ops.append(dict(kind="reorder", elem_bytes=4, n=1 << 28, idx="random"))
    ops.append(dict(kind="reorder", elem_bytes=4, n=1 << 28, idx="block4096"))
    return ops


def op_bytes(op) -> int:
    if op["kind"] == "permute":
        return 2 * int(np.prod(op["dims"])) * op["elem_bytes"]
    return 2 * op["n"] * op["elem_bytes"] + 4 * op["n"]


def op_in_bytes(op) -> int:
    if op["kind"] == "permute":
        return int(np.prod(op["dims"])) * op["elem_bytes"]
    return op["n"] * op["elem_bytes"] + 4 * op["n"]


def op_out_bytes(op) -> int:
    if op["kind"] == "permute":
        return int(np.prod(op["dims"])) * op["elem_bytes"]
    return op["n"] * op["elem_bytes"]


# Sources of the tile kernel family and of the plan that picks its shapes: a
# change to any of them invalidates the DRAM traffic taken with ncu.
TILE_SOURCES = ("bodies.cuh", "device_common.cuh", "k_single.cu", "plan.cpp", "plan.h", "rearr_internal.h",
                "tuning.cpp", "tuning.h", "variants.h")


def source_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1011_3583_gb300", "csrc")
    for f in TILE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append(dict(sm=float(parts[0]), smax=float(parts[1]), power=float(parts[2]),
                                 hw=parts[4], hwt=parts[5], swt=parts[6], swp=parts[7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["swp"] == "Active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ---------------------------------------------------------------------------
# GPU arm

class Workload:
    """Device buffers of the workload (inputs seeded, reused across ops)."""

    def __init__(self, torch, ops, device):
        import synth
        self.torch = torch
        self.ops = ops
        max_in = max(int(np.prod(o["dims"])) * o["elem_bytes"] if o["kind"] == "permute" else o["n"] * o["elem_bytes"]
                     for o in ops)
        self.src_np = synth.random_elements(20260101, max_in // 4, 4)
        self.src = torch.from_numpy(self.src_np).to(device)
        self.dst = torch.empty(max_in, dtype=torch.uint8, device=device)
        self.idx_np = {}
        self.idx = {}
        for o in ops:
            if o["kind"] == "reorder" and o["idx"] not in self.idx:
                n = o["n"]
                a = (synth.random_permutation(7, n) if o["idx"] == "random"
                     else synth.block_shuffled_permutation(8, n, 4096))
                self.idx_np[o["idx"]] = a
                self.idx[o["idx"]] = torch.from_numpy(a.view(np.uint8)).to(device)

    def run_op(self, rr, o, stream, src=None, dst=None):
        src = self.src if src is None else src
        dst = self.dst if dst is None else dst
        if o["kind"] == "permute":
            rr.permute(dst, src, o["elem_bytes"], o["dims"], o["perm"], stream)
        else:
            rr.reorder(dst, src, self.idx[o["idx"]], o["n"], o["elem_bytes"], stream)


def kernel_family(rr, o) -> str:
    if o["kind"] == "reorder":
        return "gather"
    return rr.describe_permute(o["elem_bytes"], o["dims"], o["perm"])["kind"]


def measure_memcpy(torch, rr, stream, nbytes=1 << 30, reps=10):
    a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    a.fill_(1)
    times = []
    with torch.cuda.stream(stream):
        for i in range(3 + reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            rr.memcpy_d2d(b, a, nbytes, stream)
            e.record(stream)
            e.synchronize()
            if i >= 3:
                times.append(s.elapsed_time(e) / 1e3)
    del a, b
    t = statistics.median(times)
    return 2 * nbytes / t / 1e9, min(times)


def load_traffic_summary():
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_digest") != source_digest():
        return None  # the kernels changed since the counters were taken
    return d


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if d.get("hbm_gbs"):
            return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(seconds: float, world: int, device) -> float:
    """The slowest rank's time (every rank runs a full replica of the workload)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world: int, step_bytes: int, steps: int, seconds: float) -> float:
    """Whole-job GB/s: every rank moved step_bytes per step, timed by the slowest."""
    return world * step_bytes * steps / seconds / 1e9


def run_gpu(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)

    from paper_1011_3583_gb300 import build as rbuild
    if rank == 0:
        rbuild.build()
    if world > 1:
        dist.barrier()
    import paper_1011_3583_gb300 as rr
    rr.load()

    ops = workload_ops()
    wl = Workload(torch, ops, device)
    stream = torch.cuda.Stream(device)
    step_bytes = sum(op_bytes(o) for o in ops)
    fams = [kernel_family(rr, o) for o in ops]

    def step():
        for o in ops:
            wl.run_op(rr, o, stream)

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    memcpy_gbs, _ = measure_memcpy(torch, rr, stream)
    # a device copy of each op's payload size, the same-size denominator
    memcpy_same = {nb: measure_memcpy(torch, rr, stream, nbytes=nb)[0]
                   for nb in sorted({op_out_bytes(o) for o in ops})}

    # timed region: K steps back to back, events only at its two ends (an
    # event between two kernels would stop the next one from launching while
    # the previous drains)
    try:
        gpu_id = str(torch.cuda.get_device_properties(device).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = rr.launch_count()
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            for o in ops:
                wl.run_op(rr, o, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = rr.launch_count() - launches0
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world, device)

    # per-op times (families, roofline, per-op rates): separate steps after the
    # timed region, one event between consecutive ops
    op_steps = max(1, min(args.steps, 5))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(ops) * op_steps + 1)]
    evs[0].record(stream)
    k = 1
    for _ in range(op_steps):
        for o in ops:
            wl.run_op(rr, o, stream)
            evs[k].record(stream)
            k += 1
    torch.cuda.synchronize()
    per_op = np.zeros(len(ops))
    k = 1
    for _ in range(op_steps):
        for i in range(len(ops)):
            per_op[i] += evs[k - 1].elapsed_time(evs[k]) / 1e3
            k += 1
    per_op *= args.steps / op_steps  # per-op totals over as many steps as the timed region ran
    value = replica_value(world, step_bytes, args.steps, elapsed)

    # roofline of the dominant kernel family
    fam_time, fam_bytes, fam_launch = {}, {}, {}
    for i, o in enumerate(ops):
        f = fams[i]
        fam_time[f] = fam_time.get(f, 0.0) + per_op[i]
        fam_bytes[f] = fam_bytes.get(f, 0) + op_bytes(o) * args.steps
        fam_launch[f] = fam_launch.get(f, 0) + args.steps
    dom = max(fam_time, key=fam_time.get)
    peak, peak_kind = measured_peak()
    achieved = fam_bytes[dom] / fam_time[dom] / 1e9
    traffic = load_traffic_summary()
    roofline = {"bound": "hbm", "kernel": f"k_tile_fast family ({dom})" if dom == "tile" else dom,
                "achieved": round(achieved, 1), "peak": peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "frac_of_memcpy": round(achieved / memcpy_gbs, 4),
                "algorithmic_bytes_per_launch": int(fam_bytes[dom] / fam_launch[dom]),
                "traffic": None, "traffic_source": None}
    fam_traffic = (traffic or {}).get("families", {}).get(dom)
    if fam_traffic:
        # DRAM bytes per launch from the committed ncu capture, scaled from the
        # captured case to the mean launch of this family by algorithmic bytes
        roofline["traffic"] = int(fam_traffic["ratio_to_algorithmic"] * roofline["algorithmic_bytes_per_launch"])
        roofline["traffic_source"] = "profiles/traffic.json (" + fam_traffic["measured_case"] + ", scaled)"
    families = {f: {"gbs": round(fam_bytes[f] / fam_time[f] / 1e9, 1), "time_share": round(fam_time[f] / sum(fam_time.values()), 4),
                    "launches_per_step": fam_launch[f] // args.steps} for f in fam_time}
    per_op_gbs = [round(op_bytes(o) * args.steps / per_op[i] / 1e9, 1) for i, o in enumerate(ops)]
    # payload bytes (R+W, index reads left out) per op against a copy of the same size
    per_op_frac_same = [round(2 * op_out_bytes(o) * args.steps / per_op[i] / 1e9 / memcpy_same[op_out_bytes(o)], 4)
                        for i, o in enumerate(ops)]

    # end to end through the public API with pinned host buffers
    t_e2e, e2e_steps, h2d, d2h, direct = run_e2e(torch, rr, wl, ops, stream, args)
    t_e2e = max_over_ranks(t_e2e, world, device)
    e2e = {"value": round(replica_value(world, step_bytes, e2e_steps, t_e2e), 1), "unit": "GB/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "direct_ops_per_step": direct,
           "how": "rearr_pipeline_* on pinned host buffers; ops whose plans stream run their kernel on the "
                  "host buffers over the coherent host link (direct ops), the others are staged through "
                  "device slots with overlapped copies"}

    batched = None if args.no_batched else run_batched(torch, rr, stream, device)
    serving = None if args.no_serving else run_serving(torch, rr, device)
    configs = None if (args.no_configs or rank != 0) else measure_configs(torch, rr, device, stream, 10, 3)

    result = None
    if rank == 0:
        cpu = None if (world > 1 or args.no_cpu_baseline) else cpu_baseline(wl)
        result = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded PCG64 random bit patterns)",
            "config": {"workload": WORKLOAD, "ops_per_step": len(ops), "bytes_per_step": step_bytes,
                       "elements": "2/4/8-byte elements moved as opaque bytes in 1-16-byte words, bit-exact",
                       "l2": "every operand >= 256 MiB, larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas x{world}"},
            "memcpy_d2d_gbs": round(memcpy_gbs, 1), "frac_of_memcpy": round(value / world / memcpy_gbs, 4),
            "memcpy_same_bytes_gbs": {str(k): round(v, 1) for k, v in memcpy_same.items()},
            "per_op_frac_of_memcpy_same_bytes": per_op_frac_same,
            "frac_of_8tbs": round(value / world / 8000.0, 4),
            "roofline": roofline, "families": families, "per_op_gbs": per_op_gbs,
            "gpu_launches": int(launches), "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu,
            "batched": batched, "serving": serving, "configs": configs,
            "source_digest": source_digest(),
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


# ---------------------------------------------------------------------------
# batched form: the uneven 4096-op mix, one graph replay vs one call per op

def batch_buffers(torch, ops, device):
    """Device buffers for every op of a mix, carved from one pool (256-byte
    aligned).  Payload bytes are filled by torch's device RNG (contents are not
    checked here; the parity tests check them); reorder indices are device
    random permutations."""
    def al(x):
        return (x + 255) // 256 * 256
    sizes = []
    for o in ops:
        e = o["elem_bytes"]
        if o["kind"] == "permute":
            n = int(np.prod(o["dims"]))
            sizes.append([n * e, n * e])
        elif o["kind"] == "reorder":
            sizes.append([o["n"] * e, o["n"] * 4, o["n"] * e])
        elif o["kind"] == "interlace":
            sizes.append([o["n"] * e] * o["k"] + [o["n"] * o["k"] * e])
        else:
            sizes.append([o["n"] * o["k"] * e] + [o["n"] * e] * o["k"])
    total = sum(al(x) for sz in sizes for x in sz)
    pool = torch.empty(total, dtype=torch.uint8, device=device)
    pool.random_()
    base = pool.data_ptr()
    off = 0
    bufs = []
    for o, sz in zip(ops, sizes):
        ptrs = []
        for x in sz:
            ptrs.append(base + off)
            off += al(x)
        if o["kind"] == "reorder":
            n = o["n"]
            perm = torch.randperm(n, device=device, dtype=torch.int64).to(torch.int32)
            start = ptrs[1] - base
            pool[start:start + 4 * n].copy_(perm.view(torch.uint8))
        bufs.append(ptrs)
    return pool, bufs


def issue_single(rr, o, p, stream):
    e = o["elem_bytes"]
    if o["kind"] == "permute":
        rr.permute(p[1], p[0], e, o["dims"], o["perm"], stream)
    elif o["kind"] == "reorder":
        rr.reorder(p[2], p[0], p[1], o["n"], e, stream)
    elif o["kind"] == "interlace":
        rr.interlace(p[-1], p[:-1], o["n"], e, stream)
    else:
        rr.deinterlace(p[1:], p[0], o["n"], e, stream)


def add_to_plan(plan, o, p):
    e = o["elem_bytes"]
    if o["kind"] == "permute":
        plan.add_permute(p[1], p[0], e, o["dims"], o["perm"])
    elif o["kind"] == "reorder":
        plan.add_reorder(p[2], p[0], p[1], o["n"], e)
    elif o["kind"] == "interlace":
        plan.add_interlace(p[-1], p[:-1], o["n"], e)
    else:
        plan.add_deinterlace(p[1:], p[0], o["n"], e)


def run_batched(torch, rr, stream, device, n_ops=4096, reps=5):
    import synth
    ops = synth.batch_mix(seed=1, n_ops=n_ops)
    pool, bufs = batch_buffers(torch, ops, device)
    total_bytes = sum(synth.op_bytes(o) for o in ops)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        e.synchronize()
        return s.elapsed_time(e) / 1e3 / reps

    def plain():
        for o, p in zip(ops, bufs):
            issue_single(rr, o, p, stream)

    t_plain = timed(plain, reps)
    l0 = rr.launch_count()
    plan = rr.Plan()
    t0 = time.perf_counter()
    for o, p in zip(ops, bufs):
        add_to_plan(plan, o, p)
    plan.finalize(stream)
    t_build = time.perf_counter() - t0
    t_batch = timed(lambda: plan.run(stream), reps)
    n_ops_plan, n_tiles = plan.stats()
    plan.close()

    # the same kernel on each op class of the mix alone (one plan per class)
    def op_class(o):
        if o["kind"] == "permute":
            return "permute:" + rr.describe_permute(o["elem_bytes"], o["dims"], o["perm"])["kind"]
        return "reorder" if o["kind"] == "reorder" else "interlace/de-interlace"
    classes = {}
    for o, p in zip(ops, bufs):
        classes.setdefault(op_class(o), []).append((o, p))
    per_class = {}
    for name, members in sorted(classes.items()):
        cp = rr.Plan()
        for o, p in members:
            add_to_plan(cp, o, p)
        cp.finalize(stream)
        t = timed(lambda: cp.run(stream), reps)
        cp.close()
        nb = sum(synth.op_bytes(o) for o, _ in members)
        per_class[name] = {"ops": len(members), "bytes": int(nb), "ms": round(t * 1e3, 3), "gbs": round(nb / t / 1e9, 1)}
    del pool
    peak, peak_kind = measured_peak()
    achieved = total_bytes / t_batch / 1e9
    roofline = {"bound": "hbm", "kernel": "k_batch (one persistent launch over the whole mix)",
                "achieved": round(achieved, 1), "peak": peak,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)", "unit": "GB/s",
                "frac": round(achieved / peak, 4), "algorithmic_bytes_per_launch": int(total_bytes),
                "traffic": None}
    # Most of the mix's bytes are scattered accesses: every element of a
    # reorder and every cell of a thin-plane (strided) permute is one random
    # read.  Their rate is capped by the L1's request rate, not by HBM, so the
    # mix's bound is (scattered accesses / random-read rate) + (the other
    # bytes / copy bandwidth), with the random-read rate measured here by the
    # library's own direct gather (2^24 fp32, random permutation, source in L2).
    scattered = 0
    for o in ops:
        if o["kind"] == "reorder":
            scattered += o["n"]
        elif o["kind"] == "permute" and op_class(o) == "permute:strided":
            scattered += int(np.prod(o["dims"]))
    streaming = total_bytes - sum(per_class[c]["bytes"] for c in ("reorder", "permute:strided") if c in per_class)
    rate = random_read_rate(torch, rr, stream, device)
    bound_s = scattered / rate + streaming / (peak * 1e9)
    roofline["two_resource_bound"] = {
        "scattered_accesses": int(scattered), "random_reads_per_s": round(rate, 1),
        "streaming_bytes": int(streaming), "bound_ms": round(bound_s * 1e3, 3),
        "frac": round(bound_s / t_batch, 4),
        "how": "scattered accesses at the measured random-read rate plus the other bytes at the copy peak, "
               "no overlap assumed; frac = bound / measured replay time"}
    return {"workload": f"{n_ops}-op uneven mix (seed 1): permute rank 2-5, reorder, interlace/de-interlace k 2-4; "
                        "elem 1/2/4/8 B; extents log-uniform [1,512]; op totals in [2^8, 2^22] elements",
            "bytes_per_batch": int(total_bytes), "tiles": int(n_tiles),
            "batched_ms": round(t_batch * 1e3, 3), "plain_ms": round(t_plain * 1e3, 3),
            "batched_ops_per_s": round(n_ops / t_batch, 1), "plain_ops_per_s": round(n_ops / t_plain, 1),
            "batched_gbs": round(total_bytes / t_batch / 1e9, 1), "plain_gbs": round(total_bytes / t_plain / 1e9, 1),
            "speedup": round(t_plain / t_batch, 3), "plan_build_s": round(t_build, 3),
            "launches_per_replay": 1, "kernels_per_plain_pass": n_ops, "roofline": roofline,
            "classes": per_class, "l2": "the mix's operands total about 6 GB per replay, far larger than the L2"}


def random_read_rate(torch, rr, stream, device, n=1 << 24, reps=10):
    """Elements per second of the library's direct gather by a uniform random
    permutation from a source that fits in the L2 (64 MB of fp32)."""
    import synth
    src = torch.empty(n * 4, dtype=torch.uint8, device=device).random_()
    dst = torch.empty_like(src)
    idx = torch.from_numpy(synth.random_permutation(11, n).view(np.uint8)).to(device)
    med, _ = _time_calls(torch, stream, lambda: rr.reorder(dst, src, idx, n, 4, stream), reps, 3)
    del src, dst, idx
    return n / med


# ---------------------------------------------------------------------------
# serving: Poisson arrivals into the request loop, batched vs plain

def serving_trace(n_req, seed=2):
    """95 % of requests from the uneven mix, 5 % large rank-3/4 fp32 permutes of
    256 MB - 1 GB with random perms, in a seeded random order."""
    import synth
    g = synth.rng(seed)
    mix = synth.batch_mix(seed=seed, n_ops=n_req)
    ops = []
    for i in range(n_req):
        ops.append(synth.large_permute(g) if g.random() < 0.05 else mix[i])
    return ops


def pct(v, q):
    return float(np.percentile(np.asarray(v), q))


def run_serving(torch, rr, device, n_req=6000, budget=64 << 30):
    import synth
    ops = serving_trace(n_req)
    templates, keep = [], []
    for o in ops:
        row = [None] * 4
        if o["kind"] == "reorder":  # valid indices are part of a reorder request's payload
            p = torch.randperm(o["n"], device=device, dtype=torch.int64).to(torch.int32)
            keep.append(p)
            row[1] = p
        templates += row
    total_bytes = sum(synth.op_bytes(o) for o in ops)

    def run(batching, arrivals):
        srv = rr.Server(budget_bytes=budget, n_streams=3, max_batch_ops=1024, batching=batching,
                        poll_interval_us=10)
        lat, wall = srv.run_trace(ops, arrivals, templates, timeout_us=600_000_000)
        st = srv.stats()
        srv.close()
        lat_ms = [x * 1e3 for x in lat]
        return {"p50_ms": round(pct(lat_ms, 50), 3), "p99_ms": round(pct(lat_ms, 99), 3),
                "mean_ms": round(float(np.mean(lat_ms)), 3), "ops_per_s": round(n_req / wall, 1),
                "gbs": round(total_bytes / wall / 1e9, 1), "launches": int(st["launches"]),
                "slab_peak_gb": round(st["slab_peak"] / 1e9, 2)}

    zero = np.zeros(n_req)
    run(False, zero)  # warm-up (module load, first launches)
    sat_plain = run(False, zero)
    sat_batched = run(True, zero)
    rates = []
    for f in (0.5, 0.9, 1.5):
        r = f * sat_plain["ops_per_s"]
        arr = synth.poisson_arrivals(100 + int(10 * f), r, n_req)
        rates.append({"offered_x_plain_saturated": f, "offered_ops_per_s": round(r, 1),
                      "batched": run(True, arr), "plain": run(False, arr)})
    del keep
    return {"workload": f"{n_req} requests: 95 % uneven mix (seed 2), 5 % rank-3/4 fp32 permutes of 256 MB - 1 GB; "
                        "Poisson arrivals; 64 GB device budget; 3 streams; batched = continuous batching into the "
                        "persistent kernel, plain = one single-op launch per request",
            "bytes": int(total_bytes), "saturated": {"plain": sat_plain, "batched": sat_batched}, "rates": rates}


def run_e2e(torch, rr, wl, ops, stream, args):
    """Same step through the public host-buffer API (rearr_pipeline_*): every
    op's inputs cross the host link from pinned host memory and its output
    back inside the timed region -- read and written by the kernel itself for
    direct ops, else copied with the upload of op i+1, the kernel of op i and
    the download of op i-1 overlapped on the pipeline's three streams."""
    max_in = wl.dst.numel()
    h_src = torch.empty(max_in, dtype=torch.uint8, pin_memory=True)
    h_src.copy_(torch.from_numpy(wl.src_np.view(np.uint8)))
    h_dst = torch.empty(max_in, dtype=torch.uint8, pin_memory=True)
    h_idx = {k: torch.from_numpy(v.view(np.uint8)).pin_memory() for k, v in wl.idx_np.items()}
    h2d = sum(op_in_bytes(o) for o in ops)
    d2h = sum(op_out_bytes(o) for o in ops)
    slot = max(op_in_bytes(o) + op_out_bytes(o) for o in ops) + (4 << 10)
    pipe = rr.Pipeline(slot_bytes=slot, slots=3)

    def step():
        for o in ops:
            if o["kind"] == "reorder":
                pipe.reorder(h_dst, h_src, h_idx[o["idx"]], o["n"], o["elem_bytes"])
            else:
                pipe.permute(h_dst, h_src, o["elem_bytes"], o["dims"], o["perm"])

    steps = args.steps if args.e2e_steps <= 0 else max(1, min(args.steps, args.e2e_steps))
    step()
    pipe.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    pipe.sync()
    t = time.perf_counter() - t0
    st = pipe.stats()
    direct = pipe.direct()["direct_ops"] // (steps + 1)
    pipe.close()
    assert st["h2d_bytes"] == (steps + 1) * h2d and st["d2h_bytes"] == (steps + 1) * d2h
    return t, steps, int(h2d), int(d2h), int(direct)


# ---------------------------------------------------------------------------
# CPU oracle legs

CPU_SAMPLE = [dict(kind="permute", elem_bytes=4, dims=[512, 512, 512], perm=[2, 0, 1]),
              dict(kind="permute", elem_bytes=4, dims=[64, 128, 256, 64], perm=[3, 1, 2, 0]),
              dict(kind="permute", elem_bytes=8, dims=[64, 128, 256, 64], perm=[0, 3, 2, 1]),
              dict(kind="permute", elem_bytes=2, dims=[64, 128, 256, 64], perm=[2, 3, 0, 1]),
              dict(kind="reorder", elem_bytes=4, n=1 << 28, idx="random")]


def oracle_run(orc, o, src_np, idx_np):
    if o["kind"] == "permute":
        n = int(np.prod(o["dims"])) * o["elem_bytes"]
        orc.permute(src_np.view(np.uint8)[:n], o["elem_bytes"], o["dims"], o["perm"])
    else:
        orc.reorder(src_np.view(np.uint8)[:o["n"] * o["elem_bytes"]], idx_np, o["elem_bytes"])


def cpu_baseline(wl, sample=CPU_SAMPLE):
    """The oracle (single-threaded C loop nest) on a bounded sample of the workload."""
    import oracle
    orc = oracle.get()
    total_b, total_t = 0, 0.0
    for o in sample:
        idx = wl.idx_np.get(o.get("idx")) if o["kind"] == "reorder" else None
        t0 = time.perf_counter()
        oracle_run(orc, o, wl.src_np, idx)
        total_t += time.perf_counter() - t0
        total_b += op_bytes(o)
    return {"value": round(total_b / total_t / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "one pass of: 512^3 fp32 order (2,0,1); 64x128x256x64 orders (3,1,2,0) at 4 B, (0,3,2,1) "
                      "at 8 B, (2,3,0,1) at 2 B; reorder of 2^28 fp32 by a random permutation",
            "seconds": round(total_t, 2), "cpu": cpu_model()}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip() + f" ({os.cpu_count()} cpus)"
    except OSError:
        pass
    return f"{os.cpu_count()} cpus"


class _HostWL:
    def __init__(self):
        import synth
        self.src_np = synth.random_elements(20260101, (1 << 30) // 4, 4)
        self.idx_np = {"random": synth.random_permutation(7, 1 << 28)}


def run_reference(args):
    """The oracle as it stands, timed on the host cores: each step runs one op
    of a bounded sample of the workload (rotating)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    orc = oracle.get()
    wl = _HostWL()
    seq = CPU_SAMPLE
    for i in range(args.warmup):
        o = seq[i % len(seq)]
        oracle_run(orc, o, wl.src_np, wl.idx_np.get(o.get("idx")))
    total_b, total_t = 0, 0.0
    for i in range(args.steps):
        o = seq[i % len(seq)]
        t0 = time.perf_counter()
        oracle_run(orc, o, wl.src_np, wl.idx_np.get(o.get("idx")))
        total_t += time.perf_counter() - t0
        total_b += op_bytes(o)
    value = total_b / total_t / 1e9
    # n_gpus is the launch's N (the oracle itself runs on one host thread of rank 0)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", args.gpus)),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_t / args.steps * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded PCG64 random bit patterns)",
            "config": {"workload": WORKLOAD, "parallelism": "single CPU thread (the oracle on the host)"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "each step runs one op of: 512^3 fp32 (2,0,1); 64x128x256x64 (3,1,2,0) 4 B, "
                                       "(0,3,2,1) 8 B, (2,3,0,1) 2 B; reorder 2^28 fp32 random (rotating)",
                             "cpu": cpu_model()},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def parse_case(spec: str):
    """Single-op case spec: permute:E:d0,d1,..:p0,p1,.. | reorder:E:n:random|block4096 |
    interlace:E:n:k | deinterlace:E:n:k | nm:E:dims:order:base:range (comma lists);
    batch:N, stencil:TAPS:NY:NX[:BOUNDARY] and dist:E:dims:perm:P are handled by
    their own runners."""
    parts = spec.split(":")
    kind, e = parts[0], int(parts[1])
    if kind == "permute":
        return dict(kind=kind, elem_bytes=e, dims=[int(x) for x in parts[2].split(",")],
                    perm=[int(x) for x in parts[3].split(",")])
    if kind in ("reorder", "scatter", "reorder64", "scatter64"):
        return dict(kind=kind, elem_bytes=e, n=int(parts[2]), idx=parts[3])
    if kind in ("interlace", "deinterlace"):
        return dict(kind=kind, elem_bytes=e, n=int(parts[2]), k=int(parts[3]))
    if kind == "nm":
        ints = [[int(x) for x in q.split(",")] for q in parts[2:6]]
        return dict(kind=kind, elem_bytes=e, dims=ints[0], order=ints[1], base=ints[2], range=ints[3])
    raise SystemExit(f"unknown case kind {kind}")


def stencil_taps(name: str):
    """fdN: order-N finite-difference Laplacian; boxN: (2N+1)^2 mean filter;
    crossN: seeded random weights on the full cross of radius N; genK: K
    seeded random taps within radius 4."""
    from synth.stencils import fd_laplacian
    g = np.random.default_rng(17)
    if name.startswith("fd"):
        return fd_laplacian(int(name[2:]))
    r = int(name[3:]) if name[:3] in ("box", "gen") else int(name[5:])
    if name.startswith("box"):
        return [(dy, dx, 1.0 / (2 * r + 1) ** 2) for dy in range(-r, r + 1) for dx in range(-r, r + 1)]
    if name.startswith("cross"):
        return [(d, 0, float(g.normal())) for d in range(-r, r + 1)] + \
               [(0, d, float(g.normal())) for d in range(-r, r + 1) if d]
    return [(int(g.integers(-4, 5)), int(g.integers(-4, 5)), float(g.normal())) for _ in range(r)]


def run_stencil_case(torch, rr, stream, dev, spec, args):
    """stencil:TAPS:NY:NX[:BOUNDARY] -- the 2-D stencil on a float grid (Table 4
    uses fd1 on 4096 x 4096).  L2 is flushed before every timed call (the
    4096^2 grid fits in L2), and a device copy of the same bytes is timed the
    same way as the bandwidth reference."""
    parts = spec.split(":")
    taps = stencil_taps(parts[1])
    ny, nx = int(parts[2]), int(parts[3])
    boundary = int(parts[4]) if len(parts) > 4 else 0
    gen = torch.Generator(device=dev).manual_seed(5)
    src = torch.randn((ny, nx), device=dev, generator=gen, dtype=torch.float32)
    dst = torch.empty_like(src)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    nbytes = 2 * ny * nx * 4

    def timed(call):
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            call()
            s1.record(stream)
            s1.synchronize()
            ts.append(s0.elapsed_time(s1) / 1e3)
        return ts

    t = timed(lambda: rr.stencil2d(dst, src, ny, nx, taps, boundary, stream))
    c = timed(lambda: rr.memcpy_d2d(dst, src, ny * nx * 4, stream))
    med, cmed = statistics.median(t), statistics.median(c)
    return {"case": spec, "bytes": nbytes, "median_ms": round(med * 1e3, 4), "best_ms": round(min(t) * 1e3, 4),
            "gbs_median": round(nbytes / med / 1e9, 1), "gbs_best": round(nbytes / min(t) / 1e9, 1),
            "copy_gbs_median": round(nbytes / cmed / 1e9, 1), "l2": "flushed before each call",
            "plan": rr.describe_stencil(ny, nx, taps, boundary, dst.data_ptr(), src.data_ptr()),
            "steps": args.steps}


def run_dist_case(torch, rr, stream, dev, spec, args):
    """dist:E:d0,d1,..:p0,p1,..:P -- the distributed permute's local steps for
    P ranks emulated on one GPU: every rank's pack, the exchange (a device
    permute of the P x P pieces standing in for the all-to-all) and every
    rank's unpack, each timed on its own.  GB/s counts the read + write of all
    P slabs."""
    parts = spec.split(":")
    e, P = int(parts[1]), int(parts[4])
    dims, perm = [int(x) for x in parts[2].split(",")], [int(x) for x in parts[3].split(",")]
    plan = rr.dist_permute_plan(e, dims, perm, P)
    sb = plan.slab_bytes
    glob = torch.empty(sb * P, dtype=torch.uint8, device=dev).random_()
    send, recv, out = torch.empty_like(glob), torch.empty_like(glob), torch.empty_like(glob)
    first = send if plan.exchange else out

    def pack():
        for r in range(P):
            rr.dist_permute_pack(first[r * sb:(r + 1) * sb], glob[r * sb:(r + 1) * sb], plan, e, stream)

    def exchange():
        rr.permute(recv, send, 1, [P, P, plan.piece_bytes], [1, 0, 2], stream)

    def unpack():
        for r in range(P):
            rr.dist_permute_unpack(out[r * sb:(r + 1) * sb], recv[r * sb:(r + 1) * sb], plan, e, stream)

    nbytes = 2 * sb * P
    res = {"case": spec, "bytes_per_step": nbytes, "exchange": bool(plan.exchange), "steps": args.steps,
           "pack_permute": plan.pack(), "unpack_permute": plan.unpack() if plan.exchange else None}
    for name, call in (("pack", pack), ("exchange", exchange), ("unpack", unpack)):
        if name != "pack" and not plan.exchange:
            continue
        med, best = _time_calls(torch, stream, call, args.steps, args.warmup)
        res[name] = {"median_ms": round(med * 1e3, 4), "gbs_median": round(nbytes / med / 1e9, 1)}
    return res


def run_case(args):
    """Time one op (used for profiling captures and sweeps): W untimed and K
    timed calls on one stream, CUDA events around each call."""
    import torch
    import synth
    from paper_1011_3583_gb300 import build as rbuild
    rbuild.build()
    import paper_1011_3583_gb300 as rr
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    if args.case.startswith("batch:"):
        return run_batch_case(torch, rr, stream, dev, int(args.case.split(":")[1]), args)
    if args.case.startswith("stencil:"):
        return run_stencil_case(torch, rr, stream, dev, args.case, args)
    if args.case.startswith("dist:"):
        return run_dist_case(torch, rr, stream, dev, args.case, args)
    o = parse_case(args.case)
    e = o["elem_bytes"]
    if o["kind"] == "nm":
        n = int(np.prod(o["dims"]))
        total = int(np.prod([o["range"][a] for a in o["order"]]))
        src = torch.empty(n * e, dtype=torch.uint8, device=dev).random_()
        dst = torch.empty(total * e, dtype=torch.uint8, device=dev)
        call = lambda: rr.reorder_nm(dst, src, e, o["dims"], o["order"], o["base"], o["range"], stream)  # noqa: E731
        nbytes = 2 * total * e
    elif o["kind"] in ("permute", "reorder", "scatter", "reorder64", "scatter64"):
        n = int(np.prod(o["dims"])) if o["kind"] == "permute" else o["n"]
        src = torch.empty(n * e, dtype=torch.uint8, device=dev).random_()
        dst = torch.empty(n * e, dtype=torch.uint8, device=dev)
        if o["kind"] != "permute":
            a = (synth.random_permutation(7, n) if o["idx"] == "random"
                 else synth.block_shuffled_permutation(8, n, 4096))
            wide = o["kind"].endswith("64")
            if wide:
                a = a.astype(np.uint64)
            idx = torch.from_numpy(a.view(np.uint8)).to(dev)
            fn = {"reorder": rr.reorder, "scatter": rr.scatter, "reorder64": rr.reorder64,
                  "scatter64": rr.scatter64}[o["kind"]]
            call = lambda: fn(dst, src, idx, n, e, stream)  # noqa: E731
            nbytes = 2 * n * e + (8 if wide else 4) * n
        else:
            call = lambda: rr.permute(dst, src, e, o["dims"], o["perm"], stream)  # noqa: E731
            nbytes = 2 * n * e
    else:
        n, k = o["n"], o["k"]
        planes = [torch.empty(n * e, dtype=torch.uint8, device=dev).random_() for _ in range(k)]
        inter = torch.empty(n * k * e, dtype=torch.uint8, device=dev).random_()
        if o["kind"] == "interlace":
            call = lambda: rr.interlace(inter, planes, n, e, stream)  # noqa: E731
        else:
            call = lambda: rr.deinterlace(planes, inter, n, e, stream)  # noqa: E731
        nbytes = 2 * n * k * e
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        call()
        s1.record(stream)
        s1.synchronize()
        times.append(s0.elapsed_time(s1) / 1e3)
    med = statistics.median(times)
    plan = rr.describe_permute(e, o["dims"], o["perm"]) if o["kind"] == "permute" else None
    return {"case": args.case, "bytes": nbytes, "median_ms": round(med * 1e3, 4),
            "best_ms": round(min(times) * 1e3, 4), "gbs_median": round(nbytes / med / 1e9, 1),
            "gbs_best": round(nbytes / min(times) / 1e9, 1), "plan": plan, "steps": args.steps}


def _time_calls(torch, stream, call, steps, warmup, flush=None):
    """Per-call CUDA-event times on `stream`; `flush` (untimed) runs before each."""
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        if flush is not None:
            flush()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        call()
        s1.record(stream)
        s1.synchronize()
        ts.append(s0.elapsed_time(s1) / 1e3)
    return statistics.median(ts), min(ts)


def measure_configs(torch, rr, dev, stream, steps, warmup):
    """The single-op configs beside the bench step, each timed per call with
    CUDA events against a device copy of the same bytes timed the same way
    (L2 flushed before each call where the operands are comparable to the
    L2): the 1024^2 fp32 transpose (warm and flushed), every interlace and
    de-interlace case of the interlace config, and the 2-D stencil of Table 4
    (4096^2 fp32 grid, finite-difference orders I-IV).  GB/s counts bytes
    read + bytes written."""
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def flush():
        with torch.cuda.stream(stream):
            flush_buf.fill_(1)

    out = []

    def timed_queued(call, reps=20):
        """Per-call device time of `reps` back-to-back calls on a warm L2.  A
        spin kernel of about a millisecond runs first, so that the host has
        queued every call before the GPU reaches them: the timing holds no
        host launch gap, only the calls themselves."""
        for _ in range(warmup):
            call(stream)
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                torch.cuda._sleep(2_000_000)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(reps):
                call(stream)
            s1.record(stream)
            s1.synchronize()
            ts.append(s0.elapsed_time(s1) / 1e3 / reps)
        return statistics.median(ts), min(ts)

    def record(name, nbytes_moved, call, copy_bytes, flushed):
        """call(stream) issues the op.  Flushed: one call per timing, the L2
        flushed before it (the flush also hides the host's launch gap).
        Warm: back-to-back calls queued behind a spin kernel."""
        a = torch.empty(copy_bytes, dtype=torch.uint8, device=dev)
        b = torch.empty_like(a)
        copy = lambda st: rr.memcpy_d2d(b, a, copy_bytes, st)  # noqa: E731
        if flushed:
            med, best = _time_calls(torch, stream, lambda: call(stream), steps, warmup, flush)
            cmed, _ = _time_calls(torch, stream, lambda: copy(stream), steps, warmup, flush)
        else:
            med, best = timed_queued(call)
            cmed, _ = timed_queued(copy)
        del a, b
        out.append({"config": name, "l2": "flushed" if flushed else "warm (20 back-to-back calls)",
                    "bytes": nbytes_moved,
                    "median_us": round(med * 1e6, 2), "best_us": round(best * 1e6, 2),
                    "gbs": round(nbytes_moved / med / 1e9, 1), "memcpy_gbs": round(2 * copy_bytes / cmed / 1e9, 1),
                    "frac_of_memcpy": round((nbytes_moved / med) / (2 * copy_bytes / cmed), 3)})

    # config 1: one 1024 x 1024 fp32 transpose
    n = 1024 * 1024 * 4
    src = torch.empty(n, dtype=torch.uint8, device=dev).random_()
    dst = torch.empty_like(src)
    for flushed in (False, True):
        record("transpose 1024x1024 fp32", 2 * n, lambda st: rr.permute(dst, src, 4, [1024, 1024], [1, 0], st), n,
               flushed)
    del src, dst
    # interlace config: complex split, image planes, AoS/SoA
    cases = [("complex64 2^28 <-> 2 fp32 planes", 4, 1 << 28, 2)] + \
            [(f"4096^2 uint8 x {k} planes", 1, 4096 * 4096, k) for k in (3, 4)] + \
            [(f"AoS/SoA 2^26 records x {k} fp32", 4, 1 << 26, k) for k in (2, 3, 4, 8)]
    for name, e, n, k in cases:
        planes = [torch.empty(n * e, dtype=torch.uint8, device=dev).random_() for _ in range(k)]
        inter = torch.empty(n * k * e, dtype=torch.uint8, device=dev).random_()
        flushed = n * k * e < (256 << 20)  # comparable to L2: flush
        record(name + " interlace", 2 * n * k * e, lambda st: rr.interlace(inter, planes, n, e, st), n * k * e,
               flushed)
        record(name + " de-interlace", 2 * n * k * e, lambda st: rr.deinterlace(planes, inter, n, e, st),
               n * k * e, flushed)
        del planes, inter
    # Table 4: the 2-D stencil on a 4096 x 4096 fp32 grid, orders I-IV
    gen = torch.Generator(device=dev).manual_seed(5)
    grid = torch.randn((4096, 4096), device=dev, generator=gen, dtype=torch.float32)
    gout = torch.empty_like(grid)
    for order in (1, 2, 3, 4):
        taps = stencil_taps(f"fd{order}")
        record(f"stencil 4096^2 fp32 FD order {order} (zero boundary)", 2 * grid.numel() * 4,
               lambda st: rr.stencil2d(gout, grid, 4096, 4096, taps, 0, st), grid.numel() * 4, True)
    del grid, gout, flush_buf
    return out


def run_configs(args):
    """--configs: measure_configs alone, printed as one JSON line."""
    import torch
    from paper_1011_3583_gb300 import build as rbuild
    rbuild.build()
    import paper_1011_3583_gb300 as rr
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    out = measure_configs(torch, rr, dev, stream, args.steps, args.warmup)
    return {"configs": out, "steps": args.steps, "warmup": args.warmup, "timing": "CUDA events per call"}


def run_batch_case(torch, rr, stream, dev, n_ops, args):
    """batch:N -- the first N ops of the uneven mix as one plan, replayed."""
    import synth
    ops = synth.batch_mix(seed=1, n_ops=n_ops)
    pool, bufs = batch_buffers(torch, ops, dev)
    plan = rr.Plan()
    for o, p in zip(ops, bufs):
        add_to_plan(plan, o, p)
    plan.finalize(stream)
    nbytes = sum(synth.op_bytes(o) for o in ops)
    for _ in range(args.warmup):
        plan.run(stream)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        plan.run(stream)
        s1.record(stream)
        s1.synchronize()
        times.append(s0.elapsed_time(s1) / 1e3)
    plan.close()
    med = statistics.median(times)
    return {"case": args.case, "bytes": nbytes, "median_ms": round(med * 1e3, 4),
            "gbs_median": round(nbytes / med / 1e9, 1), "ops_per_s": round(n_ops / med, 1), "steps": args.steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="librearr", choices=["librearr", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=0, help="e2e steps (0: the same as --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--case", default=None, help="time one op instead of the workload (see parse_case)")
    ap.add_argument("--configs", action="store_true", help="time the single-op configs (transpose, interlace)")
    args = ap.parse_args()
    if args.case:
        print(json.dumps(run_case(args)), flush=True)
        return
    if args.configs:
        print(json.dumps(run_configs(args)), flush=True)
        return
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
