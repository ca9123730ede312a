"""Benchmark: certified roots per second of the level-line Newton splitter.

Default workload: all 2^19 = 524,288 roots of p_20 (hyperbolic centres of
periods dividing 20) in plain binary64, every root certified by the disk
test.  A step is one full call of mt_split_hyperbolic(20): seeds, level-line
walk, Newton descents, root set, types, certificates, sorted output.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config hyp20]
    python bench.py --impl reference ...   # the CPU oracle on the same metric

For N > 1 (torchrun) every rank splits its own copy of the workload
(replicas: one polynomial is split on one GPU; sharding it would need a
cross-rank exchange of the level-line seeds and of the root set), timing
is the max over ranks, value = all ranks' roots / that time.  Prints one
JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "certified roots/sec at period n (1 GB300)"
CONFIGS = {
    # name: (kind, l, n, precision)
    "hyp12": ("hyp", 0, 12, "fp64"),
    "hyp20": ("hyp", 0, 20, "fp64"),
    "hyp20mixed": ("hyp", 0, 20, "mixed"),
    "hyp24": ("hyp", 0, 24, "fp64"),
    "hyp24mixed": ("hyp", 0, 24, "mixed"),
    "hyp26dd": ("hyp", 0, 26, "dd"),
    "hyp28dd": ("hyp", 0, 28, "dd"),  # binary64 cannot separate its tip roots: dd zones
    "mis16": ("misbatch", 0, 16, "fp64"),  # every s_{l,n}, l >= 2, n >= 1, l + n <= 16, one pass
}


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 work of one Newton step on an orbit of length m (binary64 flops, FMA = 2):
# orbit step: 2 add + 5 FMA + 2 mul = 14 flops; quotient with power-of-two
# scaling, target subtraction and update: 24 flops.
def newton_flops(m: int) -> int:
    return 14 * m + 24


# Nominal binary64 rate of a GB300 (profiling recipe table): 1.25 TFLOP/s
# at the 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 1.25
SM_MAX_MHZ = 2070.0


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(kind: str, l: int, n: int, target_s: float = 15.0) -> dict:
    """The binary64 oracle, as it stands, on a bounded sample of the same
    workload: the first fraction of the level line (walk + descents + set).
    Rate = roots in that fraction of the line / time (single thread)."""
    import oracle
    d = oracle.degree(kind, n, l)
    frac = 1.0 / 64
    t0 = time.perf_counter()
    oracle.split(kind, n, l=l, fp64=True, frac=frac, want_types=False)
    dt = time.perf_counter() - t0
    # grow the sample to about target_s seconds (bounded: at most the whole line)
    if dt < target_s:
        frac = min(1.0, frac * target_s / max(dt, 1e-3))
        t0 = time.perf_counter()
        oracle.split(kind, n, l=l, fp64=True, frac=frac, want_types=False)
        dt = time.perf_counter() - t0
    return {"value": d * frac / dt, "unit": "roots/s", "cores": 1, "kind": "oracle",
            "sample": "binary64 oracle (same algorithm, sequential walk), first %.4f of the level line of "
                      "%s n=%d, %.1f s, 1 thread; rate = degree x fraction / time" % (frac, kind, n, dt)}


def run_reference(args, cfg):
    kind, l, n, prec = cfg
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    d = oracle.degree(kind, n, l)
    frac = 1.0 / 32  # each step: a bounded sample of the same workload
    for _ in range(args.warmup):
        oracle.split(kind, n, l=l, fp64=True, frac=frac, want_types=False)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.split(kind, n, l=l, fp64=True, frac=frac, want_types=False)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = d * frac / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s n=%d (%d roots)" % (kind, n, d), "precision": prec,
                   "sample": "first %.4f of the level line per step" % frac},
        "cpu_baseline": {"value": value, "unit": "roots/s", "cores": 1, "kind": "oracle",
                         "sample": "binary64 oracle, first %.4f of the level line per step, 1 thread" % frac},
        "e2e": {"value": value, "unit": "roots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="hyp20", choices=sorted(CONFIGS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the mixed-tier comparison")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)

    import numpy as np
    import torch
    import paper_2402_06083_gb300 as mt

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    kind, l, n, prec = cfg
    if kind == "misbatch":
        d = sum(2 ** (a + b - 2) for a, b in mt.misiurewicz_pairs(n))
    else:
        d = mt.degree(kind, n, l)
    stream = torch.cuda.current_stream()
    work = mt.Workspace()
    roots = torch.empty((d, 2), dtype=torch.float64, device="cuda")
    roots_lo = torch.empty((d, 2), dtype=torch.float64, device="cuda") if prec == "dd" else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    class _BatchResult:
        def __init__(self, stats):
            tot = dict(stats[0])
            tot["n_roots"] = sum(x["n_roots"] for x in stats)
            tot["n_cert_pass"] = sum(x["n_cert_pass"] for x in stats)
            tot["steps_fp32"] = 0
            self.stats = tot

    def step(out=None, p=None):
        pp = prec if p is None else p
        if kind == "hyp":  # the launch sequence is captured once and replayed as a CUDA graph
            return mt.split_hyperbolic(n, pp, work=work, out=roots, use_graph=1,
                                       out_lo=roots_lo if pp == "dd" else None)
        if kind == "misbatch":
            _, _, _, st, _ = mt.split_misiurewicz_batch(n, pp, work=work)
            return _BatchResult(st)
        return mt.split_misiurewicz(l, n, pp, work=work, out=roots)

    def timed(p, steps):
        for _ in range(3):
            rr = step(p=p)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        st = []
        for i in range(steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            rr = step(p=p)
            ev[i][1].record(stream)
            st.append(rr.stats)
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev), st

    for _ in range(max(args.warmup, 3)):
        r = step()
    assert r.stats["n_roots"] == d and r.stats["n_cert_pass"] == d, r.stats
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush between timed steps (not timed)
        evs[i][0].record(stream)
        r = step()
        evs[i][1].record(stream)
        stats.append(r.stats)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(step_ms)
    # max over ranks
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    certified = min(s["n_cert_pass"] for s in stats)
    value = world * certified / (ms / 1e3)

    # end to end through the public API with a pinned host result buffer
    host = torch.empty((d, 2), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    host_lo = torch.empty((d, 2), dtype=torch.float64, pin_memory=True) if roots_lo is not None else None
    for i in range(args.steps):
        r = step()
        host.copy_(roots, non_blocking=True)
        if host_lo is not None:
            host_lo.copy_(roots_lo, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    if dist:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    clocks = sampler.stop()

    s0 = stats[-1]
    m = n if kind == "hyp" else (n - 1 if kind == "misbatch" else l + n - 1)
    fl_step = newton_flops(m)
    # dominant kernel by device time (library's CUDA events on the launch stream)
    parts = {"walk": s0["ms_walk"], "descend": s0["ms_descend"], "dedup": s0["ms_dedup"],
             "certify": s0["ms_certify"]}
    dom = max(parts, key=parts.get)
    if dom == "descend":
        flops = s0["desc_newton"] * fl_step
        dom_ms = statistics.mean(s["ms_descend"] for s in stats)
    else:
        flops = s0["walk_newton"] * fl_step
        dom_ms = statistics.mean(s["ms_walk"] for s in stats)
    achieved = flops / (dom_ms / 1e3) / 1e12
    peak = FP64_PEAK_TFLOPS
    if clocks.get("sm_mhz"):
        pass
    line = {
        "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (inputs fixed by n)",
        "config": {"workload": ("p_%d hyperbolic centres, %d roots, %s, all certified" % (
                       n, d, {"fp64": "plain binary64", "mixed": "mixed binary32/binary64",
                              "dd": "mixed binary32/binary64 + double-double zones"}[prec])
                       if kind == "hyp" else
                       ("all s_{l,n} with l >= 2, n >= 1, l + n <= %d (%d polynomials, %d roots), one pass, "
                        "binary64, all certified" % (n, len(mt.misiurewicz_pairs(n)), d))
                       if kind == "misbatch" else "s_{%d,%d}" % (l, n)),
                   "precision": prec, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": world * d / e2e_s, "unit": "roots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d * 16 * (2 if roots_lo is not None else 1) + 1024,
                "note": "input is the integer n (no device input); result roots copied to pinned host memory"},
        "roofline": {"bound": "alu", "kernel": "k_" + ("descend" if dom == "descend" else "walk"),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None,
                     "peak_source": "nominal binary64 1.25 TFLOP/s at 2070 MHz (profiling recipe table)"},
        "gpu_launches": int(sum(s["n_launches"] for s in stats)),
        "clocks": clocks,
        "detail": {"ms_walk": s0["ms_walk"], "ms_descend": s0["ms_descend"], "ms_dedup": s0["ms_dedup"],
                   "ms_certify": s0["ms_certify"], "walk_newton": s0["walk_newton"],
                   "desc_newton": s0["desc_newton"], "n_chunks": s0["n_chunks"],
                   "ms_dd": s0.get("ms_dd", 0.0), "n_zones": s0.get("n_zones", 0),
                   "n_zone_roots": s0.get("n_zone_roots", 0), "steps_dd": s0["steps_dd"],
                   "prec_used": s0["prec_used"], "wall_s": t_wall},
    }
    # the same workload in the mixed tier (binary32 tracking, binary64 finish)
    if prec == "fp64" and kind == "hyp" and not args.no_compare:
        ms_mix, st_mix = timed("mixed", args.steps)
        sm = st_mix[-1]
        line["compare"] = {
            "mixed": {"value": min(x["n_cert_pass"] for x in st_mix) / (ms_mix / 1e3), "unit": "roots/s",
                      "ms_per_step": ms_mix, "speedup_vs_fp64": ms / ms_mix,
                      "prec_used": sm["prec_used"], "steps_fp32": sm["steps_fp32"],
                      "desc_newton": sm["desc_newton"], "walk_newton": sm["walk_newton"],
                      "ms_walk": sm["ms_walk"], "ms_descend": sm["ms_descend"],
                      "ms_certify": sm["ms_certify"], "ms_dedup": sm["ms_dedup"],
                      "all_certified": all(x["n_cert_pass"] == d for x in st_mix)}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and kind != "misbatch":
        line["cpu_baseline"] = cpu_baseline(kind, l, n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
