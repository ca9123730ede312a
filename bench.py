"""Benchmark: certified roots per second of the level-line Newton splitter.

Default workload: all 2^19 = 524,288 roots of p_20 (hyperbolic centres of
periods dividing 20) in plain binary64, every root certified by the disk
test.  A step is one full call of mt_split_hyperbolic(20): seeds, level-line
walk, Newton descents, root set, types, certificates, sorted output.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config hyp20]
    python bench.py --impl reference ...   # the CPU oracle on the same metric

Other configurations: hyp12, hyp20mixed, hyp24, hyp24mixed (p_24 in the
mixed tier), hyp26dd / hyp28dd / hyp29dd / hyp31dd (double-double zones),
hyp32dd (streamed level line, ~245 GB), mis16 (every s_{l,n}, l + n <= 16,
one pass), mis26dd (s_{4,22}, beyond FP80), q18 (q_{9,9} with its multiple
roots).

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
    "hyp29dd": ("hyp", 0, 29, "dd"),
    "hyp31dd": ("hyp", 0, 31, "dd"),  # 2^30 roots, ~230 GB of device memory
    "hyp32dd": ("hyp", 0, 32, "dd"),  # 2^31 roots, streamed level line, ~245 GB of device memory
    "mis16": ("misbatch", 0, 16, "fp64"),  # every s_{l,n}, l >= 2, n >= 1, l + n <= 16, one pass
    "mis26dd": ("mis", 4, 22, "dd"),  # s_{4,22}: tip pair 4.86e-20 apart (Sec. 6.3.2), beyond FP80
    "q18": ("q", 9, 9, "fp64"),  # q_{9,9} = p_18 - p_9 with its multiple roots (Thm fact_mis)
}


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Work of one Newton step on an orbit of length m, in flops (FMA = 2): an
# orbit step counts 13 flops (the kernels run it as 6 FMA + 1 mul + 1 add,
# 14, so the count is on the low side); the quotient with its power-of-two
# guard, the target subtraction and the update about 24.
def newton_flops(m: int) -> int:
    return 13 * m + 24


# Nominal rates of a GB300 at the 2070 MHz maximum SM clock: binary64
# 1.25 TFLOP/s (profiling recipe table; 2 DFMA lanes per SM), binary32
# 152 SMs x 128 FMA lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
SM_MAX_MHZ = 2070.0


# DRAM bytes (read + write) per launch of the roofline kernel, from one ncu
# capture of the same kernel build and workload, keyed by (config, kernel).
# Only kernels unchanged since their capture are listed; the rest report
# null.  The last k_descend capture (profiles/kernels_hyp20_fp64.md:
# dram__bytes_read.sum 16.8 MB, write 0) predates its integer-pipe stop
# tests, so it is not listed.
TRAFFIC: dict = {}


def roofline(prec: str, m: int, stats: list, config: str = "", desc_flops: int | None = None) -> dict:
    """ALU roofline of the dominant kernel (walk or descent) from the
    library's own CUDA events (on the launch stream, inside the graph) and
    its own step counters.  Binary32 steps of the mixed tier count at the
    binary64/binary32 peak ratio, so frac is the share of the binary64 pipe
    the same work would need.  Walk time excludes the seed lifts."""
    fl = newton_flops(m)
    dfl = fl if desc_flops is None else desc_flops
    ratio = FP64_PEAK_TFLOPS / FP32_PEAK_TFLOPS
    s0 = stats[-1]
    walk_ms = statistics.mean(s["ms_walk"] - s["ms_seeds"] for s in stats)
    desc_ms = statistics.mean(s["ms_descend"] for s in stats)
    walk_steps = s0["walk_newton"] - s0["seed_newton"]
    if prec == "fp64":
        walk_eq = walk_steps * fl
        desc_eq = s0["desc_newton"] * dfl
    else:  # mixed walk: binary32 sub-steps; descents: binary32 then binary64 finish
        walk_eq = walk_steps * fl * ratio
        desc_eq = (s0["desc_newton"] - s0["desc_fp32"]) * fl + s0["desc_fp32"] * fl * ratio
    kern, eq, ms = ("k_descend", desc_eq, desc_ms) if desc_ms >= walk_ms else ("k_walk", walk_eq, walk_ms)
    if prec != "fp64" and s0["desc_fp32"] + s0["steps_fp32"] > 0:  # the attempt ran the mixed tier
        kern += "_mixed"
    achieved = eq / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
            "traffic": TRAFFIC.get((config, kern)),
            "ms_per_launch": ms, "flops_per_launch": eq,
            "peak_source": "nominal binary64 1.25 TFLOP/s at 2070 MHz (profiling recipe table)"
                           + ("" if prec == "fp64" else "; binary32 steps weighted by 1.25/80.5"),
            "work": ("Newton steps x (13 m + 24) flops, m = %d, steps counted by the kernel" % m)
                    + ("" if desc_flops is None else "; descents %d flops per step (product form)" % desc_flops)}


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


def separation_stats(mt, torch, n, roots, roots_lo, work, stream, reps=3) -> dict:
    """mt_separation over Hyp(n) (mask: exact period n from mt_classify) of
    the last split's roots: device ms per call and the minimum against the
    118.4 / 4^n law."""
    z = torch.view_as_complex(roots)
    mask = (mt.classify("hyp", n, z) == n).to(torch.uint8)
    lo = None if roots_lo is None else torch.view_as_complex(roots_lo)
    sw = mt.Workspace()
    mt.separation(z, roots_lo=lo, mask=mask, work=sw)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        nn, bands, mn = mt.separation(z, roots_lo=lo, mask=mask, work=sw)
        b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    size = int(mask.sum().item())
    return {"ms": ms, "set": "Hyp(%d)" % n, "roots": size, "roots_per_s": size / (ms / 1e3),
            "min_dist": mn, "min_x_4n": mn * 4.0 ** n, "law": 118.4,
            "double_double": roots_lo is not None}


def error_vs_fp64(mt, torch, n: int, roots) -> dict:
    """Max distance between the mixed tier's roots and a plain binary64 split
    of the same p_n (every root of either certified).  Both lists are sorted
    by (Re, Im); entries whose order differs between the two (near-equal real
    parts) are re-paired with their nearest neighbour within 16 places."""
    import numpy as np
    ref = mt.split_hyperbolic(n, "fp64")
    a = torch.view_as_complex(roots).cpu().numpy()
    b = ref.roots.cpu().numpy()
    d = np.abs(a - b)
    for i in np.nonzero(d > 1e-10)[0]:
        lo, hi = max(0, i - 16), min(b.size, i + 17)
        d[i] = np.min(np.abs(b[lo:hi] - a[i]))
    return {"max_abs": float(d.max()), "roots": int(a.size),
            "note": "mixed-tier roots against the plain binary64 split of the same polynomial"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The slowest rank's value (the job's time): all-reduce MAX, or x alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Weak scaling: every rank processes its own copy; all units / job time."""
    return world * units_per_rank / seconds


def oracle_units(kind: str, l: int, n: int) -> int:
    """Roots the whole split yields: the degree, or for q_{l,n} its distinct
    roots (Thm fact_mis, from the oracle's closed-form counts)."""
    import oracle
    if kind == "q":
        return sum(oracle.counts.type_histogram_q(l, n).values())
    return oracle.degree(kind, n, l)


def _oracle_sample(args) -> float:
    """One process: the binary64 oracle on the first `frac` of the level
    line; returns its wall time."""
    kind, l, n, frac = args
    import oracle
    t0 = time.perf_counter()
    oracle.split(kind, n, l=l, fp64=True, frac=frac, want_types=False)
    return time.perf_counter() - t0


def oracle_rate(kind: str, l: int, n: int, frac: float, procs: int) -> tuple[float, float]:
    """The oracle, as it stands, in `procs` spawned processes (one per host
    core; spawn, since CUDA is initialised in this process), each splitting
    the same first `frac` of the level line.  Returns (aggregate roots/s,
    wall seconds)."""
    d = oracle_units(kind, l, n)
    if procs <= 1:
        dt = _oracle_sample((kind, l, n, frac))
        return d * frac / dt, dt
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_sample, [(kind, l, n, min(frac, 1.0 / 4096))] * procs)  # import + load the oracle
        t0 = time.perf_counter()
        pool.map(_oracle_sample, [(kind, l, n, frac)] * procs)
        dt = time.perf_counter() - t0
    return procs * d * frac / dt, dt


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def cpu_baseline(kind: str, l: int, n: int, target_s: float = 15.0) -> dict:
    """The binary64 oracle, as it stands, on a bounded sample of the same
    workload -- the first fraction of the level line (walk + descents + set)
    -- in one process per host core.  Rate = roots in that fraction of the
    line x processes / wall time."""
    procs = host_cores()
    frac = 1.0 / 64
    _, dt = oracle_rate(kind, l, n, frac, 1)
    # grow the sample to about target_s seconds (bounded: at most the whole line)
    if dt < target_s:
        frac = min(1.0, frac * target_s / max(dt, 1e-3))
    rate, dt = oracle_rate(kind, l, n, frac, procs)
    return {"value": rate, "unit": "roots/s", "cores": procs, "kind": "oracle",
            "sample": "binary64 oracle (same algorithm, sequential walk), first %.4f of the level line of "
                      "%s n=%d in each of %d processes (one per host core), %.1f s wall; rate = roots x "
                      "fraction x processes / wall time" % (frac, kind, n, procs, dt)}


def run_reference(args, cfg):
    kind, l, n, prec = cfg
    world, rank, _ = dist_env()
    if rank != 0:
        return
    d = oracle_units(kind, l, n)
    frac = 1.0 / 32  # each step: a bounded sample of the same workload
    procs = host_cores()
    for _ in range(args.warmup):
        oracle_rate(kind, l, n, frac, procs)
    times = []
    for _ in range(args.steps):
        times.append(oracle_rate(kind, l, n, frac, procs)[1])
    ms = 1e3 * statistics.mean(times)
    value = procs * d * frac / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s n=%d (%d roots)" % (kind, n, d), "precision": prec,
                   "sample": "first %.4f of the level line per step, %d processes" % (frac, procs)},
        "cpu_baseline": {"value": value, "unit": "roots/s", "cores": procs, "kind": "oracle",
                         "sample": "binary64 oracle, first %.4f of the level line per step in each of %d processes "
                                   "(one per host core)" % (frac, procs)},
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
        d = mt.degree(kind, n, l)  # q_{l,n}: the degree bounds the distinct roots
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
            # from p_30 up the workspace of a retry with doubled (M, c_L) would
            # not fit in HBM next to the roots: one attempt per tier
            extra = {"max_retries": 0} if n >= 30 else {}
            return mt.split_hyperbolic(n, pp, work=work, out=roots, use_graph=1,
                                       out_lo=roots_lo if pp == "dd" else None, **extra)
        if kind == "misbatch":
            _, _, _, st, _ = mt.split_misiurewicz_batch(n, pp, work=work)
            return _BatchResult(st)
        if kind == "q":
            rq = mt.split_misiurewicz_q(l, n, work=work)
            roots[:rq.roots.shape[0]].copy_(torch.view_as_real(rq.roots))
            return rq
        return mt.split_misiurewicz(l, n, pp, work=work, out=roots, out_lo=roots_lo if pp == "dd" else None)

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
    if kind == "q":  # distinct roots, every one certified, multiplicities adding up to the degree
        assert r.stats["n_mult"] == d and r.stats["n_cert_pass"] == r.stats["n_roots"], r.stats
    else:
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
    ms = max_over_ranks(ms, dist)
    certified = min(s["n_cert_pass"] for s in stats)
    value = whole_job_rate(world, certified, ms / 1e3)

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
    e2e_s = max_over_ranks(e2e_s, dist)
    clocks = sampler.stop()

    s0 = stats[-1]
    m = n if kind == "hyp" else (n - 1 if kind == "misbatch" else (l + n if kind == "q" else l + n - 1))
    # q_{l,n} descents evaluate the product form: n orbit steps, then l times
    # two orbit steps (26 flops) and the product update (24 flops), + 24
    desc_flops = 13 * n + 50 * l + 24 if kind == "q" else None
    n_e2e = s0["n_roots"] if kind == "q" else d
    line = {
        "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (inputs fixed by n)",
        "config": {"workload": ("p_%d hyperbolic centres, %d roots, %s, all certified" % (
                       n, d, {"fp64": "plain binary64", "mixed": "mixed binary32/binary64",
                              "dd": ("mixed binary32/binary64" if s0["desc_fp32"] > 0 else "binary64")
                              + " + double-double zones"}[prec])
                       if kind == "hyp" else
                       ("all s_{l,n} with l >= 2, n >= 1, l + n <= %d (%d polynomials, %d roots), one pass, "
                        "binary64, all certified" % (n, len(mt.misiurewicz_pairs(n)), d))
                       if kind == "misbatch" else
                       ("q_{%d,%d} = p_%d - p_%d, %d distinct roots (degree %d with multiplicities, Thm fact_mis), "
                        "binary64, all certified" % (l, n, l + n, l, s0["n_roots"], d))
                       if kind == "q" else
                       "s_{%d,%d} = p_%d + p_%d, %d roots, %s, all certified" % (
                           l, n, l + n - 1, l - 1, d, {"fp64": "plain binary64", "mixed": "mixed binary32/binary64",
                                                       "dd": "binary64 + double-double zones"}[prec])),
                   "precision": prec, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": whole_job_rate(world, n_e2e, e2e_s), "unit": "roots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": n_e2e * 16 * (2 if roots_lo is not None else 1) + 1024,
                "note": "input is the integer n (no device input); result roots copied to pinned host memory"},
        "roofline": roofline(prec, m, stats, args.config, desc_flops),
        "gpu_launches": int(sum(s["n_launches"] for s in stats)),
        "clocks": clocks,
        "detail": {"ms_walk": s0["ms_walk"], "ms_descend": s0["ms_descend"], "ms_dedup": s0["ms_dedup"],
                   "ms_certify": s0["ms_certify"], "ms_seeds": s0["ms_seeds"],
                   "walk_newton": s0["walk_newton"], "seed_newton": s0["seed_newton"],
                   "desc_fp32": s0["desc_fp32"], "n_finish": s0["n_finish"],
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
                      "desc_fp32": sm["desc_fp32"], "n_finish": sm["n_finish"],
                      "ms_walk": sm["ms_walk"], "ms_descend": sm["ms_descend"],
                      "ms_certify": sm["ms_certify"], "ms_dedup": sm["ms_dedup"],
                      "all_certified": all(x["n_cert_pass"] == d for x in st_mix)}}
    if prec == "mixed" and kind == "hyp" and not args.no_compare:
        line["error_vs_fp64"] = error_vs_fp64(mt, torch, n, roots)
    # separation statistics of the result (Sec. 6.3.2), timed on their own
    if kind == "hyp" and not args.no_compare:
        line["separation"] = separation_stats(mt, torch, n, roots, roots_lo, work, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and kind != "misbatch":
        line["cpu_baseline"] = cpu_baseline(kind, l, n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
