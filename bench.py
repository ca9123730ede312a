"""Benchmark: certified roots per second of the level-line Newton splitter.

Default workload (the headline line): all 2^27 = 134,217,728 roots of p_28
in the double-double tier (MT_DD: a mixed binary32/binary64 pass, then
double-double zones where binary64 cannot separate the roots), every root
certified by the disk test.  A step is one full call of
mt_split_hyperbolic(28): seeds, level-line walk, Newton descents, root set,
types, certificates, the double-double pass and the sorted output.

The same line carries one record per other workload ("configs"): p_20 in
plain binary64 (with the mixed tier beside it), p_24 in the mixed tier, and
every s_{l,n} with l + n <= 16 in one pass.  Each record has its own rate,
step time, per-kernel ALU rooflines, the largest distance of its roots from
the binary128 oracle's, and the oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config hyp28dd]
    python bench.py --impl reference ...   # the CPU oracle on the same metric

Other configurations (--config): hyp12, hyp20, hyp20mixed, hyp24,
hyp24mixed, hyp26dd, hyp29dd, hyp31dd, hyp32dd (streamed level line, ~245
GB), mis16, mis26dd (s_{4,22}, beyond FP80), q18 (q_{9,9} with its multiple
roots).  --sub '' drops the per-config records.

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
DEFAULT_CONFIG = "hyp28dd"
DEFAULT_SUB = "hyp20,hyp24mixed,mis16"
M_TURN = 8  # level-line points per turn (the library's and the oracle's default)

# Oracle tolerances of the root values (the binary64 and double-double tiers)
TOL_FP64 = 1e-12
TOL_DD = 1e-20


# ---------------------------------------------------------------------------
# Algorithmic work per Newton step (flops, FMA = 2), counted from the
# kernels' arithmetic for an orbit of length m:
#  - binary64 orbit with the scaled derivative: 6 FMA + 1 mul + 1 add per
#    step, counted 13; the quotient with its range guard, the target or the
#    update and the stop test 24;
#  - binary32 perturbation orbit (mixed tier): 19 flops per step in 12
#    instructions (two FMA pairs for e, one FMA pair and an FMA/mul for g,
#    four adds); the binary32 quotient, update and tests 25;
#  - binary64 finish of the mixed tier (value in binary64, derivatives in
#    binary32): 7 binary64 flops per orbit step (three FMA, the doubling on
#    the integer pipe) and 2 for z - q; the quotient and tests run in binary32.
def newton_flops(m: int) -> int:
    return 13 * m + 24


def newton_flops_fp32(m: int) -> int:
    return 19 * (m - 1) + 25  # the first orbit step (from Z_0 = 0) is exact and skipped


def anchor_flops_fp32(m: int) -> int:
    # the float-float reference orbit the binary32 descent computes per start:
    # per step two TwoProd squares (10 each), a TwoProd product (10), its
    # doubling (2) and three float-float additions (11 each); then P(c0) (two
    # additions) and the jump bound (6)
    return 65 * m + 28


def finish_flops_fp64(m: int) -> int:
    return 7 * m + 2  # the orbit's value and z - q; the quotient and the tests run in binary32


MIX_BATCH = 1 << 23  # starts per launch of the binary32 descent


def nominal_peak(pipe: str, sm_mhz: float | None) -> float | None:
    """Rate from unit counts and the SM clock: 152 SMs x (2 binary64 / 128
    binary32 FMA lanes) x 2 flops x clock."""
    if not sm_mhz:
        return None
    lanes = 2 if pipe == "fp64" else 128
    return 152 * lanes * 2 * sm_mhz * 1e6 / 1e12


def _kernel(name, pipe, flops, ms, launches, peak, peak_nominal, work) -> dict:
    achieved = flops / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    return {"kernel": name, "pipe": pipe, "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
            "frac_of_nominal": achieved / peak_nominal if peak_nominal else None,
            "ms_per_launch": ms / max(1, launches), "launches": launches,
            "flops_per_launch": flops / max(1, launches), "traffic": None, "work": work}


# DRAM traffic per unit of work, from one ncu capture of the current kernels
# (profiles/kernels_hyp24_mixed.md: p_24 mixed and p_20 binary64, dram__bytes
# read + write per launch divided by the units that launch processed), as a
# function of the orbit length m; a bench launch's traffic is this times its
# own units.  k_descend_mixed reads its start and writes (delta, scale) and
# the status, its anchor slots staying in L2: 135 + 134 MB per 2^23 starts at
# p_24, 32.1 B a start.  k_descend (binary64 tier) reads its start (16 B;
# 16.8 MB per 2^20 starts).  k_finish_f64: 389 + 141 MB per 4.47 M finishes
# at p_24, 118.5 B each.  A kernel missing here has changed since its last
# capture (its traffic is reported as null).
TRAFFIC = {
    "k_descend_mixed": (lambda m: 32.1, "start"),
    "k_descend": (lambda m: 16, "start"),
    "k_finish_f64": (lambda m: 118.5, "finish"),
}


def kernel_rooflines(kind: str, l: int, n: int, stats: list, pk: dict, sm_mhz: float | None = None) -> list:
    """ALU roofline of each timed hot kernel against the FMA rate of its own
    pipe: algorithmic flops (the kernels' own step counters x flops per step)
    over the kernel's device time (CUDA events around its launches on the
    launch stream, inside the CUDA graph), mean over the timed steps."""
    s0 = stats[-1]
    m = n if kind == "hyp" else (l + n if kind == "q" else l + n - 1)

    def mean(key):
        return statistics.mean(float(s[key]) for s in stats)

    out = []
    p64, p32 = pk.get("fp64"), pk.get("fp32")
    n64, n32 = nominal_peak("fp64", sm_mhz), nominal_peak("fp32", sm_mhz)
    if s0.get("ms_k_desc64", 0) > 0 and s0.get("desc_orbit_steps", 0) > 0:  # the batched split
        steps, orb = s0["desc_newton"], s0["desc_orbit_steps"]
        out.append(_kernel("k_descend_batch", "fp64", 13 * orb + 24 * steps, mean("ms_k_desc64"), 1, p64, n64,
                           "binary64 Newton steps %d: 13 flops x %d orbit steps + 24 x steps" % (steps, orb)))
    elif s0.get("ms_k_desc64", 0) > 0:
        per = 13 * n + 50 * l + 24 if kind == "q" else newton_flops(m)
        # in the mixed tier desc_newton also counts the binary32 steps and the
        # binary64 finish; the binary64 descent kernel ran the tip redo only
        steps = s0["desc_newton"] - s0.get("desc_fp32", 0) - s0.get("finish_newton", 0)
        out.append(_kernel("k_descend_q" if kind == "q" else "k_descend", "fp64", steps * per, mean("ms_k_desc64"),
                           1, p64, n64, "binary64 Newton steps %d x %d flops" % (steps, per)))
    if s0.get("ms_k_desc32", 0) > 0:
        steps = s0["desc_fp32"]
        launches = -(-s0["n_starts"] // MIX_BATCH)
        nst = s0["n_starts"]
        out.append(_kernel("k_descend_mixed", "fp32", steps * newton_flops_fp32(m) + nst * anchor_flops_fp32(m),
                           mean("ms_k_desc32"), launches, p32, n32,
                           "binary32 Newton steps %d x %d flops + float-float anchor orbits %d x %d flops" %
                           (steps, newton_flops_fp32(m), nst, anchor_flops_fp32(m))))
    if s0.get("ms_k_finish", 0) > 0:
        steps = s0["finish_newton"]
        out.append(_kernel("k_finish_f64", "fp64", steps * finish_flops_fp64(m), mean("ms_k_finish"), 1, p64, n64,
                           "binary64 finish steps %d x %d flops" % (steps, finish_flops_fp64(m))))
    if s0.get("ms_k_walk", 0) > 0:
        steps = s0["walk_newton"] - s0["seed_newton"]
        if s0["steps_fp32"] > 0:  # binary32 walk sub-steps (the binary64 anchors are not counted)
            out.append(_kernel("k_walk_mixed", "fp32", steps * newton_flops_fp32(m), mean("ms_k_walk"), 1, p32,
                               n32, "binary32 walk steps %d x %d flops (anchors not counted)" %
                               (steps, newton_flops_fp32(m))))
        else:
            out.append(_kernel("k_walk", "fp64", steps * newton_flops(m), mean("ms_k_walk"), 1, p64, n64,
                               "binary64 walk steps %d x %d flops" % (steps, newton_flops(m))))
    mixed = s0.get("desc_fp32", 0) > 0
    for k in out:  # DRAM bytes per launch: measured bytes per unit x this launch's units
        t = TRAFFIC.get(k["kernel"])
        if t is None or (k["kernel"] == "k_descend" and mixed) or kind != "hyp":
            continue
        units = s0.get("n_finish", 0) if t[1] == "finish" else s0.get("n_starts", 0)
        k["traffic"] = t[0](m) * units / max(1, k["launches"])
        k["traffic_unit"] = "bytes per launch (%.1f B per %s, from the ncu capture)" % (t[0](m), t[1])
    return out


def roofline_of(kernels: list, peak_source: str) -> dict | None:
    """The roofline entry of the JSON line: the kernel with the largest
    device time."""
    if not kernels:
        return None
    k = max(kernels, key=lambda x: x["ms_per_launch"] * x["launches"])
    r = dict(k)
    r["peak_source"] = peak_source
    return r


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


def separation_stats(mt, torch, n, roots, roots_lo, stream, reps=3) -> dict:
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
    if kind == "misbatch":
        return sum(oracle.counts.deg_s(a, b) for a, b in oracle.counts.misiurewicz_pairs(n))
    return oracle.degree(kind, n, l)


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# The oracle on the host cores: one spawned process per core (spawn, since
# CUDA is initialised in this process), created once and reused, so that
# process start-up stays outside every timed map.
_POOL = None


def host_pool(procs: int):
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        _POOL = mp.get_context("spawn").Pool(procs)
        _POOL.map(_warm, range(procs))  # import the oracle and load its library in every process
    return _POOL


def _warm(_):
    import oracle
    oracle.degree("hyp", 4)
    oracle._lib(True)
    return 0


def _job(task) -> tuple:
    """One unit of oracle work in a pool process; returns (roots, seconds)."""
    import oracle
    what = task[0]
    t0 = time.perf_counter()
    if what == "window":  # a window of the level line of p_n from its lifted seed (binary64 oracle)
        _, n, jbeg, jend = task
        oracle.split_window(n, jbeg, jend, fp64=True)
        units = (jend - jbeg) * 2 // M_TURN  # d / (M d / 2) roots per sub-step of the upper half
    elif what == "mis":  # a whole s_{l,n}
        _, l, n = task
        units = oracle.split("mis", n, l=l, fp64=True, want_types=False)["n_roots"]
    elif what == "q":  # a whole q_{l,n} (union of its factors)
        _, l, n = task
        units = oracle.split_q(l, n, fp64=True)["n_roots"]
    elif what == "hyp":  # a whole p_n
        _, n = task
        units = oracle.split("hyp", n, fp64=True, want_types=False)["n_roots"]
    elif what == "polish":  # binary128 polish of a list: (max displacement, max last step, count)
        _, kind, l, n, z, zl = task
        disp, last = oracle.polish_many(kind, n, z, l=l, roots_lo=zl)
        return (float(disp.max()) if disp.size else 0.0, float(last.max()) if last.size else 0.0, int(disp.size)), \
            time.perf_counter() - t0
    else:
        raise ValueError(what)
    return units, time.perf_counter() - t0


def windows(n: int, frac: float, strata: int) -> list:
    """A stratified sample of the upper half of the level line of p_n: one
    window in each of 'strata' equal parts, centred in it, the windows
    together covering 'frac' of the line (sub-step indices, M = 8)."""
    d = 2 ** (n - 1)
    J = M_TURN * d // 2
    strata = max(1, min(strata, J // 64))
    w = max(64, int(frac * J / strata) // M_TURN * M_TURN)
    w = min(w, J // strata // M_TURN * M_TURN)
    out = []
    for i in range(strata):
        c = (2 * i + 1) * J // (2 * strata)
        a = max(0, min(J - w, (c - w // 2) // M_TURN * M_TURN))
        out.append(("window", n, a, a + w))
    return out


def oracle_tasks(kind: str, l: int, n: int, target_s: float, procs: int) -> tuple[list, str]:
    """The oracle's work for one bounded sample of the workload, sized to
    about target_s seconds on 'procs' host cores; returns (tasks, description)."""
    if kind == "misbatch":
        import oracle
        pairs = oracle.counts.misiurewicz_pairs(n)
        pairs.sort(key=lambda p: -oracle.counts.deg_s(*p))  # largest first: balanced over the pool
        return [("mis", a, b) for a, b in pairs], "every s_{l,n} with l + n <= %d whole (the full workload)" % n
    if kind == "mis":
        return [("mis", l, n)], "s_{%d,%d} whole" % (l, n)
    if kind == "q":
        return [("q", l, n)], "q_{%d,%d} whole (union of its p_n and s_{j,n} splits)" % (l, n)
    # p_n: calibrate one window in this process, then size the stratified sample
    d = 2 ** (n - 1)
    J = M_TURN * d // 2
    if J <= 4096 * procs:
        return [("hyp", n)], "p_%d whole" % n
    probe = windows(n, 16384 / J, 1)[0]
    units, dt = _job(probe)
    rate = units / max(dt, 1e-6)  # roots per second per core
    frac = min(1.0, target_s * procs * rate / d)
    strata = 16 * procs
    tasks = windows(n, frac, strata)
    w = tasks[0][3] - tasks[0][2]
    return tasks, ("stratified: %d windows of %d level-line sub-steps (%.4f of the upper half of p_%d), one "
                   "centred in each of %d equal parts of the line, each walked from its lifted seed with its "
                   "descents and root set" % (len(tasks), w, len(tasks) * w / J, n, len(tasks)))


def run_oracle(tasks: list, procs: int) -> tuple[float, float]:
    """Run the tasks on the host pool (largest first); returns (units, wall seconds)."""
    pool = host_pool(procs)
    t0 = time.perf_counter()
    res = pool.map(_job, tasks, chunksize=1)
    dt = time.perf_counter() - t0
    return float(sum(u for u, _ in res)), dt


def cpu_baseline(kind: str, l: int, n: int, target_s: float = 12.0) -> dict:
    """The binary64 oracle, as it stands, on a bounded sample of the same
    workload, one process per host core.  Rate = roots in the sample / wall
    time of the whole map."""
    procs = host_cores()
    tasks, desc = oracle_tasks(kind, l, n, target_s, procs)
    units, dt = run_oracle(tasks, procs)
    return {"value": units / dt, "unit": "roots/s", "cores": procs, "kind": "oracle",
            "sample": "binary64 oracle (sequential walk, descents, sorted set); %s; %d processes (one per host "
                      "core), %.1f s wall" % (desc, procs, dt)}


def error_vs_oracle(kind: str, l: int, n: int, z, zl=None, sample: int = 1 << 17) -> dict:
    """Largest distance of the GPU's roots from the binary128 oracle's: each
    checked root is Newton-polished in binary128 (3 steps of the oracle's
    own evaluation); the displacement is its distance to the root it
    converges to.  Checked: every double-double root (nonzero low part),
    and every root, or a stratified sample of 'sample' of the rest plus the
    64 left-most (the tip cluster).  Run on the host pool."""
    import numpy as np
    z = np.asarray(z, dtype=np.complex128).ravel()
    zl = None if zl is None else np.asarray(zl, dtype=np.complex128).ravel()
    dd = np.zeros(z.size, bool) if zl is None else (zl != 0)
    rest = np.nonzero(~dd)[0]
    if rest.size > sample:
        pick = np.unique(np.concatenate([rest[np.linspace(0, rest.size - 1, sample).astype(np.int64)], rest[:64]]))
        how = "stratified sample of %d of the %d binary64 roots (every %dth in (Re, Im) order, plus the 64 " \
              "left-most)" % (pick.size, rest.size, rest.size // sample)
    else:
        pick = rest
        how = "every one of the %d binary64 roots" % rest.size
    idd = np.nonzero(dd)[0]
    procs = host_cores()
    pk = "hyp" if kind == "hyp" else "mis"
    tasks = []
    for idx, lo in ((pick, False), (idd, True)):
        for part in np.array_split(idx, max(1, min(4 * procs, idx.size // 256 + 1))):
            if part.size:
                tasks.append((("polish", pk, l, n, z[part], zl[part] if lo else None), lo))
    pool = host_pool(procs)
    t0 = time.perf_counter()
    res = pool.map(_job, [t for t, _ in tasks], chunksize=1)
    dt = time.perf_counter() - t0
    m64 = max([r[0][0] for r, (t, lo) in zip(res, tasks) if not lo], default=0.0)
    mdd = max([r[0][0] for r, (t, lo) in zip(res, tasks) if lo], default=None)
    last = max([r[0][1] for r in res], default=0.0)
    out = {"max_abs": m64 if mdd is None else max(m64, mdd), "max_abs_fp64_roots": m64, "tol_fp64": TOL_FP64,
           "checked_fp64": int(pick.size), "checked_dd": int(idd.size), "roots": int(z.size),
           "within_tol": bool(m64 <= TOL_FP64 and (mdd is None or mdd <= TOL_DD)),
           "polish_last_step_max": last, "host_s": dt,
           "how": "binary128 Newton polish by the oracle (3 steps); " + how +
                  ("; every one of the %d double-double roots (hi + lo)" % idd.size if idd.size else "")}
    if mdd is not None:
        out["max_abs_dd_roots"] = mdd
        out["tol_dd"] = TOL_DD
    return out


def error_vs_oracle_batch(roots, offs, pairs) -> dict:
    """error_vs_oracle over every root of every polynomial of a batch."""
    res = []
    for p, (l, n) in enumerate(pairs):
        z = roots[offs[p]:offs[p + 1]]
        res.append(error_vs_oracle("mis", l, n, z, sample=1 << 30))
    return {"max_abs": max(r["max_abs"] for r in res), "tol_fp64": TOL_FP64,
            "checked_fp64": sum(r["checked_fp64"] for r in res), "roots": sum(r["roots"] for r in res),
            "within_tol": all(r["within_tol"] for r in res),
            "polish_last_step_max": max(r["polish_last_step_max"] for r in res),
            "host_s": sum(r["host_s"] for r in res),
            "how": "binary128 Newton polish by the oracle (3 steps) of every root of every s_{l,n}"}


def run_reference(args, cfg):
    """The reference arm: the oracle, as it stands, on the host cores, on the
    same metric; each step a bounded stratified sample of the workload."""
    kind, l, n, prec = cfg
    world, rank, _ = dist_env()
    if rank != 0:
        return
    procs = host_cores()
    tasks, desc = oracle_tasks(kind, l, n, getattr(args, "ref_step_s", 4.0), procs)
    host_pool(procs)
    for _ in range(args.warmup):
        run_oracle(tasks, procs)
    times, units = [], 0.0
    for _ in range(args.steps):
        u, dt = run_oracle(tasks, procs)
        times.append(dt)
        units = u
    ms = 1e3 * statistics.mean(times)
    value = units / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "roots/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (inputs fixed by n)",
        "config": {"workload": workload_name(kind, l, n, prec, None), "precision": "binary64 oracle",
                   "sample": desc},
        "cpu_baseline": {"value": value, "unit": "roots/s", "cores": procs, "kind": "oracle",
                         "sample": "binary64 oracle per step: %s; %d processes (one per host core)" % (desc, procs)},
        "e2e": {"value": value, "unit": "roots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_name(kind, l, n, prec, s0, npairs=None, d=None) -> str:
    tier = {"fp64": "plain binary64", "mixed": "mixed binary32/binary64",
            "dd": "mixed binary32/binary64 + double-double zones"}[prec]
    if s0 is not None and prec == "dd" and s0.get("desc_fp32", 0) == 0:
        tier = "binary64 + double-double zones"
    if kind == "hyp":
        return "p_%d hyperbolic centres, %d roots, %s, all certified" % (n, 2 ** (n - 1), tier)
    if kind == "misbatch":
        return ("all s_{l,n} with l >= 2, n >= 1, l + n <= %d (%s polynomials, %s roots), one pass, binary64, all "
                "certified" % (n, npairs if npairs else "105", d if d else "all"))
    if kind == "q":
        return ("q_{%d,%d} = p_%d - p_%d, distinct roots with multiplicities (Thm fact_mis), binary64, all certified"
                % (l, n, l + n, l))
    return "s_{%d,%d} = p_%d + p_%d, %d roots, %s, all certified" % (l, n, l + n - 1, l - 1, 2 ** (l + n - 2), tier)


# ---------------------------------------------------------------------------
class Bench:
    """One GPU's measurements: the split of one workload timed with CUDA
    events on the launch stream, L2 flushed between timed steps."""

    def __init__(self, mt, torch, stream, dist=None):
        self.mt, self.torch, self.stream, self.dist = mt, torch, stream, dist
        self.work = mt.Workspace()
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def setup(self, cfg):
        mt, torch = self.mt, self.torch
        kind, l, n, prec = cfg
        if kind == "misbatch":
            self.d = sum(2 ** (a + b - 2) for a, b in mt.misiurewicz_pairs(n))
        else:
            self.d = mt.degree(kind, n, l)  # q_{l,n}: the degree bounds the distinct roots
        self.cfg = cfg
        self.roots = torch.empty((self.d, 2), dtype=torch.float64, device="cuda")
        self.roots_lo = torch.empty((self.d, 2), dtype=torch.float64, device="cuda") if prec == "dd" else None
        self.batch = None

    def step(self, p=None):
        mt = self.mt
        kind, l, n, prec = self.cfg
        pp = prec if p is None else p
        if kind == "hyp":  # the launch sequence is captured once and replayed as a CUDA graph
            # from p_30 up the workspace of a retry with doubled (M, c_L) would
            # not fit in HBM next to the roots: one attempt per tier
            extra = {"max_retries": 0} if n >= 30 else {}
            return mt.split_hyperbolic(n, pp, work=self.work, out=self.roots, use_graph=1,
                                       out_lo=self.roots_lo if pp == "dd" else None, **extra)
        if kind == "misbatch":
            roots, mis, offs, st, pairs = mt.split_misiurewicz_batch(n, pp, work=self.work)
            self.batch = (roots, offs, pairs)
            tot = dict(st[0])  # batch-wide counters and times are reported on every entry
            for key in ("n_roots", "n_cert_pass", "n_starts"):
                tot[key] = sum(x[key] for x in st)
            return type("R", (), {"stats": tot})()
        if kind == "q":
            rq = mt.split_misiurewicz_q(l, n, work=self.work)
            self.roots[:rq.roots.shape[0]].copy_(self.torch.view_as_real(rq.roots))
            return rq
        return mt.split_misiurewicz(l, n, pp, work=self.work, out=self.roots,
                                    out_lo=self.roots_lo if pp == "dd" else None)

    def check(self, r):
        kind = self.cfg[0]
        if kind == "q":  # distinct roots, every one certified, multiplicities adding up to the degree
            assert r.stats["n_mult"] == self.d and r.stats["n_cert_pass"] == r.stats["n_roots"], r.stats
        else:
            assert r.stats["n_roots"] == self.d and r.stats["n_cert_pass"] == self.d, r.stats

    def timed(self, steps, warmup, p=None, barrier=False):
        torch = self.torch
        for _ in range(max(warmup, 3)):
            r = self.step(p)
        self.check(r)
        if barrier and self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        st = []
        if barrier and self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            self.flush.fill_(float(i))  # L2 flush between timed steps (not timed)
            ev[i][0].record(self.stream)
            r = self.step(p)
            ev[i][1].record(self.stream)
            st.append(r.stats)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if barrier and self.dist:
            self.dist.barrier()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        return ms, st, wall

    def e2e(self, steps) -> tuple[float, int]:
        """The public API end to end: each step splits and copies its sorted
        roots (and low parts) to pinned host memory.  Splits of p_n and
        s_{l,n} write into two output buffers in turn, so the copy of step i
        (on a second stream) overlaps the split of step i + 1; the time runs
        until the last copy has landed."""
        torch = self.torch
        kind = self.cfg[0]
        if kind in ("misbatch", "q"):
            return self._e2e_serial(steps)
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream()
        outs = [(self.roots, self.roots_lo),
                (torch.empty_like(self.roots), None if self.roots_lo is None else torch.empty_like(self.roots_lo))]
        hosts = [(torch.empty((self.d, 2), dtype=torch.float64, pin_memory=True),
                  None if self.roots_lo is None else torch.empty((self.d, 2), dtype=torch.float64, pin_memory=True))
                 for _ in range(2)]
        copied = [None, None]  # event: the copy out of buffer k has finished
        keep = (self.roots, self.roots_lo)
        self.step()  # the second buffer's launch sequence is captured outside the timed loop
        self.roots, self.roots_lo = outs[1]
        self.step()
        torch.cuda.synchronize()
        nbytes = self.d * 16 * (1 if self.roots_lo is None else 2)
        cev = []
        t0 = time.perf_counter()
        self.e2e_step_ms = []
        for i in range(steps):
            k = i % 2
            if copied[k] is not None:
                main.wait_event(copied[k])  # buffer k is free again
            self.roots, self.roots_lo = outs[k]
            ts = time.perf_counter()
            self.step()
            self.e2e_step_ms.append((time.perf_counter() - ts) * 1e3)  # the call's host time
            done = torch.cuda.Event()
            done.record(main)
            with torch.cuda.stream(cs):
                cs.wait_event(done)
                c0 = torch.cuda.Event(enable_timing=True)
                c0.record(cs)
                hosts[k][0].copy_(outs[k][0], non_blocking=True)
                if hosts[k][1] is not None:
                    hosts[k][1].copy_(outs[k][1], non_blocking=True)
                copied[k] = torch.cuda.Event(enable_timing=True)
                copied[k].record(cs)
                cev.append((c0, copied[k]))
        cs.synchronize()
        main.synchronize()
        dt = (time.perf_counter() - t0) / steps
        self.e2e_copy_ms = [a.elapsed_time(c) for a, c in cev]
        self.roots, self.roots_lo = keep
        return dt, nbytes + 1024  # + the counters read by the call

    def _e2e_serial(self, steps) -> tuple[float, int]:
        """e2e for the batch and q_{l,n}: split, copy, synchronise, in turn."""
        torch = self.torch
        host = torch.empty((self.d, 2), dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nbytes = 0
        for _ in range(steps):
            self.step()
            if self.cfg[0] == "misbatch":
                roots = self.batch[0]
                hb = host[:roots.shape[0]]
                hb.copy_(torch.view_as_real(roots), non_blocking=True)
                nbytes = roots.shape[0] * 16
            else:
                host.copy_(self.roots, non_blocking=True)
                nbytes = self.d * 16
            torch.cuda.current_stream().synchronize()
        return (time.perf_counter() - t0) / steps, nbytes + 1024

    def roots_host(self):
        """The last split's roots (and low parts) as numpy complex arrays."""
        torch = self.torch
        if self.cfg[0] == "misbatch":
            roots, offs, pairs = self.batch
            return roots.cpu().numpy(), None, offs, pairs
        z = torch.view_as_complex(self.roots).cpu().numpy()
        zl = torch.view_as_complex(self.roots_lo).cpu().numpy() if self.roots_lo is not None else None
        return z, zl, None, None


def measure(b: Bench, name: str, steps: int, warmup: int, pk: dict, peak_source: str, world: int, rank: int,
            with_cpu: bool, with_compare: bool, with_sep: bool) -> dict:
    """One workload's record: rate, step time, e2e, per-kernel rooflines,
    error against the binary128 oracle, and the oracle's own rate."""
    mt, torch = b.mt, b.torch
    cfg = CONFIGS[name]
    kind, l, n, prec = cfg
    b.setup(cfg)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ms, stats, wall = b.timed(steps, warmup, barrier=True)
    ms = max_over_ranks(ms, b.dist)
    certified = min(s["n_cert_pass"] for s in stats)
    clocks = sampler.stop()  # the clocks of the device-timed region
    e2e_s, d2h = b.e2e(steps)
    e2e_s = max_over_ranks(e2e_s, b.dist)
    s0 = stats[-1]
    n_units = s0["n_roots"] if kind in ("q", "misbatch") else b.d
    kern = kernel_rooflines(kind if kind != "misbatch" else "mis", l, n if kind != "misbatch" else n - 1, stats, pk,
                            clocks.get("sm_mhz"))
    rec = {
        "config_name": name, "workload": workload_name(kind, l, n, prec, s0, d=n_units),
        "value": whole_job_rate(world, certified, ms / 1e3), "unit": "roots/s", "ms_per_step": ms,
        "steps": steps, "precision": prec,
        "e2e": {"value": whole_job_rate(world, n_units, e2e_s), "unit": "roots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3,
                "call_ms": [round(x, 1) for x in getattr(b, "e2e_step_ms", [])],
                "copy_ms": [round(x, 1) for x in getattr(b, "e2e_copy_ms", [])],
                "note": "the input is the integer n (no device input); each step's sorted roots (and low parts) "
                        "are copied to pinned host memory inside the timed loop, on a second stream while the "
                        "next step splits into the other of two output buffers; the time ends when the last "
                        "copy has landed"},
        "roofline": roofline_of(kern, peak_source), "kernels": kern,
        "gpu_launches": int(sum(s["n_launches"] for s in stats)), "clocks": clocks,
        "detail": {k: s0.get(k) for k in (
            "ms_walk", "ms_seeds", "ms_descend", "ms_dedup", "ms_certify", "ms_dd", "ms_k_walk", "ms_k_desc64",
            "ms_k_desc32", "ms_k_finish", "walk_newton", "seed_newton", "desc_newton", "desc_fp32",
            "finish_newton", "n_finish", "n_chunks", "n_zones", "n_zone_roots", "steps_dd", "prec_used")},
    }
    rec["detail"]["wall_s"] = wall
    if rank == 0 and world == 1 and kind != "q":
        z, zl, offs, pairs = b.roots_host()
        rec["max_abs_err_vs_oracle"] = error_vs_oracle_batch(z, offs, pairs) if kind == "misbatch" else \
            error_vs_oracle(kind, l, n, z, zl)
    if with_compare and prec == "fp64" and kind == "hyp":  # the same workload in the mixed tier
        ms_mix, st_mix, _ = b.timed(steps, 3, p="mixed")
        sm = st_mix[-1]
        km = kernel_rooflines(kind, l, n, st_mix, pk, clocks.get("sm_mhz"))
        rec["compare"] = {"mixed": {
            "value": min(x["n_cert_pass"] for x in st_mix) / (ms_mix / 1e3), "unit": "roots/s",
            "ms_per_step": ms_mix, "speedup_vs_fp64": ms / ms_mix, "prec_used": sm["prec_used"],
            "kernels": km, "all_certified": all(x["n_cert_pass"] == b.d for x in st_mix),
            "detail": {k: sm.get(k) for k in ("ms_walk", "ms_descend", "ms_dedup", "ms_certify", "desc_newton",
                                              "desc_fp32", "finish_newton", "n_finish", "walk_newton")}}}
        if rank == 0 and world == 1:
            b.step(p="mixed")
            z, _, _, _ = b.roots_host()
            rec["compare"]["mixed"]["max_abs_err_vs_oracle"] = error_vs_oracle(kind, l, n, z)
    if with_sep and kind == "hyp":
        b.step()
        rec["separation"] = separation_stats(mt, torch, n, b.roots, b.roots_lo, b.stream)
    if with_cpu and rank == 0 and world == 1:
        rec["cpu_baseline"] = cpu_baseline(kind, l, n)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(CONFIGS))
    ap.add_argument("--sub", default=None, help="comma-separated configs reported beside the main one "
                                                "(default with the default config: %s)" % DEFAULT_SUB)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the mixed-tier comparison and separation")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        return run_reference(args, cfg)

    import torch
    import paper_2402_06083_gb300 as mt

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # every launch on a created (non-blocking) stream, not the legacy default
    # stream, which would wait for the e2e copy stream's transfers
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # FMA rates of this GPU, measured here (the ALU rooflines' denominators)
    pk = {"fp64": mt.fma_peak("fp64"), "fp32": mt.fma_peak("fp32")}
    peak_source = ("measured in this run by mt_fma_peak (independent FMA chains on every SM, CUDA events): "
                   "binary64 %.3f, binary32 %.1f TFLOP/s" % (pk["fp64"], pk["fp32"]))
    b = Bench(mt, torch, stream, dist)
    with_cpu = not args.no_cpu_baseline
    main_rec = measure(b, args.config, args.steps, args.warmup, pk, peak_source, world, rank, with_cpu,
                       not args.no_compare, not args.no_compare)
    sub = args.sub if args.sub is not None else (DEFAULT_SUB if args.config == DEFAULT_CONFIG else "")
    subs = {}
    for name in [x for x in sub.split(",") if x and x != args.config]:
        subs[name] = measure(b, name, min(args.steps, 10), 3, pk, peak_source, world, rank, with_cpu,
                             not args.no_compare, False)
    kind, l, n, prec = cfg
    line = {
        "metric": METRIC, "value": main_rec["value"], "unit": "roots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (inputs fixed by n)",
        "config": {"workload": main_rec["workload"], "precision": prec,
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": main_rec["e2e"], "roofline": main_rec["roofline"], "kernels": main_rec["kernels"],
        "peaks": {"fp64_tflops": pk["fp64"], "fp32_tflops": pk["fp32"], "source": peak_source},
        "gpu_launches": main_rec["gpu_launches"], "clocks": main_rec["clocks"], "detail": main_rec["detail"],
    }
    for key in ("max_abs_err_vs_oracle", "compare", "separation", "cpu_baseline"):
        if key in main_rec:
            line[key] = main_rec[key]
    if subs:
        line["configs"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if _POOL is not None:
        _POOL.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
