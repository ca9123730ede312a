"""The N > 1 logic of bench.py on CPU: two gloo ranks (one GPU per rank on a
GB300 node runs the same code over NCCL).  The path has no data exchange
(replicas: every rank splits its own copy), so what must hold is the
timing rule -- the job time is the slowest rank's -- and the whole-job
rate, plus the reference arm's "rank 0 only" rule."""
from __future__ import annotations

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, times, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        assert (w, r) == (world, rank)
        dist.barrier()
        t = bench.max_over_ranks(times[rank], dist, device="cpu")
        out[rank] = (t, bench.whole_job_rate(world, 1000, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    import torch.multiprocessing as mp
    world = 2
    times = [0.25, 0.75]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == max(times)  # the job takes as long as its slowest rank
        assert rate == world * 1000 / max(times)  # all ranks' units over that time


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(1, 524288, 0.5) == 1048576.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, bench.CONFIGS["hyp12"])
    assert buf.getvalue() == ""  # other ranks exit without work or output
    monkeypatch.setenv("RANK", "0")
    with redirect_stdout(buf):
        bench.run_reference(args, bench.CONFIGS["hyp12"])
    import json
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


@pytest.mark.parametrize("cfg", ["hyp12", "hyp20", "hyp24mixed", "hyp28dd", "mis16"])
def test_configs_are_well_formed(cfg):
    import bench
    kind, l, n, prec = bench.CONFIGS[cfg]
    assert kind in ("hyp", "mis", "misbatch") and prec in ("fp64", "mixed", "dd")
    assert 1 <= n <= 40


def _stats(**kw):
    st = {"ms_walk": 2.0, "ms_seeds": 0.5, "ms_descend": 3.0, "walk_newton": 1000, "seed_newton": 100,
          "desc_newton": 2000, "desc_fp32": 0, "steps_fp32": 0, "finish_newton": 0, "n_starts": 4096,
          "ms_k_walk": 1.5, "ms_k_desc64": 3.0, "ms_k_desc32": 0.0, "ms_k_finish": 0.0, "desc_orbit_steps": 0}
    st.update(kw)
    return st


def test_kernel_rooflines_arithmetic():
    """achieved = counted steps x flops per step / the kernel's own time; frac
    = achieved / the measured rate of the kernel's pipe; the kernel with the
    largest time is the line's roofline."""
    import bench
    pk = {"fp64": 1.2, "fp32": 75.0}
    ks = bench.kernel_rooflines("hyp", 0, 20, [_stats()], pk)
    by = {k["kernel"]: k for k in ks}
    flops = 2000 * (13 * 20 + 24)
    assert abs(by["k_descend"]["achieved"] - flops / 3e-3 / 1e12) < 1e-12
    assert abs(by["k_descend"]["frac"] - by["k_descend"]["achieved"] / 1.2) < 1e-12
    assert by["k_walk"]["flops_per_launch"] == 900 * (13 * 20 + 24) and by["k_walk"]["pipe"] == "fp64"
    assert bench.roofline_of(ks, "x")["kernel"] == "k_descend"
    # the mixed tier: binary32 descents against the binary32 rate, the finish against binary64
    st = _stats(ms_k_desc64=0.0, desc_fp32=1500, steps_fp32=1600, finish_newton=500, ms_k_desc32=1.0,
                ms_k_finish=2.5, n_starts=(1 << 23) + 1)
    by = {k["kernel"]: k for k in bench.kernel_rooflines("hyp", 0, 20, [st], pk)}
    assert set(by) == {"k_descend_mixed", "k_finish_f64", "k_walk_mixed"}
    assert by["k_descend_mixed"]["launches"] == 2 and by["k_descend_mixed"]["peak"] == 75.0
    flops32 = 1500 * (19 * 19 + 25) + ((1 << 23) + 1) * (65 * 20 + 28)  # Newton steps + anchor orbits
    assert abs(by["k_descend_mixed"]["achieved"] - flops32 / 1e-3 / 1e12) < 1e-12
    assert abs(by["k_finish_f64"]["achieved"] - 500 * (7 * 20 + 2) / 2.5e-3 / 1e12) < 1e-12
    assert bench.roofline_of(list(by.values()), "x")["kernel"] == "k_finish_f64"
    # the binary64 descents of the mixed tier (the tip redo): desc_newton less
    # the binary32 steps and the finish steps
    st = _stats(ms_k_desc64=0.5, desc_newton=2100, desc_fp32=1500, steps_fp32=1600, finish_newton=500,
                ms_k_desc32=1.0, ms_k_finish=2.5, n_finish=300)
    by = {k["kernel"]: k for k in bench.kernel_rooflines("hyp", 0, 20, [st], pk)}
    assert by["k_descend"]["flops_per_launch"] == 100 * (13 * 20 + 24)
    # DRAM traffic per launch: the captured bytes per unit x this launch's units
    assert by["k_descend"]["traffic"] is None  # the tip redo (a list), not captured
    assert abs(by["k_descend_mixed"]["traffic"] - 32.1 * 4096) < 1e-6
    assert abs(by["k_finish_f64"]["traffic"] - 118.5 * st["n_finish"]) < 1e-6
    st = _stats(n_starts=1 << 20)
    by = {k["kernel"]: k for k in bench.kernel_rooflines("hyp", 0, 20, [st], pk)}
    assert by["k_descend"]["traffic"] == 16 * (1 << 20)
    # the batched split: orbit lengths differ per polynomial, counted by the kernel
    st = _stats(desc_orbit_steps=30000)
    k = bench.kernel_rooflines("mis", 0, 15, [st], pk)[0]
    assert k["kernel"] == "k_descend_batch" and k["flops_per_launch"] == 13 * 30000 + 24 * 2000


def test_stratified_windows():
    """One window centred in each of the equal parts of the upper half of
    the level line, aligned to whole turns, inside the line, together
    covering the requested fraction."""
    import bench
    n = 20
    J = 8 * 2 ** (n - 1) // 2
    w = bench.windows(n, 0.1, 64)
    assert len(w) == 64
    for i, (what, nn, a, b) in enumerate(w):
        assert what == "window" and nn == n and 0 <= a < b <= J and a % 8 == 0
        assert i * J // 64 <= a and b <= (i + 1) * J // 64  # inside its own part
    cover = sum(b - a for _, _, a, b in w) / J
    assert 0.09 < cover <= 0.1


def test_error_vs_oracle_on_the_host():
    """The bench's error report: the oracle's own roots of p_10 move by less
    than binary64 rounding under its binary128 polish; one root moved by
    1e-9 shows as a 1e-9 error."""
    import numpy as np
    import bench
    import oracle
    z = oracle.split("hyp", 10, want_types=False)["roots"]
    e = bench.error_vs_oracle("hyp", 0, 10, z)
    assert e["checked_fp64"] == z.size and e["max_abs"] < 1e-15 and e["within_tol"]
    z2 = z.copy()
    z2[100] += 1e-9
    e = bench.error_vs_oracle("hyp", 0, 10, z2)
    assert abs(e["max_abs"] - 1e-9) < 1e-12 and not e["within_tol"]
    zl = np.zeros_like(z2)
    zl[5] = 1e-17  # a double-double root: checked with its low part, against the dd tolerance
    e = bench.error_vs_oracle("hyp", 0, 10, z, zl, sample=64)
    assert e["checked_dd"] == 1 and e["checked_fp64"] >= 64 and e["max_abs_dd_roots"] > 5e-18
