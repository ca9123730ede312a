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
          "desc_newton": 2000, "desc_fp32": 0, "steps_fp32": 0}
    st.update(kw)
    return st


def test_roofline_arithmetic():
    """achieved = counted steps x flops per step / kernel time; frac = / 1.25
    TFLOP/s; the slower of walk and descents is the roofline kernel; binary32
    steps count at the peak ratio; the mixed label only when binary32 ran."""
    import bench
    r = bench.roofline("fp64", 20, [_stats()])
    assert r["kernel"] == "k_descend"
    flops = 2000 * (13 * 20 + 24)
    assert abs(r["achieved"] - flops / 3e-3 / 1e12) < 1e-12 and abs(r["frac"] - r["achieved"] / 1.25) < 1e-12
    r = bench.roofline("fp64", 20, [_stats(ms_descend=1.0)])
    assert r["kernel"] == "k_walk" and abs(r["flops_per_launch"] - 900 * 284) < 1e-6
    mixed = bench.roofline("mixed", 20, [_stats(desc_fp32=1500, steps_fp32=1500)])
    ratio = bench.FP64_PEAK_TFLOPS / bench.FP32_PEAK_TFLOPS
    assert mixed["kernel"] == "k_descend_mixed"
    assert abs(mixed["flops_per_launch"] - (500 * 284 + 1500 * 284 * ratio)) < 1e-6
    assert bench.roofline("dd", 20, [_stats()])["kernel"] == "k_descend"  # no binary32 steps: binary64 label
    q = bench.roofline("fp64", 18, [_stats()], desc_flops=13 * 9 + 50 * 9 + 24)
    assert abs(q["flops_per_launch"] - 2000 * (13 * 9 + 50 * 9 + 24)) < 1e-6


def test_oracle_units_count_distinct_roots_of_q():
    import bench
    from oracle import counts
    assert bench.oracle_units("q", 2, 4) == sum(counts.type_histogram_q(2, 4).values()) == 23  # 8 Hyp + 15 Mis
    assert bench.oracle_units("hyp", 0, 12) == 2048


def test_error_vs_fp64_repairs_local_order_swaps():
    """The mixed-vs-binary64 error report pairs each root with its counterpart
    even where near-equal real parts put the two lists in different orders."""
    import numpy as np
    import torch
    import bench

    rng = np.random.default_rng(7)
    b = np.sort_complex(rng.standard_normal(64) + 1j * rng.standard_normal(64))
    a = b.copy()
    a[[10, 11]] = a[[11, 10]]          # a local order swap
    a[30] += 3e-13                      # a small genuine difference
    ref = type("R", (), {"roots": torch.from_numpy(b)})()
    fake = type("MT", (), {"split_hyperbolic": staticmethod(lambda n, prec: ref)})()
    roots = torch.view_as_real(torch.from_numpy(a)).contiguous()
    e = bench.error_vs_fp64(fake, torch, 6, roots)
    assert e["roots"] == 64
    assert e["max_abs"] == pytest.approx(3e-13, rel=1e-3)
