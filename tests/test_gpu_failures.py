"""Failure paths of the split, forced through options and inputs only (no
device fault, no hang): the count check with the (M, c_L) doubling of Sec.
4.1 ("if some roots are missing, N can be increased"), the chunk-end check
that detects a walk skipping a turn (the "skip modulo 2 pi" failure of Sec.
6.4.1), and the outcome of descents that leave the finite numbers or the
disk around the roots ("long-distance jump", Sec. 6.4.1)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


def test_coarse_line_misses_roots_without_retries(mt):
    """M = 2 points per turn and c_L = 1 start per root: the line is too
    coarse (one start per turn, and about three in four descents repeat a
    root), so with no retry allowed the split reports MT_EINCOMPLETE."""
    from paper_2402_06083_gb300._lib import MT_EINCOMPLETE
    n = 12
    res = mt.split_hyperbolic(n, "fp64", M=2, c_L=1, max_retries=0, check_status=False)
    st = res.stats
    assert res.status == MT_EINCOMPLETE, (res.status, st["n_roots"])
    assert st["n_roots"] < 2 ** (n - 1) and st["retries"] == 0
    assert st["M"] == 2 and st["c_L"] == 1


def test_retries_double_the_line_until_complete(mt):
    """The same coarse start with retries: (M, c_L) doubles, (2, 1) -> (4, 2)
    -> (8, 4), and the split completes, every root certified, with the
    exact Moebius histogram."""
    n = 12
    res = mt.split_hyperbolic(n, "fp64", M=2, c_L=1, max_retries=3)
    st = res.stats
    d = 2 ** (n - 1)
    assert res.status == 0 and st["n_roots"] == d and st["n_cert_pass"] == d
    assert st["retries"] >= 1 and st["M"] == 2 << st["retries"] and st["c_L"] == 1 << st["retries"]
    assert {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]} == counts.period_histogram(n)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_skipped_turns_are_detected(mt, prec):
    """Two sub-steps per turn (half a turn each) make walk chunks skip turns;
    the chunk-end check counts them (walk_fail), which alone makes the split
    retry.  With no retry the failures are reported in the statistics."""
    n = 14
    res = mt.split_hyperbolic(n, prec, M=2, c_L=2, max_retries=0, check_status=False)
    st = res.stats
    assert st["walk_fail"] > 0 or st["n_roots"] < 2 ** (n - 1)
    res2 = mt.split_hyperbolic(n, prec, M=2, c_L=2, max_retries=3)
    assert res2.status == 0 and res2.stats["n_roots"] == 2 ** (n - 1) and res2.stats["retries"] >= 1


def test_descent_outcomes(mt):
    """mt_descend's outcome byte: c = 3 on p_20 (the orbit overflows binary64
    within ten steps), a start at the critical point -1/2 of p_2 (P' = 0)
    and a start at 1e200 all stop as divergent (1); a start on a root
    converges (0)."""
    import torch
    out, status, st = mt.descend("hyp", 20, torch.tensor([3.0 + 0j, 0.0 + 0j], dtype=torch.complex128,
                                                         device="cuda"))
    s = status.cpu().numpy()
    assert s[0] == 1 and s[1] == 0
    out, status, _ = mt.descend("hyp", 2, torch.tensor([-0.5 + 0j, 1e200 + 0j, -1.0 + 0j], dtype=torch.complex128,
                                                        device="cuda"))
    s = status.cpu().numpy()
    assert list(s) == [1, 1, 0]
    assert np.isclose(out.cpu().numpy()[2], -1.0)


def test_split_of_an_invalid_polynomial_is_rejected(mt):
    """Out of the domain: no device work, MT_EINVAL with a message."""
    from paper_2402_06083_gb300._lib import MtError
    for bad in (0, 41):
        with pytest.raises((ValueError, MtError)):
            mt.split_hyperbolic(bad)
    with pytest.raises((ValueError, MtError)):
        mt.split_misiurewicz(1, 5)  # l >= 2
