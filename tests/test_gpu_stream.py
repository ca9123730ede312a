"""Streamed splits (mt_options.stream_pieces): the level line walked and
descended a range of chunks at a time, each piece's root set appended to one
list whose root set is the result.  Automatic from p_32 on (more than 2^31
starts in the upper half); forced here at small sizes, where the same
polynomial split in one pass is the reference: the same roots (within the
1e-12 binary64 parity tolerance), types, counts and certificates."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import counts
from tests.rootsets import match_sets, match_sorted

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


def _same(a, b, tol=TOL_FP64):
    perm, dmax = match_sets(a, b)
    assert dmax < tol, dmax
    return perm


@pytest.mark.parametrize("pieces", [4, 16])
def test_streamed_p20_equals_one_pass(mt, pieces):
    ref = mt.split_hyperbolic(20)
    res = mt.split_hyperbolic(20, stream_pieces=pieces)
    d = 2 ** 19
    assert res.stats["n_roots"] == d and res.stats["n_cert_pass"] == d
    assert {k: res.stats["count_by_type"][k] for k in range(64) if res.stats["count_by_type"][k]} == \
        counts.period_histogram(20)
    _same(res.roots.cpu().numpy(), ref.roots.cpu().numpy())
    r = res.roots.cpu().numpy()
    assert np.all(np.diff(r.real) >= 0)


def test_streamed_mixed_equals_one_pass(mt):
    """The mixed tier in streamed pieces (binary32 walk and descents with
    their binary64 repairs and finishes, piece by piece)."""
    ref = mt.split_hyperbolic(20, "mixed")
    res = mt.split_hyperbolic(20, "mixed", stream_pieces=8)
    d = 2 ** 19
    assert res.stats["n_roots"] == d and res.stats["n_cert_pass"] == d
    assert res.stats["prec_used"] == 1 and res.stats["steps_fp32"] > 0
    _same(res.roots.cpu().numpy(), ref.roots.cpu().numpy())


def test_streamed_misiurewicz_equals_one_pass(mt):
    ref = mt.split_misiurewicz(4, 12)
    res = mt.split_misiurewicz(4, 12, stream_pieces=8)
    assert res.stats["n_cert_pass"] == res.stats["n_roots"] == 2 ** 14
    perm = _same(res.roots.cpu().numpy(), ref.roots.cpu().numpy())
    assert np.array_equal(res.is_mis.cpu().numpy(), ref.is_mis.cpu().numpy()[perm])


def test_streamed_q_equals_one_pass(mt):
    ref = mt.split_misiurewicz_q(6, 10)
    res = mt.split_misiurewicz_q(6, 10, stream_pieces=8)
    assert res.stats["n_mult"] == 2 ** 15 and res.stats["n_cert_pass"] == res.stats["n_roots"]
    perm = _same(res.roots.cpu().numpy(), ref.roots.cpu().numpy())
    for f in ("mult", "pre", "per"):
        assert np.array_equal(getattr(res, f).cpu().numpy(), getattr(ref, f).cpu().numpy()[perm])


def test_streamed_double_double_p26(mt):
    """p_26 in MT_DD with 8 pieces: the dd zones are found from the binary32
    end points of the streamed descents; every root certified, the tip in
    double-double as in one pass."""
    n = 26
    ref = mt.split_hyperbolic(n, "dd", want_lo=True, max_retries=0)
    res = mt.split_hyperbolic(n, "dd", want_lo=True, max_retries=0, stream_pieces=8)
    d = 2 ** (n - 1)
    st = res.stats
    assert st["n_roots"] == d and st["n_cert_pass"] == d and st["prec_used"] == 2 and st["n_zones"] > 0
    z, zl = res.roots.cpu().numpy(), res.roots_lo.cpu().numpy()
    zr, zrl = ref.roots.cpu().numpy(), ref.roots_lo.cpu().numpy()
    dmax, _ = match_sorted(z, zr, 4e-15)  # the whole list, vectorised
    assert dmax < 4e-15
    # the roots redone in dd (low parts set): the same in both, within 1e-28
    a, b = zl != 0, zrl != 0
    assert a.sum() == b.sum() > 0
    perm, _ = match_sets(z[a], zr[b])
    dd = np.abs((z[a] - zr[b][perm]) + (zl[a] - zrl[b][perm]))
    assert dd.max() < 1e-28
