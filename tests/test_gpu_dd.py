"""Parity of the double-double tier (MT_DD) with the binary128 oracle.

dd_all mode redoes every root in double-double: each root hi + lo must lie
within 1e-28 of the oracle's binary128 root.  The dd Newton stops at
|step| < tol_dd <= 1e-26; the error left after that step is of order
step^2 / separation, and the double-double rounding floor is ~1e-31, so
1e-28 leaves room for both.  Counts, types and certificate flags are exact.

The default MT_DD mode keeps binary64 roots wherever the binary64 pass is
certified and redoes in double-double only the zones around roots it could
not separate: p_26 and p_28, whose left-most roots lie 118.4 / 4^n apart
(Sec. 6.3.2), a few ulps of 2.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import counts
from tests import goldens
from tests.rootsets import lexsorted, match_sets

SEP = goldens.table("separation_law.txt")  # Sec. 6.3.2

pytestmark = pytest.mark.gpu

TOL_DD = 1e-28


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


def _hist(st):
    return {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]}


def _dd_dist(g, gl, r4):
    """|(g + gl) - (r4 hi + r4 lo)| per pair, differences taken part by part
    so the double-double digits survive."""
    dre = (g.real - r4[:, 0]) + (gl.real - r4[:, 1])
    dim = (g.imag - r4[:, 2]) + (gl.imag - r4[:, 3])
    return np.hypot(dre, dim)


def _split(mt, kind, n, l=0, **kw):
    if kind == "hyp":
        return mt.split_hyperbolic(n, "dd", want_lo=True, **kw)
    return mt.split_misiurewicz(l, n, "dd", want_lo=True, **kw)


@pytest.mark.parametrize("kind,n,l", [("hyp", 1, 0), ("hyp", 2, 0), ("hyp", 8, 0), ("hyp", 10, 0),
                                      ("hyp", 12, 0), ("mis", 1, 2), ("mis", 5, 3), ("mis", 4, 4),
                                      ("mis", 6, 3)])
def test_dd_all_matches_binary128_oracle(mt, kind, n, l):
    res = _split(mt, kind, n, l, dd_all=1)
    st = res.stats
    z = res.roots.cpu().numpy()
    zl = res.roots_lo.cpu().numpy()
    ref = oracle.split(kind, n, l=l)
    d = oracle.degree(kind, n, l)
    assert z.size == ref["n_roots"] == d
    assert st["prec_used"] == 2 and st["n_cert_pass"] == d
    assert st["n_zone_roots"] == int(np.sum(z.imag >= 0))  # every root (upper half) came from dd
    assert lexsorted(z, zl)
    perm, dmax_hi = match_sets(z, ref["roots"])
    assert dmax_hi < 1e-15
    err = _dd_dist(z, zl, ref["roots4"][perm])
    assert err.max() < TOL_DD, float(err.max())
    if kind == "hyp":
        assert _hist(st) == counts.period_histogram(n)
    else:
        for (a, k), cnt in counts.type_histogram_s(l, n).items():
            assert st["count_by_type"][k if a == l else 32 + k] == cnt
        mis = res.is_mis.cpu().numpy().astype(bool)
        to = ref["type"][perm]
        assert np.array_equal(mis, (to[:, 0] == l) & (to[:, 1] == n))
    # real roots exactly real in both parts, conjugates exact in both parts
    real = z.imag == 0
    assert np.all(zl.imag[real] == 0)
    key = np.lexsort((z.imag, z.real))
    zs, zls = z[key], zl[key]
    cj = np.lexsort((-z.imag, z.real))
    assert np.array_equal(zs.real, z[cj].real) and np.array_equal(zs.imag, -z[cj].imag)
    assert np.array_equal(zls.real, zl[cj].real) and np.array_equal(zls.imag, -zl[cj].imag)


def test_dd_keeps_binary64_where_it_is_certified(mt):
    """p_12: the binary64 pass is certified complete, so MT_DD returns it
    unchanged (no dd pass, zero low parts)."""
    res = _split(mt, "hyp", 12)
    st = res.stats
    assert st["prec_used"] == 1 and st["n_zone_roots"] == 0 and st["steps_dd"] == 0
    assert not np.any(res.roots_lo.cpu().numpy())
    ref = mt.split_hyperbolic(12, "mixed").roots.cpu().numpy()
    assert np.array_equal(res.roots.cpu().numpy(), ref)


def test_dd_certify_list_rejects_shifted_points(mt):
    """mt_certify with low parts: dd roots pass at the 1e-20 default radius;
    the same points moved by 1e-18 (far outside any 1e-20 disk) all fail."""
    import torch
    res = _split(mt, "hyp", 10, dd_all=1)
    ok, rad, npass = mt.certify("hyp", 10, res.roots, roots_lo=res.roots_lo)
    assert npass == res.roots.shape[0]
    assert float(rad.max()) <= 1e-20
    lo = torch.view_as_real(res.roots_lo.clone())
    lo[:, 0] += 1e-18
    ok2, _, npass2 = mt.certify("hyp", 10, res.roots, roots_lo=torch.view_as_complex(lo))
    assert npass2 == 0


def _tip_checks(mt, n, res, k=24):
    """The k left-most roots (the real cluster at -2): binary128 Newton from
    the dd value moves it by less than TOL_DD."""
    z = res.roots[:k].cpu().numpy()
    zl = res.roots_lo[:k].cpu().numpy()
    # increasing in double-double (from p_29 on the tip gap is below one ulp of 2)
    gaps = (z.real[1:] - z.real[:-1]) + (zl.real[1:] - zl.real[:-1])
    assert np.all(z.imag == 0) and np.all(gaps > 0)
    for i in range(k):
        c4 = np.array([z[i].real, zl[i].real, 0.0, 0.0])
        out, _ = oracle.polish("hyp", n, c4, steps=3)
        move = abs((out[0] - c4[0]) + (out[1] - c4[1]))
        assert move < TOL_DD, (i, move)
    # the two left-most roots are 118.4 / 4^n apart to 0.1 % (Sec. 6.3.2)
    gap = (z[1].real - z[0].real) + (zl[1].real - zl[0].real)
    assert abs(gap * 4.0 ** n / SEP["hyp_constant"] - 1) < 2 * SEP["hyp_rel_error"]


@pytest.mark.parametrize("n", [26, 28, 29, 30, 31])
def test_dd_complete_and_certified(mt, n):
    """p_26 (33.5M roots) up to p_31 (1.07G): binary64 cannot separate the
    tip cluster (from p_29 on its two left-most roots lie under one ulp of 2
    apart); MT_DD returns every root, each one certified, with the exact
    Moebius histogram and Vieta's first sum.  The first attempt (binary32
    descents with their binary64 finish, binary64 redo of the descents that
    end at the left tip, dd zones) is complete: no retry ran (max_retries=0
    would report MT_EINCOMPLETE otherwise)."""
    import torch
    res = _split(mt, "hyp", n, max_retries=0)
    st = res.stats
    d = 2 ** (n - 1)
    assert st["n_roots"] == d and res.roots.shape[0] == d
    assert st["n_cert_pass"] == d
    assert st["prec_used"] == 2 and st["n_zones"] > 0 and st["n_zone_roots"] > 0
    assert st["retries"] == 0 and st["desc_fp32"] > 0, (st["retries"], st["desc_fp32"])
    assert st["first_n_roots"] == d
    if n >= 29:  # the tip redo ran (about 0.8 % of the descents at p_30)
        assert 0 < st["n_tip64"] < st["n_starts"] // 50, st["n_tip64"]
    assert _hist(st) == counts.period_histogram(n)
    r = torch.view_as_real(res.roots)
    assert bool(torch.all(r[1:, 0] >= r[:-1, 0]))  # sorted by Re (hi parts)
    s1 = torch.sum(r[:, 0]).item()
    assert abs(s1 + 2 ** (n - 2)) < 1e-3
    assert abs(torch.sum(r[:, 1]).item()) < 1e-6
    _tip_checks(mt, n, res)
    ok, rad, npass = mt.certify("hyp", n, res.roots, roots_lo=res.roots_lo, tol=1e-12)
    assert npass == d


def test_dd_zone_radius_changes_work_not_roots(mt):
    """A larger zone radius (1e-8 against the default 1e-11 of p_26) redoes more roots
    in dd but returns the same certified set (every root within 4e-15, roots
    redone in dd by both runs within TOL_DD)."""
    n = 26
    a = _split(mt, "hyp", n, max_retries=0)
    b = _split(mt, "hyp", n, max_retries=0, dd_radius=1e-8)
    assert b.stats["n_zone_roots"] > a.stats["n_zone_roots"]
    assert a.stats["n_cert_pass"] == b.stats["n_cert_pass"] == 2 ** (n - 1)
    za, zb = a.roots[:4096].cpu().numpy(), b.roots[:4096].cpu().numpy()
    la, lb = a.roots_lo[:4096].cpu().numpy(), b.roots_lo[:4096].cpu().numpy()
    assert np.max(np.abs(za - zb)) < 4e-15  # binary64 roots in one run, dd in the other
    both = (la != 0) & (lb != 0)
    dd = np.abs((za - zb) + (la - lb))[both]
    assert dd.size > 0 and dd.max() < TOL_DD


@pytest.mark.parametrize("l,n", [(3, 23), (4, 22)])
def test_dd_misiurewicz_order_26(mt, l, n):
    """s_{3,23} and s_{4,22} (16.8M roots each): the first Misiurewicz order
    that FP80 cannot resolve (Sec. 6.3.2: two real points of Mis(3,23) and
    of Mis(4,22) at the left end of M lie less than 4.86e-20 < 2^-64 apart).
    MT_DD returns every root certified with the exact type histogram, and the
    closest left-tip pair lies below 2^-64 -- for Mis(4,22) at the paper's
    4.86e-20 -- as binary128 Newton of the oracle confirms."""
    res = mt.split_misiurewicz(l, n, "dd", want_lo=True, max_retries=0)
    st = res.stats
    d = 2 ** (l + n - 2)
    assert st["n_roots"] == d and st["n_cert_pass"] == d and st["prec_used"] == 2
    for (a, k), cnt in counts.type_histogram_s(l, n).items():
        assert st["count_by_type"][k if a == l else 32 + k] == cnt
    z, zl = res.roots[:64].cpu().numpy(), res.roots_lo[:64].cpu().numpy()
    o = np.lexsort((zl.real, z.real))
    z, zl = z[o], zl[o]
    assert np.all(z.imag[:16] == 0)
    gaps = (z.real[1:16] - z.real[:15]) + (zl.real[1:16] - zl.real[:15])
    i = int(np.argmin(gaps))
    assert 0 < gaps[i] < 2.0 ** -64
    # the pair in binary128: the oracle's Newton moves neither point by 1e-28
    pts = []
    for j in (i, i + 1):
        c4 = np.array([z[j].real, zl[j].real, 0.0, 0.0])
        out, _ = oracle.polish("mis", n, c4, l=l, steps=3)
        assert abs((out[0] - c4[0]) + (out[1] - c4[1])) < TOL_DD
        pts.append(out)
    gap128 = (pts[1][0] - pts[0][0]) + (pts[1][1] - pts[0][1])
    assert abs(gap128 - gaps[i]) < 1e-27
    if (l, n) == (4, 22):
        assert 4.8e-20 < gaps[i] < SEP["mis_tip_gap"]
