"""q_{l,n} = p_{l+n} - p_l with its multiple roots (Thm fact_mis) on the GPU
(mt_split_misiurewicz_q) against the binary128 oracle.

The oracle's q_{l,n} is the union of its own splits of p_n and s_{j,n},
j = 2..l (eq. polySimple telescoped: q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n}),
a root's multiplicity the number of factors it belongs to: it shares no
step with the GPU's descents on q, which take the multiplicity step of
eq. newtonAcc.  Every pair with l + n <= 12, three of order 14 and two of
order 16 (q_{11,5}, with period-5 centres of multiplicity 4 among simple
roots, and q_{6,10}): the same distinct roots (within 1e-12, the binary64
parity tolerance of the other splits), the same types (preperiod, period)
and multiplicities, exactly.  Larger orders: the types follow Thm fact_mis
with eq. MisCount, and the multiplicities add up to the degree.  Every root
carries its certificate (Mis as a root of q, Hyp of p_n)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import counts
from tests.rootsets import lexsorted, match_sets

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


def _hist(pre, per):
    h = {}
    for a, b in zip(pre, per):
        h[(int(a), int(b))] = h.get((int(a), int(b)), 0) + 1
    return h


@pytest.mark.parametrize("l,n", [(l, s - l) for s in range(2, 13) for l in range(1, s)]
                         + [(3, 11), (7, 7), (12, 2), (11, 5), (6, 10)])
def test_q_matches_binary128_oracle(mt, l, n):
    res = mt.split_misiurewicz_q(l, n)
    st = res.stats
    z = res.roots.cpu().numpy()
    ref = oracle.split("q", n, l=l)
    assert ref["n_conflict"] == 0
    assert z.size == ref["n_roots"]
    assert st["n_mult"] == counts.deg_q(l, n) and st["n_cert_pass"] == z.size
    perm, dmax = match_sets(z, ref["roots"])
    assert dmax < TOL_FP64, dmax
    pre, per, mu = res.pre.cpu().numpy(), res.per.cpu().numpy(), res.mult.cpu().numpy()
    assert np.array_equal(pre, ref["type"][perm, 0]) and np.array_equal(per, ref["type"][perm, 1])
    assert np.array_equal(mu, ref["mult"][perm])
    # sorted by (Re, Im)
    assert np.all(np.diff(z.real) >= 0)


@pytest.mark.parametrize("l,n", [(l, 16 - l) for l in range(1, 16)] + [(10, 8), (11, 7), (12, 6), (13, 5), (3, 15)])
def test_q_larger_orders_follow_thm_fact_mis(mt, l, n):
    """every pair of order 16, and order 18 where multiple roots of
    multiplicity 3 and 4 lie next to the tip cluster"""
    res = mt.split_misiurewicz_q(l, n)
    st = res.stats
    pre, per, mu = res.pre.cpu().numpy(), res.per.cpu().numpy(), res.mult.cpu().numpy()
    assert _hist(pre, per) == counts.type_histogram_q(l, n)
    assert int(mu.sum()) == st["n_mult"] == counts.deg_q(l, n)
    assert st["n_cert_pass"] == res.roots.shape[0]


def test_q_rejects_other_tiers(mt):
    from paper_2402_06083_gb300._lib import MtError
    with pytest.raises((MtError, ValueError)):
        mt.split_misiurewicz_q(3, 4, "mixed")


@pytest.mark.parametrize("l,n", [(1, 5), (2, 4), (3, 4), (4, 6), (5, 3), (6, 6), (9, 3)])
def test_q_dd_factors_match_binary128_oracle(mt, l, n):
    """MT_DD: q_{l,n} through its factors (eq. polySimple telescoped), each
    split by its certified double-double split, against the binary128
    oracle: the same distinct roots, types and multiplicities."""
    res = mt.split_misiurewicz_q(l, n, "dd")
    st = res.stats
    z = res.roots.cpu().numpy()
    ref = oracle.split("q", n, l=l)
    assert z.size == ref["n_roots"] and st["prec_used"] == 2
    assert st["n_mult"] == counts.deg_q(l, n) and st["n_cert_pass"] == z.size
    perm, dmax = match_sets(z, ref["roots"])
    assert dmax < TOL_FP64, dmax
    pre, per, mu = res.pre.cpu().numpy(), res.per.cpu().numpy(), res.mult.cpu().numpy()
    assert np.array_equal(pre, ref["type"][perm, 0]) and np.array_equal(per, ref["type"][perm, 1])
    assert np.array_equal(mu, ref["mult"][perm])
    assert lexsorted(z)
    assert st["n_real"] == int(np.sum(z.imag == 0))


@pytest.mark.parametrize("l,n", [(11, 5), (6, 10), (3, 13)])
def test_q_dd_factors_equal_the_binary64_descents(mt, l, n):
    """Two GPU routes to q_{l,n} of order 16: the binary64 descents on q
    itself (misQuick, multiplicity step of eq. newtonAcc) and the union of
    the double-double splits of its factors give the same roots (1e-12),
    types and multiplicities."""
    a = mt.split_misiurewicz_q(l, n)
    b = mt.split_misiurewicz_q(l, n, "dd")
    za, zb = a.roots.cpu().numpy(), b.roots.cpu().numpy()
    assert za.size == zb.size
    perm, dmax = match_sets(za, zb)
    assert dmax < TOL_FP64, dmax
    for f in ("pre", "per", "mult"):
        assert np.array_equal(getattr(a, f).cpu().numpy(), getattr(b, f).cpu().numpy()[perm])


@pytest.mark.parametrize("order", [20, 22])
def test_q_dd_orders_20_and_22_complete(mt, order):
    """Orders where binary64 descents on q lose tip Mis points (about
    6.4e3/8^(l+n) apart, 5.6e-15 at order 20: below the binary64 pixel of
    64 ulp(2)): through the double-double factors every pair (l, n) of the
    order is complete, with Thm fact_mis' type histogram and multiplicities,
    every root certified, sorted by (Re, Im)."""
    work = mt.Workspace()
    for l in range(1, order):
        n = order - l
        res = mt.split_misiurewicz_q(l, n, "dd", work=work)
        st = res.stats
        pre, per, mu = res.pre.cpu().numpy(), res.per.cpu().numpy(), res.mult.cpu().numpy()
        assert _hist(pre, per) == counts.type_histogram_q(l, n), (l, n)
        assert int(mu.sum()) == st["n_mult"] == counts.deg_q(l, n), (l, n)
        assert st["n_cert_pass"] == res.roots.shape[0], (l, n)
        assert lexsorted(res.roots.cpu().numpy()), (l, n)


def test_q_list_entry_points(mt):
    """mt_certify(kind 2) on the split's roots: Hyp roots proven on p_n, Mis
    roots on q, all pass; mt_classify(kind 2): 32 + k for Hyp(k), k for
    Mis(l,k), 0 for Mis(j,k) with j < l -- consistent with pre / per."""
    import torch
    l, n = 4, 6
    res = mt.split_misiurewicz_q(l, n)
    ok, rad, npass = mt.certify("q", n, res.roots, l=l)
    assert npass == res.roots.shape[0] and bool(torch.all(rad > 0))
    t = mt.classify("q", n, res.roots, l=l).cpu().numpy()
    pre, per = res.pre.cpu().numpy(), res.per.cpu().numpy()
    want = np.where(pre == 0, 32 + per, np.where(pre == l, per, 0))
    assert np.array_equal(t, want)


def test_q_rejects_out_of_range(mt):
    from paper_2402_06083_gb300._lib import MtError
    with pytest.raises((MtError, ValueError)):
        mt.split_misiurewicz_q(0, 5)   # l >= 1
    with pytest.raises((MtError, ValueError)):
        mt.split_misiurewicz_q(30, 11)  # l + n <= 40
