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
from tests.rootsets import match_sets

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
