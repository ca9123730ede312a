"""Pins of the oracle's split of q_{l,n} = p_{l+n} - p_l, whose roots are
multiple (Thm fact_mis).  Each pin comes from outside the oracle:

* Thm fact_mis with eq. MisCount and Thm countingHyp: the distinct roots are
  Hyp(k) (k | n), each of multiplicity eta_l(k) = floor((l-1)/k) + 2, and
  Mis(j,k) (2 <= j <= l, k | n), simple; the multiplicities add up to
  deg q_{l,n} = 2^(l+n-1).  Checked type by type for every l + n <= 10.
* the worked factorisation q_{2,4} = h_1^3 h_2^2 h_4^2 m_{2,1} m_{2,2} m_{2,4}
  (Appendix, proof of Thm fact_mis).
* eq. hypCase: q_{1,n} = p_n^2, so its roots are those of p_n, each double.
* a library root finder on the exact integer coefficients of q_{l,n} (built
  here with Python integers from p_{k+1} = p_k^2 + c): its roots, clustered,
  give the same distinct roots and cluster sizes (the multiplicities).

The oracle's q_{l,n} is the union of its own splits of p_n and s_{j,n},
j = 2..l (eq. polySimple telescoped: q_{l,n} = p_n^2 prod_{j=2..l} s_{j,n}),
with a root's multiplicity the number of factors it belongs to.  None of the
pins above is that identity: Thm fact_mis's eta_l(k) and the worked
factorisation come from the paper's counting, the library roots from the
integer coefficients of p_{l+n} - p_l itself.  A plausible slip in the union
fails one of them: the product taken from s_{1,n} (p_n three times), p_n
counted once, or a factor missed (the multiplicities fall short of the
degree)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import goldens
from oracle import counts


def _hist(r):
    h = {}
    for (a, b) in map(tuple, r["type"]):
        h[(int(a), int(b))] = h.get((int(a), int(b)), 0) + 1
    return h


@pytest.mark.parametrize("l,n", [(l, s - l) for s in range(2, 11) for l in range(1, s)])
def test_types_and_multiplicities_follow_thm_fact_mis(l, n):
    r = oracle.split("q", n, l=l)
    assert r["n_conflict"] == 0  # the factors agree on the type of every shared root
    assert _hist(r) == counts.type_histogram_q(l, n)
    assert int(r["mult"].sum()) == counts.deg_q(l, n) == r["stats"]["n_mult"]
    hyp = r["type"][:, 0] == 0
    assert np.all(r["mult"][hyp] == (l - 1) // r["type"][hyp, 1] + 2)
    assert np.all(r["mult"][~hyp] == 1)


def test_worked_factorisation_q_2_4():
    """q_{2,4} = h_1^3 h_2^2 h_4^2 m_{2,1} m_{2,2} m_{2,4} (App. A;
    tests/golden/q_2_4_factorisation.txt): c = 0 triple, c = -1 double, the 6
    centres of period 4 double, the Misiurewicz points simple."""
    r = oracle.split("q", 4, l=2)
    mult = {}
    for (a, b), m in zip(map(tuple, r["type"]), r["mult"]):
        mult.setdefault((int(a), int(b)), set()).add(int(m))
    want = {(j, k): {e} for j, k, e in goldens.rows("q_2_4_factorisation.txt")}
    assert mult == want
    z = r["roots"]
    assert np.min(np.abs(z)) < 1e-30 and np.min(np.abs(z + 1)) < 1e-30


@pytest.mark.parametrize("n", [3, 5, 6])
def test_q_1_n_is_p_n_squared(n):
    rq = oracle.split("q", n, l=1)
    rp = oracle.split("hyp", n)
    assert np.all(rq["mult"] == 2) and rq["n_roots"] == rp["n_roots"]
    assert np.max(np.abs(np.sort_complex(rq["roots"]) - np.sort_complex(rp["roots"]))) < 1e-25


def _q_coeffs(l, n):
    """Integer coefficients of q_{l,n}(c), highest degree first."""
    p = [[0]]  # p_0 = 0, as coefficient lists lowest degree first
    for _ in range(l + n):
        a = p[-1]
        sq = [0] * (2 * len(a) - 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(a):
                    sq[i + j] += x * y
        sq += [0]
        sq[1] += 1  # + c
        while len(sq) > 1 and sq[-1] == 0:
            sq.pop()
        p.append(sq)
    hi, lo = p[l + n], p[l] + [0] * (len(p[l + n]) - len(p[l]))
    q = [x - y for x, y in zip(hi, lo)]
    while q and q[-1] == 0:
        q.pop()
    return [float(x) for x in reversed(q)]


@pytest.mark.parametrize("l,n", [(2, 2), (3, 2), (2, 3), (4, 1), (1, 4)])
def test_library_roots_of_exact_coefficients(l, n):
    """numpy.roots on the exact coefficients: a root of multiplicity mu comes
    out as mu close copies (spread ~ roundoff^(1/mu)); clustering them gives
    the distinct roots and their multiplicities."""
    lib = np.roots(_q_coeffs(l, n))
    r = oracle.split("q", n, l=l)
    z, mu = r["roots"], r["mult"]
    # each library root is nearest to one oracle root; count them per root
    owner = np.array([np.argmin(np.abs(z - w)) for w in lib])
    assert np.array_equal(np.bincount(owner, minlength=z.size), mu)
    for w, k in zip(lib, owner):
        assert abs(w - z[k]) < 10 * 1e-12 ** (1.0 / mu[k])  # a root of multiplicity mu moves ~ eps^(1/mu)


@pytest.mark.parametrize("l,n", [(1, 2), (2, 2), (2, 3), (3, 2)])
def test_level_line_iso_angle_zero_q(l, n):
    """The level line |q_{l,n}| = 100 (Sec. 4.2): its iso-angle-0 starts and their
    conjugates are q^{-1}(100), simple points away from the multiple roots;
    brute force on the exact integer polynomial q_{l,n} - 100."""
    import mpmath
    from tests.rootsets import match_sets
    mpmath.mp.dps = 40
    st = oracle.level_line("q", n, l=l)["starts"]
    d = 2 ** (l + n - 1)
    assert st.size == 2 * d + 1
    iso0 = st[::4]
    full = np.concatenate([iso0, np.conj(iso0[(np.abs(iso0.imag) > 1e-12)])])
    co = [int(x) for x in _q_coeffs(l, n)]  # highest degree first
    co[-1] -= 100
    ref = np.array([complex(x) for x in mpmath.polyroots(co, maxsteps=400, extraprec=8 * len(co))])
    assert full.size == ref.size == d
    _, dmax = match_sets(full, ref)
    assert dmax < 1e-12


@pytest.mark.parametrize("l,n", [(11, 5), (6, 9)])
def test_order_16_follows_thm_fact_mis(l, n):
    """Order 16, where a descent on q itself meets roots of multiplicity 4
    next to other roots (q_{11,5}: period-5 centres of multiplicity 4): the
    union of the factors' roots is exact, type by type (Thm fact_mis)."""
    r = oracle.split("q", n, l=l)
    assert r["n_conflict"] == 0
    assert _hist(r) == counts.type_histogram_q(l, n)
    assert int(r["mult"].sum()) == counts.deg_q(l, n)
    hyp = r["type"][:, 0] == 0
    assert np.all(r["mult"][hyp] == (l - 1) // r["type"][hyp, 1] + 2)


def test_q_roots_are_roots_of_q():
    """Every distinct root of the union is a root of q_{l,n} = p_{l+n} - p_l
    as the paper writes it: binary128 Newton on the difference form, with the
    multiplicity step z - mu q / q' of eq. newtonAcc (quadratic at a root of
    multiplicity mu), moves no root by more than 1e-20."""
    l, n = 4, 4
    r = oracle.split("q", n, l=l)
    for z, mu in zip(r["roots4"], r["mult"]):
        w = np.array(z, dtype=np.float64)
        v, dv = oracle.evaluate("q", n, w, l=l)
        P = complex(v[0] + v[1], v[2] + v[3])
        D = complex(dv[0] + dv[1], dv[2] + dv[3])
        if mu == 1:
            assert abs(P) <= 1e-20 * abs(D)
        else:  # q' vanishes too: the value is tiny next to the scale of q
            assert abs(P) < 1e-20
