"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/, binary128) against something other than
itself: closed forms, a textbook formula, an independent root finder on exact
integer coefficients, exact Sturm counts, or the counts of Thm countingHyp and
eq. MisCount.  A plausible mistake in the oracle (a dropped term, a wrong
sign, a wrong index) fails at least one of them (see test_oracle_mutants.py).
"""
from __future__ import annotations

from fractions import Fraction

import mpmath
import numpy as np
import pytest

import oracle
from oracle import counts
from tests import goldens
from tests.polyexact import p_coeffs, s_coeffs
from tests.rootsets import lexsorted, match_sets, min_separation

SEPARATION = goldens.table("separation_law.txt")  # Sec. 6.3.2


def _exact(v4) -> Fraction:
    return Fraction(float(v4[0])) + Fraction(float(v4[1]))


# --- the recurrence and its derivative -----------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 10, 20, 26, 33, 40])
def test_orbit_at_minus_two(n):
    """f_{-2}^k(-2) = 2 and p_n'(-2) = -(4^n + 2)/6 (Sec. 6.3.2, after eq. DerParamDyna)."""
    v, dv = oracle.evaluate("hyp", n, -2.0)
    assert _exact(v[0:2]) == 2 and _exact(v[2:4]) == 0
    assert _exact(dv[0:2]) == Fraction(-(4 ** n + 2), 6)
    assert _exact(dv[2:4]) == 0


def test_orbit_off_axis_against_integer_polynomial():
    """P and P' at a complex point agree with the exact integer coefficients."""
    mpmath.mp.dps = 60
    c = mpmath.mpc("0.2731", "-0.4417")
    for n in (1, 2, 4, 7):
        co = p_coeffs(n)
        want = mpmath.polyval(list(reversed(co)), c)
        dco = [k * co[k] for k in range(1, len(co))]
        dwant = mpmath.polyval(list(reversed(dco)), c) if dco else mpmath.mpf(0)
        v, dv = oracle.evaluate("hyp", n, complex(c))
        assert abs(complex(v[0] + v[1], v[2] + v[3]) - complex(want)) < 1e-14 * max(1, abs(want))
        assert abs(complex(dv[0] + dv[1], dv[2] + dv[3]) - complex(dwant)) < 1e-14 * max(1, abs(dwant))
    for (l, n) in ((2, 1), (3, 2), (4, 3)):
        co = s_coeffs(l, n)
        want = mpmath.polyval(list(reversed(co)), c)
        dco = [k * co[k] for k in range(1, len(co))]
        dwant = mpmath.polyval(list(reversed(dco)), c)
        v, dv = oracle.evaluate("mis", n, complex(c), l=l)
        assert abs(complex(v[0] + v[1], v[2] + v[3]) - complex(want)) < 1e-14 * max(1, abs(want))
        assert abs(complex(dv[0] + dv[1], dv[2] + dv[3]) - complex(dwant)) < 1e-14 * max(1, abs(dwant))


# --- small root sets --------------------------------------------------------

def test_hyp_1_and_2():
    """Hyp(1) = {0}, Hyp(2) = {-1} (Sec. 2.1; tests/golden/hyp_small.txt)."""
    want = {k: complex(re, im) for k, re, im in goldens.rows("hyp_small.txt")}
    r1 = oracle.split("hyp", 1)
    assert r1["n_roots"] == 1 and abs(r1["roots"][0] - want[1]) < 1e-30
    r2 = oracle.split("hyp", 2)
    assert r2["n_roots"] == 2
    got = {int(b): z for (a, b), z in zip(r2["type"].tolist(), r2["roots"])}
    assert sorted(got) == [1, 2]
    assert all(abs(got[k] - want[k]) < 1e-30 for k in (1, 2))


def test_period3_cardano():
    """p_3 = z^4 + 2z^3 + z^2 + z = z (z^3 + 2z^2 + z + 1) (Sec. 3.1;
    tests/golden/p3_coefficients.txt); the cubic's roots by Cardano's formula."""
    (co,) = goldens.rows("p3_coefficients.txt")
    assert co[-1] == 0 and co[0] == 1  # p_3 = z * (monic cubic)
    assert list(reversed(p_coeffs(3))) == co  # the test's own recurrence agrees
    mpmath.mp.dps = 50
    # depressed cubic of z^3 + a z^2 + b z + c via z = t - a/3
    a, b, c = (mpmath.mpf(x) for x in co[1:4])
    p = b - a * a / 3
    q = 2 * a ** 3 / 27 - a * b / 3 + c
    disc = (q / 2) ** 2 + (p / 3) ** 3
    assert disc > 0  # one real root and a conjugate pair

    def rcbrt(x):  # real cube root
        return mpmath.sign(x) * abs(x) ** (mpmath.mpf(1) / 3)
    u = rcbrt(-q / 2 + mpmath.sqrt(disc))
    v = rcbrt(-q / 2 - mpmath.sqrt(disc))
    w = mpmath.exp(2j * mpmath.pi / 3)
    cubic = [u + v - a / 3, u * w + v * w ** 2 - a / 3, u * w ** 2 + v * w - a / 3]
    r = oracle.split("hyp", 3)
    z4 = r["roots4"]
    got = [mpmath.mpc(mpmath.mpf(x[0]) + x[1], mpmath.mpf(x[2]) + x[3]) for x in z4]
    assert r["n_roots"] == 4
    for want in cubic + [mpmath.mpc(0)]:
        assert min(abs(g - want) for g in got) < 1e-28
    # the values the paper quotes
    assert abs(float(cubic[0].real) + 1.7548776662466927) < 1e-15


@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_small_n_against_polyroots(n):
    """n <= 7: roots of the exact integer polynomial by an independent method
    (mpmath's simultaneous iteration), Sec. 3.2 / 3.3."""
    mpmath.mp.dps = 40
    co = p_coeffs(n)
    ref = mpmath.polyroots(list(reversed(co)), maxsteps=400, extraprec=8 * len(co))
    ref = np.array([complex(x) for x in ref])
    r = oracle.split("hyp", n)
    assert r["n_roots"] == 2 ** (n - 1)
    _, dmax = match_sets(r["roots"], ref)
    assert dmax < 1e-13


@pytest.mark.parametrize("l,n", [(2, 1), (2, 2), (3, 1), (2, 3), (3, 2), (4, 1), (2, 4), (3, 3), (4, 2)])
def test_small_s_against_polyroots(l, n):
    mpmath.mp.dps = 40
    co = s_coeffs(l, n)
    ref = mpmath.polyroots(list(reversed(co)), maxsteps=400, extraprec=8 * len(co))
    ref = np.array([complex(x) for x in ref])
    r = oracle.split("mis", n, l=l)
    assert r["n_roots"] == counts.deg_s(l, n) == len(ref)
    _, dmax = match_sets(r["roots"], ref)
    assert dmax < 1e-13


def test_tiny_misiurewicz():
    """Mis(2,1) = {-2}; Mis(2,2) = {+-i} with s_{2,2} = z (z+2)(z^2+1);
    Mis(3,1) = roots of z^3 + 2 z^2 + 2 z + 2 (eq. def:mis, eq. polySimple)."""
    r = oracle.split("mis", 1, l=2)
    types = {tuple(t): z for t, z in zip(r["type"].tolist(), r["roots"])}
    assert abs(types[(2, 1)] + 2) < 1e-30 and abs(types[(0, 1)]) < 1e-30
    r = oracle.split("mis", 2, l=2)
    mis = sorted([z for t, z in zip(r["type"].tolist(), r["roots"]) if t == [2, 2]], key=lambda z: z.imag)
    assert len(mis) == 2 and abs(mis[0] + 1j) < 1e-30 and abs(mis[1] - 1j) < 1e-30
    r = oracle.split("mis", 1, l=3)
    cub = np.roots([1, 2, 2, 2])
    mis = np.array([z for t, z in zip(r["type"].tolist(), r["roots"]) if t == [3, 1]])
    _, dmax = match_sets(mis, cub)
    assert len(mis) == 3 and dmax < 1e-12


def test_s_2_4_example():
    """q_{2,4} = h1^3 h2^2 h4^2 m21 m22 m24 (App. A); s_{2,4} = h1 m21 m22 m24: 1+1+2+12 roots."""
    r = oracle.split("mis", 4, l=2)
    hist = {}
    for t in map(tuple, r["type"].tolist()):
        hist[t] = hist.get(t, 0) + 1
    assert hist == {(0, 1): 1, (2, 1): 1, (2, 2): 2, (2, 4): 12}


# --- counts, Vieta, symmetry ------------------------------------------------

@pytest.mark.parametrize("n", list(range(1, 13)))
def test_counts_and_exact_periods(n):
    """d = 2^(n-1) simple roots; the exact periods follow Thm countingHyp."""
    r = oracle.split("hyp", n)
    assert r["n_roots"] == 2 ** (n - 1)
    hist = {}
    for a, b in r["type"].tolist():
        assert a == 0
        hist[b] = hist.get(b, 0) + 1
    assert hist == counts.period_histogram(n)
    assert r["stats"]["retries"] == 0 and r["stats"]["endpoint_ok"] == 1
    assert lexsorted(r["roots"])


def test_known_period_counts():
    """Spot values of eq. HypCount (e.g. |Hyp(12)| = 2010, |Hyp(20)| = 523770)."""
    assert counts.period_histogram(12) == {1: 1, 2: 1, 3: 3, 4: 6, 6: 27, 12: 2010}
    assert counts.period_histogram(20) == {1: 1, 2: 1, 4: 6, 5: 15, 10: 495, 20: 523770}
    assert counts.hyp_count(24) == 8386440 and counts.hyp_count(28) == 134209530
    assert sum(counts.period_histogram(28).values()) == 2 ** 27


@pytest.mark.parametrize("n", [2, 3, 6, 9, 12])
def test_vieta_power_sums(n):
    """sum c = -2^(n-2) and sum c^2 = 2^(n-2) (top coefficients of the
    recurrence; the 'Viete checks' of Sec. 5)."""
    mpmath.mp.dps = 50
    r = oracle.split("hyp", n)
    zs = [mpmath.mpc(mpmath.mpf(x[0]) + x[1], mpmath.mpf(x[2]) + x[3]) for x in r["roots4"]]
    s1 = mpmath.fsum(zs)
    s2 = mpmath.fsum(z * z for z in zs)
    assert abs(s1 - (-(2 ** (n - 2)) if n >= 2 else 0)) < 1e-25 * 2 ** n
    if n >= 2:
        assert abs(s2 - 2 ** (n - 2)) < 1e-25 * 4 ** n


@pytest.mark.parametrize("n", [5, 8, 11, 12])
def test_conjugate_symmetry(n):
    r = oracle.split("hyp", n)
    z = r["roots"]
    _, dmax = match_sets(z, np.conj(z))
    assert dmax == 0.0


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_real_root_count_sturm(n):
    """Exact number of real roots of the integer polynomial (Sturm)."""
    sympy = pytest.importorskip("sympy")
    x = sympy.Symbol("x")
    co = p_coeffs(n)
    poly = sympy.Poly(list(reversed(co)), x)
    want = poly.count_roots()  # real roots, with multiplicity (simple here)
    r = oracle.split("hyp", n)
    assert r["stats"]["n_real"] == want
    assert int(np.sum(r["roots"].imag == 0)) == want


@pytest.mark.parametrize("n", list(range(SEPARATION["hyp_n_min"], 13)))
def test_separation_law(n):
    """min |c - c'| over Hyp(n) ~ 118.4 / 4^n, relative error < 0.1% for n >= 9
    (Sec. 6.3.2; tests/golden/separation_law.txt); allowed twice that here to
    absorb the rounding of the printed constant."""
    r = oracle.split("hyp", n)
    z = r["roots"][r["type"][:, 1] == n]
    sep = min_separation(z)
    law = SEPARATION["hyp_constant"] / 4.0 ** n
    assert abs(sep / law - 1) < 2 * SEPARATION["hyp_rel_error"]


# --- Misiurewicz counts -----------------------------------------------------

def test_misiurewicz_degree_identities():
    """deg s_{l,n} = sum_{k | gcd(n,l-1)} |Hyp(k)| + sum_{k | n} |Mis(l,k)| (eq. polyMisSimple),
    and eq. MisDeg for q_{l,n}; the totals for l + n <= 16."""
    pairs = counts.misiurewicz_pairs(16)
    assert len(pairs) == 105
    tot_deg = tot_mis = tot_q = 0
    for (l, n) in pairs:
        h = counts.type_histogram_s(l, n)
        assert sum(h.values()) == counts.deg_s(l, n)
        eta = lambda k: (l - 1) // k + 2  # noqa: E731  (eq. defMultHyp)
        q = sum(eta(k) * counts.hyp_count(k) + sum(counts.mis_count(j, k) for j in range(2, l + 1))
                for k in counts.divisors(n))
        assert q == 2 ** (l + n - 1)
        tot_deg += counts.deg_s(l, n)
        tot_mis += counts.mis_count(l, n)
        tot_q += 2 ** (l + n - 1)
    assert (tot_deg, tot_mis, tot_q) == (425986, 381108, 851972)


@pytest.mark.parametrize("order", [3, 4, 5, 6, 7, 8, 9, 10])
def test_misiurewicz_types(order):
    """Every (l, n) with l + n = order: the root count is deg s_{l,n} and the
    type histogram follows eq. MisCount / eq. polyMisSimple."""
    for l in range(2, order):
        n = order - l
        r = oracle.split("mis", n, l=l)
        assert r["n_roots"] == counts.deg_s(l, n)
        hist = {}
        for t in map(tuple, r["type"].tolist()):
            hist[t] = hist.get(t, 0) + 1
        assert hist == counts.type_histogram_s(l, n)
        z = r["roots"]
        _, dmax = match_sets(z, np.conj(z))
        assert dmax == 0.0


# --- the level line ----------------------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_level_line_iso_angle_zero(n):
    """The starts with P(z) = lambda0 (every 4th start, iso-angle 0), closed
    under conjugation, are exactly P^{-1}(lambda0) (Sec. 4.1: L_{z0,deg P} =
    P^{-1}(zeta0)); brute force on p_n - 5."""
    mpmath.mp.dps = 40
    r = oracle.split("hyp", n, want_starts=True)
    st = r["starts"]
    d = 2 ** (n - 1)
    assert st.size == 2 * d + 1
    iso0 = st[::4]
    full = np.concatenate([iso0, np.conj(iso0[(np.abs(iso0.imag) > 1e-12)])])
    co = p_coeffs(n)
    co[0] -= 5
    ref = np.array([complex(x) for x in mpmath.polyroots(list(reversed(co)), maxsteps=400,
                                                          extraprec=8 * len(co))])
    assert full.size == ref.size == d
    _, dmax = match_sets(full, ref)
    assert dmax < 1e-12
    # every start sits on |P| = 5 at the phase pi j / 2 of its index
    for j, s4 in enumerate(r["starts4"]):
        v, _ = oracle.evaluate("hyp", n, s4)
        val = complex(v[0] + v[1], v[2] + v[3])
        assert abs(val - 5 * 1j ** (j % 4)) < 1e-20
    assert abs(st[0].imag) == 0 and st[0].real > 0 and abs(st[-1].imag) < 1e-20 and st[-1].real < -2


def test_descent_statistics_band():
    """Behaviour (not result): at n = 12 about a quarter of the descents find a
    new root, ~73% are repeats and ~1% are discarded (Table newtonSteps, rows
    n = 28 .. 41; tests/golden/newton_steps.txt).  n = 12 is far below the
    table's periods, so the bands are wide."""
    tab = goldens.rows("newton_steps.txt")
    new_pc = [row[2] for row in tab]
    rep_pc = [row[5] for row in tab]
    div_pc = [row[8] for row in tab]
    r = oracle.split("hyp", 12)
    st = r["stats"]
    n_new = (r["n_roots"] + st["n_real"]) // 2  # upper-half representatives
    assert min(new_pc) / 100 - 0.06 < n_new / st["n_starts"] < max(new_pc) / 100 + 0.07
    assert min(rep_pc) / 100 - 0.13 < st["n_repeat"] / st["n_starts"] < max(rep_pc) / 100 + 0.07
    assert (st["n_diverge"] + st["n_timeout"]) / st["n_starts"] < 5 * max(div_pc) / 100


def test_fp64_build_agrees_at_n12():
    """The binary64 build (timed CPU baseline) finds the same set to ~1e-13."""
    q = oracle.split("hyp", 12)
    d = oracle.split("hyp", 12, fp64=True)
    assert d["n_roots"] == q["n_roots"] == 2048
    _, dmax = match_sets(d["roots"], q["roots"])
    assert dmax < 1e-13


def test_count_in_disk_and_polish():
    r = oracle.split("hyp", 6)
    z4 = r["roots4"]
    c = z4[3]
    assert oracle.count_in_disk(z4, c, 1e-6) == 1
    out, disp = oracle.polish("hyp", 6, c)
    assert disp < 1e-30
    # a point off a root moves by about its offset
    off = c.copy()
    off[0] += 1e-9
    out, disp = oracle.polish("hyp", 6, off, steps=6)
    assert abs(disp - 1e-9) < 1e-15


def test_golden_fixtures_carry_their_citation():
    """Every fixture under tests/golden/ names its source passage in the paper."""
    import os
    names = sorted(f for f in os.listdir(goldens.GOLDEN) if f.endswith(".txt"))
    assert names
    for name in names:
        cite = goldens.citation(name)
        assert "2402.06083" in cite, name
        assert any(w in cite for w in ("Sec.", "Table", "App.")), name
        assert goldens.rows(name), name


@pytest.mark.parametrize("l,n", [(2, 2), (2, 3), (3, 2), (3, 3), (4, 2)])
def test_level_line_iso_angle_zero_misiurewicz(l, n):
    """The same for s_{l,n} = p_{l+n-1} + p_{l-1} on its level |s| = 100 (Sec. 4.2):
    the iso-angle-0 starts and their conjugates are s^{-1}(100), brute force on
    the exact integer polynomial s_{l,n} - 100."""
    mpmath.mp.dps = 40
    r = oracle.split("mis", n, l=l, want_starts=True)
    st = r["starts"]
    d = 2 ** (l + n - 2)
    assert st.size == 2 * d + 1
    iso0 = st[::4]
    full = np.concatenate([iso0, np.conj(iso0[(np.abs(iso0.imag) > 1e-12)])])
    co = s_coeffs(l, n)
    co[0] -= 100
    ref = np.array([complex(x) for x in mpmath.polyroots(list(reversed(co)), maxsteps=400,
                                                          extraprec=8 * len(co))])
    assert full.size == ref.size == d
    _, dmax = match_sets(full, ref)
    assert dmax < 1e-12
    for j, s4 in enumerate(r["starts4"]):
        v, _ = oracle.evaluate("mis", n, s4, l=l)
        val = complex(v[0] + v[1], v[2] + v[3])
        assert abs(val - 100 * 1j ** (j % 4)) < 1e-18


@pytest.mark.parametrize("n", [3, 6, 9, 12])
def test_lifted_seed_is_the_walked_point(n):
    """Sec. 4.2: a point of |p_1| = lambda0 lifted through the nested family
    p_k -> p_{k+1} (target lambda0^2 at the doubled phase, radius brought
    back to lambda0) lands on the level line of p_n at the same external
    angle: the point the sequential walk from the real end point reaches at
    that index (pinned above against p_n^{-1}(5)), and P there is
    lambda0 e^{2 i pi j / M}."""
    st = oracle.level_line("hyp", n)["starts4"]  # M = 8, c_L = 4: start s is sub-step 2 s
    idx = sorted(set(np.linspace(0, len(st) - 1, min(len(st), 120)).astype(int)))
    for s in idx:
        p, fails = oracle.lift_seed(n, 2 * s)
        assert fails == 0
        d = abs(complex((p[0] - st[s, 0]) + (p[1] - st[s, 1]), (p[2] - st[s, 2]) + (p[3] - st[s, 3])))
        assert d < 1e-24, (s, d)
        v, _ = oracle.evaluate("hyp", n, p)
        t = 5 * 1j ** ((2 * s % 8) // 2)  # phase 2 pi (2 s) / 8: a multiple of pi / 2, exact
        assert abs(complex((v[0] - t.real) + v[1], (v[2] - t.imag) + v[3])) < 1e-24


def test_windows_together_find_every_root():
    """The level line cut into windows, each walked from its lifted seed with
    its own descents and root set (the bounded sample the timed CPU baseline
    draws), finds together exactly the upper-half roots of the whole split."""
    n = 12
    d = 2 ** (n - 1)
    J = 8 * d // 2
    cuts = [0, 1000, 2900, 2901, 4096, 6000, J - 17, J]
    found = [oracle.split_window(n, a, b, fp64=False, want_roots=True)["roots4"] for a, b in zip(cuts, cuts[1:])]
    w = np.concatenate(found)
    z = w[:, 0] + 1j * w[:, 2]
    uz = np.unique(np.round(z, 11))
    ref = oracle.split("hyp", n)["roots"]
    up = ref[ref.imag >= 0]
    assert uz.size == up.size == (d + int(np.sum(ref.imag == 0))) // 2
    _, dmax = match_sets(np.sort_complex(uz), np.sort_complex(np.round(up, 11)))
    assert dmax < 1e-10


def test_polish_many_is_polish():
    """The list form of the binary128 polish gives the one-point form's
    results, point by point; a true root (Cardano's period-3 centre) does not
    move."""
    z = np.array([-1.7548776662466927, -0.12256116687665362 + 0.7448617666197442j, 0.3 + 0.1j])
    disp, last, pts = oracle.polish_many("hyp", 3, z, steps=3, want_points=True)
    for i, c in enumerate(z):
        p, dd = oracle.polish("hyp", 3, c, steps=3)
        assert np.array_equal(p, pts[i]) and dd == disp[i]
    assert disp[0] < 1e-15 and last[0] < 1e-30
