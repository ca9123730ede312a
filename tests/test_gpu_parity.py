"""Parity of the CUDA path (through the C ABI) with the oracle, step by step
and end to end.  Every test here needs a GB300 and the built library.

Tolerances: roots within |dc| <= 1e-12 of the oracle in FP64 mode, counts
and types exact (integers), certificate flags exact for true roots.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import counts
from tests.rootsets import lexsorted, match_sets, match_sorted

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


def _t(x):
    import torch
    return torch.as_tensor(np.asarray(x, dtype=np.complex128), device="cuda")


# --- a0: orbit evaluation ------------------------------------------------------

def test_eval_at_minus_two(mt):
    """p_n(-2) = 2 and p_n'(-2) = -(4^n+2)/6, exact in binary64 for n <= 26."""
    for n in range(2, 27):
        out = mt.evaluate("hyp", n, _t([-2.0])).cpu().numpy()[0]
        assert out[0] == 2.0
        assert out[1] == -(4 ** n + 2) / 6


def test_eval_vs_oracle_on_level_line(mt):
    """P and P' at the oracle's level-line points agree to rounding."""
    for kind, n, l in (("hyp", 9, 0), ("hyp", 12, 0), ("mis", 5, 3)):
        st = oracle.split(kind, n, l=l, want_starts=True, want_types=False)["starts4"]
        c = st[:, 0] + 1j * st[:, 2]
        g = mt.evaluate(kind, n, _t(c), l=l).cpu().numpy()
        for i in range(0, len(c), max(1, len(c) // 200)):
            v, dv = oracle.evaluate(kind, n, st[i], l=l)
            P = complex(v[0] + v[1], v[2] + v[3])
            D = complex(dv[0] + dv[1], dv[2] + dv[3])
            assert abs(g[i, 0] - P) <= 1e-12 * abs(D) + 1e-13 * abs(P)
            assert abs(g[i, 1] - D) <= 1e-11 * abs(D)


# --- a1-a3: the level line -----------------------------------------------------

@pytest.mark.parametrize("kind,n,l", [("hyp", 3, 0), ("hyp", 8, 0), ("hyp", 12, 0), ("mis", 6, 2),
                                      ("mis", 4, 4)])
def test_level_line_matches_oracle(mt, kind, n, l):
    """Same starts, same external-angle order: start s satisfies
    P = lambda0 e^{i pi s / 2} and equals the oracle's s-th start."""
    g, st = mt.level_line(kind, n, l=l)
    g = g.cpu().numpy()
    ref = oracle.split(kind, n, l=l, want_starts=True, want_types=False)["starts"]
    d = oracle.degree(kind, n, l)
    assert g.size == ref.size == 2 * d + 1
    assert st["walk_fail"] == 0
    h = np.abs(np.diff(ref))
    hl = np.minimum(np.concatenate([h, [np.inf]]), np.concatenate([[np.inf], h]))
    err = np.abs(g - ref)
    assert np.all(err <= 1e-2 * hl), float(np.max(err / hl))
    lam = oracle.default_lambda0(kind)
    vals = mt.evaluate(kind, n, _t(g), l=l).cpu().numpy()[:, 0]
    want = lam * (1j ** (np.arange(g.size) % 4))
    assert np.max(np.abs(vals - want)) < 1e-2 * lam
    assert g[0].imag == 0 and g[-1].imag == 0


def test_level_line_n20_sampled(mt):
    """n = 20: every chunk ends on the next seed; sampled starts sit on the
    right phase; the first 1/64 of the line equals the oracle's walk."""
    g, st = mt.level_line("hyp", 20)
    g = g.cpu().numpy()
    assert g.size == 2 ** 20 + 1 and st["walk_fail"] == 0
    ref = oracle.split("hyp", 20, want_starts=True, want_types=False, fp64=True, frac=1 / 64)["starts"]
    k = ref.size
    h = np.abs(np.diff(ref))
    hl = np.minimum(np.concatenate([h, [np.inf]]), np.concatenate([[np.inf], h]))
    # the walk stops each sub-step at 1e-3 of the sub-step length: the same
    # point of the discrete level line is matched to a percent of its spacing
    rel = np.abs(g[:k] - ref) / hl
    assert np.all(rel <= 1e-2), (float(rel.max()), int(np.argmax(rel)))


# --- a4: descents -----------------------------------------------------------------

def test_descend_from_oracle_starts(mt):
    """Descents from the oracle's starts: every converged iterate is a true
    root (binary128 polish moves it < 1e-12) and together they find all roots."""
    n = 11
    r = oracle.split("hyp", n, want_starts=True)
    out, status, st = mt.descend("hyp", n, _t(r["starts"]))
    out = out.cpu().numpy()
    status = status.cpu().numpy()
    conv = out[status == 0]
    assert conv.size > 0.9 * out.size
    for z in conv[:: max(1, conv.size // 300)]:
        _, disp = oracle.polish("hyp", n, z, steps=3)
        assert disp < TOL_FP64
    up = np.unique(np.round(np.concatenate([conv, np.conj(conv)]), 9))
    assert up.size == 2 ** (n - 1)
    assert st["desc_newton"] > 0


# --- a5-a7: whole path at small sizes ----------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 9, 10, 11, 12])
def test_split_hyperbolic_small(mt, n, prec):
    res = mt.split_hyperbolic(n, prec)
    z = res.roots.cpu().numpy()
    ref = oracle.split("hyp", n)
    assert z.size == ref["n_roots"] == 2 ** (n - 1)
    dmax, _ = match_sorted(z, ref["roots"], TOL_FP64)
    assert dmax < TOL_FP64
    assert lexsorted(z)
    st = res.stats
    hist = {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]}
    assert hist == counts.period_histogram(n)
    assert st["n_cert_pass"] == z.size
    assert st["n_real"] == int(np.sum(z.imag == 0)) == ref["stats"]["n_real"]
    assert np.all(z.imag[z.imag == 0] == 0) and not np.any(np.signbit(z.imag[z.imag == 0]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("l,n", [(2, 1), (2, 2), (3, 1), (2, 4), (3, 3), (4, 2), (5, 4), (3, 7), (7, 3),
                                 (2, 8)])
def test_split_misiurewicz_small(mt, l, n, prec):
    res = mt.split_misiurewicz(l, n, prec)
    z = res.roots.cpu().numpy()
    ref = oracle.split("mis", n, l=l)
    assert z.size == ref["n_roots"] == counts.deg_s(l, n)
    dmax, _ = match_sorted(z, ref["roots"], TOL_FP64)
    assert dmax < TOL_FP64
    assert lexsorted(z)
    # Mis(l, n) mask vs the oracle's types, root by root (nearest-neighbour pairing)
    mis = res.is_mis.cpu().numpy().astype(bool)
    perm, _ = match_sets(z, ref["roots"])
    to = ref["type"][perm]
    want = (to[:, 0] == l) & (to[:, 1] == n)
    assert int(mis.sum()) == counts.mis_count(l, n) == int(want.sum())
    assert np.array_equal(mis, want)
    st = res.stats
    for (a, k), cnt in counts.type_histogram_s(l, n).items():
        code = k if a == l else 32 + k
        assert st["count_by_type"][code] == cnt
    assert st["n_cert_pass"] == z.size


# --- full size (the benchmarked configuration) -------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_split_hyperbolic_n20_full(mt, prec):
    """n = 20, 524288 roots: exact count and Moebius histogram, Vieta sums,
    conjugate symmetry, all certified, sampled roots polished in binary128,
    and the whole set against the binary64 oracle."""
    n = 20
    res = mt.split_hyperbolic(n, prec)
    assert res.stats["prec_used"] == (1 if prec == "mixed" else 0), res.stats
    z = res.roots.cpu().numpy()
    d = 2 ** (n - 1)
    st = res.stats
    assert z.size == d and st["n_roots"] == d
    hist = {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]}
    assert hist == counts.period_histogram(n)
    assert st["n_cert_pass"] == d
    assert lexsorted(z)
    s1 = np.sum(z)
    assert abs(s1.real + 2 ** (n - 2)) < 1e-6 and abs(s1.imag) < 1e-9
    s2 = np.sum(z * z)
    assert abs(s2.real - 2 ** (n - 2)) < 1e-5
    zc = np.conj(z)
    assert np.array_equal(np.sort_complex(zc), np.sort_complex(z))
    assert 0.04 < st["n_real"] / d < 0.12
    rng = np.random.default_rng(0)
    for i in rng.choice(d, 400, replace=False):
        _, disp = oracle.polish("hyp", n, z[i], steps=3)
        assert disp < TOL_FP64
    ref = oracle.split("hyp", n, fp64=True, want_types=False)
    assert ref["n_roots"] == d
    dmax, _ = match_sorted(z, ref["roots"], TOL_FP64)
    assert dmax < TOL_FP64  # binary64 oracle: both sides carry binary64 rounding (~1e-15)


# --- certificate ---------------------------------------------------------------------

def test_certify_accepts_roots_and_rejects_shifted_points(mt):
    n = 10
    ref = oracle.split("hyp", n)
    z = ref["roots"]
    ok, rad, npass = mt.certify("hyp", n, _t(z))
    ok = ok.cpu().numpy()
    rad = rad.cpu().numpy()
    assert npass == z.size and ok.all()
    # each certified disk holds exactly one root of the binary128 list
    for i in range(0, z.size, 7):
        assert oracle.count_in_disk(ref["roots4"], z[i], rad[i]) == 1
    # points shifted by 10 radii hold no root: none may pass
    shifted = z + 10 * rad * np.exp(1j * np.linspace(0, 2 * np.pi, z.size))
    ok2, _, npass2 = mt.certify("hyp", n, _t(shifted))
    assert npass2 == 0


def test_classify_matches_oracle_types(mt):
    n = 12
    ref = oracle.split("hyp", n)
    t = mt.classify("hyp", n, _t(ref["roots"])).cpu().numpy()
    assert np.array_equal(t, ref["type"][:, 1])
    l, n = 3, 6
    ref = oracle.split("mis", n, l=l)
    t = mt.classify("mis", n, _t(ref["roots"]), l=l).cpu().numpy()
    want = np.where(ref["type"][:, 0] == 0, 32 + ref["type"][:, 1], ref["type"][:, 1])
    assert np.array_equal(t, want)


# --- edge cases -------------------------------------------------------------------

def test_errors_and_capacity(mt):
    import ctypes
    import torch
    L = mt.load()
    o = mt.options()
    n = 8
    ws = mt.Workspace(mt.workspace_bytes("hyp", n, opts=o))
    small = torch.empty((10, 2), dtype=torch.float64, device="cuda")
    n_out = ctypes.c_int64(0)
    rc = L.mt_split_hyperbolic(n, ctypes.byref(o), small.data_ptr(), None, 10, ws.buf.data_ptr(),
                               ws.buf.numel(), ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_ECAPACITY and n_out.value == 2 ** (n - 1)
    rc = L.mt_split_hyperbolic(n, ctypes.byref(o), small.data_ptr(), None, 10, ws.buf.data_ptr(),
                               100, ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_ENOMEM
    with pytest.raises((ValueError, mt.MtError)):
        mt.split_hyperbolic(41)
    rc = L.mt_split_hyperbolic(41, ctypes.byref(o), small.data_ptr(), None, 10, ws.buf.data_ptr(),
                               ws.buf.numel(), ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_EINVAL


def test_repeated_calls_are_identical(mt):
    """Bit-identical output on repeated calls (the set and its order)."""
    a = mt.split_hyperbolic(14).roots.cpu().numpy()
    b = mt.split_hyperbolic(14).roots.cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_split_hyperbolic_n24_invariants(mt, prec):
    """n = 24 (8,388,608 roots): exact count and Moebius histogram, every root
    certified, conjugate symmetry, Vieta sums, and sampled roots polished in
    binary128 (the binary128 oracle is too slow for the whole set)."""
    n = 24
    res = mt.split_hyperbolic(n, prec)
    st = res.stats
    d = 2 ** (n - 1)
    z = res.roots.cpu().numpy()
    assert z.size == d and st["n_cert_pass"] == d
    hist = {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]}
    assert hist == counts.period_histogram(n)
    assert lexsorted(z)
    s1 = np.sum(z)
    assert abs(s1.real + 2 ** (n - 2)) < 1e-4 and abs(s1.imag) < 1e-7
    zc = np.conj(z)
    assert np.array_equal(np.sort_complex(zc), np.sort_complex(z))
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(d, 200, replace=False), np.arange(20)])  # + the left tip
    for i in idx:
        _, disp = oracle.polish("hyp", n, z[i], steps=3)
        assert disp < TOL_FP64


# --- the batched Misiurewicz split (all s_{l,n}, l + n <= max_order, one pass) ----

def _batch(mt, max_order):
    roots, mis, offs, stats, pairs = mt.split_misiurewicz_batch(max_order)
    return roots.cpu().numpy(), mis.cpu().numpy().astype(bool), offs, stats, pairs


def test_batch_small_orders_match_oracle(mt):
    """Every pair with l + n <= 9 against the binary128 oracle, root by root."""
    roots, mis, offs, stats, pairs = _batch(mt, 9)
    assert len(pairs) == len(counts.misiurewicz_pairs(9))
    for p, (l, n) in enumerate(pairs):
        z = roots[offs[p]:offs[p + 1]]
        ref = oracle.split("mis", n, l=l)
        assert z.size == ref["n_roots"] == counts.deg_s(l, n), (l, n)
        dmax, _ = match_sorted(z, ref["roots"], TOL_FP64)
        assert dmax < TOL_FP64, (l, n, dmax)
        assert lexsorted(z)
        perm, _ = match_sets(z, ref["roots"])
        to = ref["type"][perm]
        assert np.array_equal(mis[offs[p]:offs[p + 1]], (to[:, 0] == l) & (to[:, 1] == n)), (l, n)
        assert stats[p]["n_cert_pass"] == z.size


def test_batch_order16_full(mt):
    """The whole l + n <= 16 batch (105 polynomials, 425,986 roots): per
    polynomial exact count and type histogram (eq. MisCount /
    eq. polyMisSimple), every root certified, conjugate symmetry; the largest
    polynomials of each preperiod against the binary64 oracle."""
    roots, mis, offs, stats, pairs = _batch(mt, 16)
    assert len(pairs) == 105 and offs[-1] == 425986
    assert int(mis.sum()) == 381108
    for p, (l, n) in enumerate(pairs):
        z = roots[offs[p]:offs[p + 1]]
        st = stats[p]
        assert z.size == counts.deg_s(l, n) and st["n_cert_pass"] == z.size, (l, n)
        for (a, k), cnt in counts.type_histogram_s(l, n).items():
            assert st["count_by_type"][k if a == l else 32 + k] == cnt, (l, n, a, k)
        assert int(mis[offs[p]:offs[p + 1]].sum()) == counts.mis_count(l, n)
        assert np.array_equal(np.sort_complex(np.conj(z)), np.sort_complex(z))
    for (l, n) in [(2, 14), (3, 13), (5, 11), (8, 8), (12, 4), (15, 1)]:
        p = pairs.index((l, n))
        z = roots[offs[p]:offs[p + 1]]
        ref = oracle.split("mis", n, l=l, fp64=True, want_types=False)
        assert ref["n_roots"] == z.size
        dmax, _ = match_sorted(z, ref["roots"], 1e-11)
        assert dmax < 1e-11, (l, n, dmax)


# --- CUDA-graph replay and the autotuner ---------------------------------------------

@pytest.mark.parametrize("n,prec", [(12, "fp64"), (20, "mixed")])
def test_graph_replay_is_identical(mt, n, prec):
    """Captured once, replayed twice: the same roots as the plain launch sequence."""
    a = mt.split_hyperbolic(n, prec).roots.cpu().numpy()
    w = mt.Workspace()
    b = mt.split_hyperbolic(n, prec, use_graph=1, work=w)
    c = mt.split_hyperbolic(n, prec, use_graph=1, work=w)
    assert np.array_equal(a, b.roots.cpu().numpy()) and np.array_equal(a, c.roots.cpu().numpy())
    assert c.stats["n_cert_pass"] == a.size and c.stats["ms_total"] > 0


def test_autotune_picks_a_valid_layout(mt):
    cl, blk, ms = mt.autotune("hyp", 14)
    assert 3 <= cl <= 10 and blk in (32, 64, 128) and ms > 0
    res = mt.split_hyperbolic(14)
    assert res.stats["n_roots"] == 2 ** 13 and res.stats["n_cert_pass"] == 2 ** 13
    assert res.stats["n_chunks"] == (8 * 2 ** 13 >> cl) // 2
