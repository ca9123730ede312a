"""Separation statistics (mt_separation) against the oracle's definition
and the paper's separation law (Sec. 6.3.2).

The nearest-neighbour distance of every root is checked against the
oracle's minimum over all pairs, with and without a mask, and per bin
I_k = (-2 + 4^-(k+1), -2 + 4^-k] of Fig. separationHistogram; lists too
large for all pairs against scipy's k-d tree in full and against the
oracle on sampled roots (one row of all pairs each).  A synthetic column of points (Re spread far below the
neighbour distance) sends every point of it through the strip pass.  On GPU splits the minimum over
Hyp(n) (mask: exact period n) must follow 118.4 / 4^n to 0.2 % (Sec. 6.3.2
reports 0.1 % for n >= 9) and be the gap of the two left-most real roots;
at p_28 this needs the double-double low parts (the gap is 1.6e-15).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import goldens

SEP = goldens.table("separation_law.txt")  # Sec. 6.3.2

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("kind,n,l", [("hyp", 10, 0), ("hyp", 12, 0), ("mis", 6, 3)])
def test_nearest_neighbours_match_oracle(mt, kind, n, l):
    ref = oracle.split(kind, n, l=l)
    z = ref["roots"]
    nn, bands, mn = mt.separation(_t(z))
    want = oracle.nearest_neighbours(z)
    got = nn.cpu().numpy()
    assert np.allclose(got, want, rtol=1e-15, atol=0)  # hypot may round the last bit differently
    assert np.isclose(mn, want.min(), rtol=1e-15, atol=0)
    per = oracle.separation_bands(z, want)
    for k in range(64):
        w = per[k]
        assert (bands[k] == w) if np.isinf(w) else np.isclose(bands[k], w, rtol=1e-15, atol=0)


def test_mask_restricts_the_set(mt):
    """Hyp(12) only (exact period 12): neighbours outside the set do not count."""
    n = 12
    ref = oracle.split("hyp", n)
    z = ref["roots"]
    mask = ref["type"][:, 1] == n
    import torch
    nn, bands, mn = mt.separation(_t(z), mask=torch.as_tensor(mask.astype(np.uint8), device="cuda"))
    want = oracle.nearest_neighbours(z, mask)
    got = nn.cpu().numpy()
    assert np.allclose(got[mask], want[mask], rtol=1e-15, atol=0) and np.all(got[~mask] == 0)
    assert np.isclose(mn, want[mask].min(), rtol=1e-15, atol=0)


def _kd_nn(z, mask):
    spatial = pytest.importorskip("scipy.spatial")
    pts = np.stack([z.real[mask], z.imag[mask]], axis=1)
    d, _ = spatial.cKDTree(pts).query(pts, k=2)
    return d[:, 1]


def test_edge_cases(mt):
    """Empty list, one root (alone: +inf), two roots, duplicates (0)."""
    nn, bands, mn = mt.separation(_t(np.zeros(0)))
    assert nn.numel() == 0 and mn == np.inf and all(b == np.inf for b in bands)
    nn, bands, mn = mt.separation(_t([-1.0]))
    assert float(nn[0]) == np.inf and mn == np.inf
    nn, bands, mn = mt.separation(_t([-1.0, 0.25 + 0.5j]))
    assert np.allclose(nn.cpu().numpy(), abs(1.25 + 0.5j), rtol=1e-15) and bands[0] == mn
    nn, bands, mn = mt.separation(_t([-1.0, 0.0, -1.0]))
    assert list(nn.cpu().numpy()) == [0.0, 1.0, 0.0] and mn == 0.0


def test_isolated_roots_take_the_strip_pass(mt):
    """150k points in a column 1e-6 wide in Re (each Re window holds the
    whole column, so the Re-window scan leaves every one of them to the
    strip walk) plus 20k points spread over [-2, 0.25] x [-1.1, 1.1], about
    0.01 apart (dozens of strips: the block walk); 10 % masked out."""
    import torch
    rng = np.random.default_rng(5)
    col = (rng.uniform(0, 1e-6, 150000) - 0.5) + 1j * rng.uniform(-1, 1, 150000)
    far = rng.uniform(-2, 0.25, 20000) + 1j * rng.uniform(-1.1, 1.1, 20000)
    z = np.concatenate([col, far])
    mask = rng.uniform(size=z.size) < 0.9
    nn, bands, mn = mt.separation(_t(z), mask=torch.as_tensor(mask.astype(np.uint8), device="cuda"))
    got = nn.cpu().numpy()
    want = _kd_nn(z, mask)
    assert np.allclose(got[mask], want, rtol=1e-15, atol=0) and np.all(got[~mask] == 0)
    assert np.isclose(mn, want.min(), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [12, 16, 20, 24])
def test_separation_law(mt, n):
    """min distance within Hyp(n) ~ 118.4 / 4^n, between the two left-most
    roots; up to p_20 every distance against scipy's k-d tree."""
    res = mt.split_hyperbolic(n, "mixed" if n >= 22 else "fp64")
    z = res.roots
    t = mt.classify("hyp", n, z)
    mask = (t == n).to(dtype=__import__("torch").uint8)
    nn, bands, mn = mt.separation(z, mask=mask)
    assert abs(mn * 4.0 ** n / SEP["hyp_constant"] - 1) < 2 * SEP["hyp_rel_error"], mn * 4.0 ** n
    zz = z[:2].cpu().numpy()
    assert abs(abs(zz[1] - zz[0]) - mn) <= 1e-12 * mn
    if n <= 20:
        m = mask.cpu().numpy().astype(bool)
        got = nn.cpu().numpy()
        zc = z.cpu().numpy()
        assert np.allclose(got[m], _kd_nn(zc, m), rtol=1e-15, atol=0)
        rows = np.random.default_rng(n).choice(np.nonzero(m)[0], 64, replace=False)
        assert np.allclose(got[rows], oracle.nearest_neighbours(zc, m, idx=rows), rtol=1e-15, atol=0)


def test_separation_law_double_double_p28(mt):
    """p_28: the two left-most roots of Hyp(28) are 1.6e-15 apart; with the
    low parts of the MT_DD split the minimum over Hyp(28) follows the law,
    and matches a binary128 evaluation of that gap.  Over all roots of p_28
    the minimum is smaller: near -2 the components of period 14 are of size
    ~4^-28, so each centre lies that close to its period-28 satellite."""
    import torch
    n = 28
    res = mt.split_hyperbolic(n, "dd", want_lo=True, max_retries=0)
    mask = (mt.classify("hyp", n, res.roots) == n).to(torch.uint8)
    _, _, mn_all = mt.separation(res.roots, roots_lo=res.roots_lo)
    nn, bands, mn = mt.separation(res.roots, roots_lo=res.roots_lo, mask=mask)
    assert mn_all < 0.6 * mn
    assert abs(mn * 4.0 ** n / SEP["hyp_constant"] - 1) < 2 * SEP["hyp_rel_error"], mn * 4.0 ** n
    z = res.roots[:2].cpu().numpy()
    zl = res.roots_lo[:2].cpu().numpy()
    # the binary128 oracle's Newton limits of the two left-most roots
    a, _ = oracle.polish("hyp", n, np.array([z[0].real, zl[0].real, 0.0, 0.0]), steps=3)
    b, _ = oracle.polish("hyp", n, np.array([z[1].real, zl[1].real, 0.0, 0.0]), steps=3)
    gap = (b[0] - a[0]) + (b[1] - a[1])
    assert abs(mn - gap) <= 1e-12 * gap
    nn_set = torch.where(mask.bool(), nn, torch.full_like(nn, float("inf")))  # 0 outside the set
    assert int(torch.argmin(nn_set)) in (0, 1)
    # sampled roots against the oracle's row of all pairs, in double-double
    m = mask.cpu().numpy().astype(bool)
    rows = np.concatenate([[0, 1], np.random.default_rng(28).choice(np.nonzero(m)[0], 4, replace=False)])
    zc, zlc = res.roots.cpu().numpy(), res.roots_lo.cpu().numpy()
    want = oracle.nearest_neighbours(zc, m, z_lo=zlc, idx=rows)
    assert np.allclose(nn.cpu().numpy()[rows], want, rtol=1e-13, atol=0)
