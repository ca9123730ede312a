"""Every configuration against the binary128 oracle at the stated tolerance:
each GPU root within |dc| <= 1e-12 of a root of P in binary64 modes, and
within 1e-20 in double-double mode.

The analogue of the paper's a-posteriori check of its FP80 lists against
MPFR (Sec. 6.3): every GPU root of p_20 and p_24 (and a stratified sample of
p_28 with every one of its double-double roots) is Newton-polished by the
oracle in binary128 on the host cores.  The displacement is the root's
distance to the root of P it converges to; the last binary128 step shows
that convergence.  The polished roots are pairwise distinct, so with the
count equal to the degree the GPU list is the whole root set.

The certificate is pinned on the same lists: every checked disk D(c_j, r_j)
that mt_certify proves holds exactly one of the binary128 roots, also at the
left tip of p_24, where the two left-most roots lie 4.2e-13 apart, closer
than the 1e-12 radius cap, so the radius is cut by the neighbour rule.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import counts
from tests import hostpool
from tests.rootsets import lexsorted

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_DD = 1e-20
CONVERGED = 1e-25  # last binary128 step of a polish that reached a simple root


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


_CACHE: dict = {}


def _polished(mt, n, prec):
    """The split of p_n in this tier with every root polished by the oracle."""
    key = (n, prec)
    if key not in _CACHE:
        res = mt.split_hyperbolic(n, prec)
        z = res.roots.cpu().numpy()
        disp, last, pts = hostpool.polish_all("hyp", n, z)
        _CACHE[key] = (res, z, disp, last, pts)
    return _CACHE[key]


@pytest.mark.parametrize("n,prec", [(20, "fp64"), (20, "mixed"), (24, "mixed")])
def test_every_root_within_tolerance_of_binary128(mt, n, prec):
    res, z, disp, last, pts = _polished(mt, n, prec)
    d = 2 ** (n - 1)
    assert z.size == d and res.stats["n_cert_pass"] == d
    assert np.all(np.isfinite(disp)) and np.all(last < CONVERGED), float(np.max(last))
    assert float(disp.max()) <= TOL_FP64, float(disp.max())
    # distinct binary128 roots: the list is the whole root set of p_n
    assert hostpool.min_gap(pts) > 1e-16
    print("p_%d %s: max |dc| vs binary128 = %.3e over %d roots" % (n, prec, disp.max(), z.size))


def test_p24_whole_set_matches_the_binary64_oracle(mt):
    """The oracle's own split of p_24 in binary64 (the timed baseline build),
    run as windows tiling the level line on the host cores, against the
    GPU's roots: every oracle root lies within 1e-12 of a GPU root and every
    GPU root within 1e-12 of an oracle root.  (The binary64 oracle keeps a
    few duplicates at the left tip, where roots 4.2e-13 apart meet its
    binary64 stopping rule, so the comparison is by nearest neighbours, and
    its few roots more than 1e-12 from a GPU root are polished in binary128
    before they are compared.)"""
    from scipy.spatial import cKDTree
    res, z, _, _, _ = _polished(mt, 24, "mixed")
    r4 = hostpool.oracle_windows(24, 256)
    u = r4[:, 0] + 1j * r4[:, 2]
    g = z[z.imag >= 0]
    assert u.size >= g.size
    tg = cKDTree(np.stack([g.real, g.imag], axis=1))
    tu = cKDTree(np.stack([u.real, u.imag], axis=1))
    d1, _ = tg.query(np.stack([u.real, u.imag], axis=1))
    d2, _ = tu.query(np.stack([g.real, g.imag], axis=1))
    assert float(d2.max()) < TOL_FP64, float(d2.max())
    # the binary64 oracle's own error at the tip can exceed 1e-12: its roots
    # farther than that from every GPU root are polished in binary128 first
    far = np.nonzero(d1 >= TOL_FP64)[0]
    assert far.size < 64, far.size
    if far.size:
        _, _, pts = hostpool.polish_all("hyp", 24, u[far], zl=r4[far, 1] + 1j * r4[far, 3])
        d3, _ = tg.query(np.stack([pts[:, 0], pts[:, 2]], axis=1))
        assert float(d3.max()) < TOL_FP64, float(d3.max())


@pytest.mark.parametrize("n,prec", [(20, "fp64"), (24, "mixed")])
def test_certified_disks_hold_exactly_one_root(mt, n, prec):
    """Thm proofRoots: each passing disk D(c_j, r_j) holds exactly one root
    of P.  Checked against the binary128 roots for the 64 left-most roots
    (the tip cluster, where the radius is cut by the neighbour rule) and
    1000 sampled ones."""
    res, z, _, _, pts = _polished(mt, n, prec)
    ok, rad, npass = mt.certify("hyp", n, res.roots)
    ok, rad = ok.cpu().numpy(), rad.cpu().numpy()
    assert npass == z.size and ok.all()
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([np.arange(64), rng.choice(z.size, 1000, replace=False)]))
    order = np.argsort(pts[:, 0])
    xs = pts[order, 0]
    for j in idx:
        lo = np.searchsorted(xs, z[j].real - 2 * rad[j] - 1e-15)
        hi = np.searchsorted(xs, z[j].real + 2 * rad[j] + 1e-15)
        near = pts[order[lo:hi]]
        assert oracle.count_in_disk(near, z[j], rad[j]) == 1, (j, rad[j])
    if n == 24:  # the tip pair is closer than the radius cap: the neighbour rule set the radius
        gap = abs(z[1] - z[0])
        assert gap < 1e-12 and rad[0] <= 0.45 * gap * (1 + 1e-12)


def test_certificate_of_a_list_missing_a_tip_root(mt):
    """p_24 without its left-most root, then with that root replaced by a
    point next to its partner: the list no longer certifies as complete.
    Without the root the partner's first radius, 0.45 of the distance to its
    next neighbour, would hold both roots: the disk the certificate does
    prove must hold exactly one of the binary128 roots (the removed one
    included).  With the stand-in point the count is the degree again; the
    stand-in's disk holds no root, so it must fail."""
    import torch
    res, z, _, _, pts = _polished(mt, 24, "mixed")
    d = z.size
    tip = pts[:256]  # the binary128 roots of the left tip (sorted like z), the removed one included
    zz = z[1:].copy()
    ok, rad, npass = mt.certify("hyp", 24, torch.as_tensor(zz, device="cuda"))
    ok, rad = ok.cpu().numpy(), rad.cpu().numpy()
    assert npass < d
    for j in np.nonzero(ok[:64])[0]:
        assert oracle.count_in_disk(tip, zz[j], rad[j]) == 1, (j, rad[j])
    fake = z.copy()
    fake[0] = z[1] + 0.25 * (z[0] - z[1])  # count == degree, one point is no root
    ok2, rad2, npass2 = mt.certify("hyp", 24, torch.as_tensor(fake, device="cuda"))
    ok2, rad2 = ok2.cpu().numpy(), rad2.cpu().numpy()
    assert npass2 < d and not ok2[0]
    for j in np.nonzero(ok2[:64])[0]:
        assert oracle.count_in_disk(tip, fake[j], rad2[j]) == 1, (j, rad2[j])


def test_p28_dd_against_binary128(mt):
    """p_28 in MT_DD (134M roots): every double-double root (nonzero low
    part) polished with its low part within 1e-20, a stratified sample of
    131,072 binary64 roots plus the 64 left-most within 1e-12, and the
    polished double-double roots pairwise distinct."""
    n = 28
    d = 2 ** (n - 1)
    res = mt.split_hyperbolic(n, "dd", want_lo=True, max_retries=0)
    st = res.stats
    assert st["n_roots"] == d and st["n_cert_pass"] == d and st["prec_used"] == 2
    assert {k: st["count_by_type"][k] for k in range(64) if st["count_by_type"][k]} == counts.period_histogram(n)
    z = res.roots.cpu().numpy()
    zl = res.roots_lo.cpu().numpy()
    assert lexsorted(z, zl)
    dd = np.nonzero(zl != 0)[0]
    assert dd.size > 0
    disp, last, pts = hostpool.polish_all("hyp", n, z[dd], zl=zl[dd])
    assert np.all(last < 1e-28) and float(disp.max()) <= TOL_DD, float(disp.max())
    assert hostpool.min_gap(pts) > 1e-25
    rest = np.nonzero(zl == 0)[0]  # the binary64 roots (no low part)
    pick = np.unique(np.concatenate([rest[np.linspace(0, rest.size - 1, 1 << 17).astype(np.int64)], rest[:64]]))
    disp2, last2, _ = hostpool.polish_all("hyp", n, z[pick])
    assert np.all(last2 < CONVERGED) and float(disp2.max()) <= TOL_FP64, float(disp2.max())
    print("p_28 dd: %d dd roots max %.3e; %d binary64 roots max %.3e" % (dd.size, disp.max(), pick.size,
                                                                       disp2.max()))
