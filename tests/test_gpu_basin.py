"""The Newton-basin certificate (Thm proofContract) against the binary128
oracle.

mt_certify_basin claims that Newton's map, started anywhere in D(c_j, eps_j),
converges to the root proven in D(c_j, r_j).  The pin is that claim executed
independently: binary128 Newton iterations of the oracle from points on the
boundary circle |z - c_j| = 0.99 eps_j must end at the same root as Newton
from c_j itself (and at no other root of the oracle's list).  A radius that
the theorem cannot prove (eps_max below 3 eta) must give 0.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as m
    m.load()
    return m


def _newton128(kind, n, l, c, steps=80):
    out, _ = oracle.polish(kind, n, np.asarray(c, dtype=np.float64), l=l, steps=steps)
    return out


def _check_basin(kind, n, l, z, zl, eps, ref4, sample, rng):
    """binary128 Newton from 4 points at 0.99 eps_j around c_j ends at c_j's root"""
    roots = ref4[:, 0] + ref4[:, 1] + 1j * (ref4[:, 2] + ref4[:, 3])
    for j in sample:
        base = np.array([z[j].real, zl[j].real if zl is not None else 0.0,
                         z[j].imag, zl[j].imag if zl is not None else 0.0])
        target = _newton128(kind, n, l, base)
        t = complex(target[0] + target[1], target[2] + target[3])
        k = int(np.argmin(np.abs(roots - t)))
        assert abs(roots[k] - t) < 1e-25  # c_j's Newton limit is a root of the oracle's list
        for th in rng.uniform(0, 2 * np.pi, 4):
            d = 0.99 * eps[j] * np.exp(1j * th)
            # the perturbation added part by part keeps the dd digits of c_j
            start = base + np.array([d.real, 0.0, d.imag, 0.0])
            w = _newton128(kind, n, l, start)
            assert abs(complex(w[0] - target[0] + w[1] - target[1], w[2] - target[2] + w[3] - target[3])) < 1e-25


@pytest.mark.parametrize("kind,n,l", [("hyp", 10, 0), ("hyp", 16, 0), ("mis", 5, 3), ("mis", 7, 4)])
def test_basin_binary64_roots(mt, kind, n, l):
    res = mt.split_hyperbolic(n) if kind == "hyp" else mt.split_misiurewicz(l, n)
    ok, rad, npass = mt.certify(kind, n, res.roots, l=l)
    assert npass == res.roots.shape[0]
    eps, nb = mt.certify_basin(kind, n, res.roots, rad, l=l)
    e = eps.cpu().numpy()
    r = rad.cpu().numpy()
    assert nb == e.size and np.all(e > 0)  # every root gets a basin radius
    z = res.roots.cpu().numpy()
    ref = oracle.split(kind, n, l=l)
    rng = np.random.default_rng(n)
    sample = rng.choice(z.size, min(z.size, 24), replace=False)
    _check_basin(kind, n, l, z, None, e, ref["roots4"], sample, rng)
    assert np.all(e <= 1e-6) and np.all(r > 0)  # eps <= eps_max (default 1e-6)


def test_basin_refuses_radii_below_three_eta(mt):
    """Thm proofContract needs eps > 3 eta: binary64 roots carry eta ~ 1e-17
    or more, so eps_max = 1e-20 proves nothing -- except at the root c = 0,
    which binary64 resolves to ~1e-28 (so eta is that small there)."""
    res = mt.split_hyperbolic(12)
    _, rad, _ = mt.certify("hyp", 12, res.roots)
    eps, nb = mt.certify_basin("hyp", 12, res.roots, rad, eps_max=1e-20)
    z = res.roots.cpu().numpy()
    e = eps.cpu().numpy()
    assert nb == 1 and abs(z[e != 0][0]) < 1e-20


def test_basin_zero_where_no_root_is_proven(mt):
    """r_j = 0 (no localisation) gives no basin."""
    import torch
    res = mt.split_hyperbolic(9)
    rad = torch.zeros(res.roots.shape[0], dtype=torch.float64, device="cuda")
    eps, nb = mt.certify_basin("hyp", 9, res.roots, rad)
    assert nb == 0


def test_basin_double_double_roots(mt):
    """dd roots (dd_all split): the certificate with dd centres; binary128
    Newton from the disk boundary ends at the dd root's limit."""
    n = 10
    res = mt.split_hyperbolic(n, "dd", want_lo=True, dd_all=1)
    ok, rad, npass = mt.certify("hyp", n, res.roots, roots_lo=res.roots_lo)
    assert npass == res.roots.shape[0]
    eps, nb = mt.certify_basin("hyp", n, res.roots, rad, roots_lo=res.roots_lo)
    e = eps.cpu().numpy()
    assert nb == e.size and np.all(e > 0)
    z = res.roots.cpu().numpy()
    zl = res.roots_lo.cpu().numpy()
    ref = oracle.split("hyp", n)
    rng = np.random.default_rng(7)
    _check_basin("hyp", n, 0, z, zl, e, ref["roots4"], rng.choice(z.size, 16, replace=False), rng)
