"""Comparison helpers for root sets (test-only; no method arithmetic here)."""
from __future__ import annotations

import numpy as np


def match_sets(a: np.ndarray, b: np.ndarray) -> tuple[np.ndarray, float]:
    """Pair each point of ``a`` with its nearest point of ``b``.

    Both are 1-D complex arrays of the same length.  Returns (perm, maxdist)
    where b[perm[i]] is the partner of a[i]; raises AssertionError unless the
    pairing is a bijection.  Works by sorting both sets on the real part and
    searching a window, so it scales to millions of points."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    assert a.shape == b.shape, (a.shape, b.shape)
    n = a.size
    if n == 0:
        return np.zeros(0, dtype=np.int64), 0.0
    ob = np.argsort(b.real, kind="stable")
    br = b.real[ob]
    perm = np.empty(n, dtype=np.int64)
    best = np.full(n, np.inf)
    # candidates within a growing real-part window
    idx = np.searchsorted(br, a.real)
    width = 1
    todo = np.arange(n)
    while todo.size:
        lo = np.clip(idx[todo] - width, 0, n)
        hi = np.clip(idx[todo] + width, 0, n)
        for t, (i, l, h) in enumerate(zip(todo, lo, hi)):
            seg = ob[l:h]
            d = np.abs(b[seg] - a[i])
            k = int(np.argmin(d))
            perm[i] = seg[k]
            best[i] = d[k]
        # a pairing is final once the window edges are farther than the best
        left_ok = (lo == 0) | (np.abs(a.real[todo] - br[np.maximum(lo - 1, 0)]) >= best[todo])
        right_ok = (hi == n) | (np.abs(br[np.minimum(hi, n - 1)] - a.real[todo]) >= best[todo])
        todo = todo[~(left_ok & right_ok)]
        width *= 4
    counts = np.bincount(perm, minlength=n)
    assert np.all(counts == 1), "nearest-neighbour pairing is not a bijection (%d collisions)" % int(
        np.sum(counts > 1))
    return perm, float(best.max())


def match_sorted(a: np.ndarray, b: np.ndarray, tol: float) -> tuple[float, int]:
    """Compare two root sets of equal size: sort both by (Re, Im), compare
    entry by entry, and re-pair by nearest neighbour only the entries whose
    order differs (near-equal real parts).  Returns (max distance, number of
    re-paired entries)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    assert a.shape == b.shape, (a.shape, b.shape)
    sa = a[np.lexsort((a.imag, a.real))]
    sb = b[np.lexsort((b.imag, b.real))]
    d = np.abs(sa - sb)
    bad = d > tol
    if not bad.any():
        return float(d.max()) if d.size else 0.0, 0
    # pair the mismatched entries of both sides among themselves
    _, dm = match_sets(sa[bad], sb[bad])
    return max(float(d[~bad].max()) if (~bad).any() else 0.0, dm), int(bad.sum())


def lexsorted(z: np.ndarray, zl: np.ndarray | None = None) -> bool:
    """True if z is sorted by (Re, Im) (eq. defLexi).  With low parts zl
    (double-double values z + zl, normalised pairs) the order is that of the
    values: equal hi parts are ordered by their low parts."""
    z = np.asarray(z)
    if z.size < 2:
        return True
    r0, r1 = z.real[:-1], z.real[1:]
    i0, i1 = z.imag[:-1], z.imag[1:]
    if zl is None:
        return bool(np.all((r0 < r1) | ((r0 == r1) & (i0 <= i1))))
    zl = np.asarray(zl)
    rl0, rl1 = zl.real[:-1], zl.real[1:]
    il0, il1 = zl.imag[:-1], zl.imag[1:]
    re_lt = (r0 < r1) | ((r0 == r1) & (rl0 < rl1))
    re_eq = (r0 == r1) & (rl0 == rl1)
    im_le = (i0 < i1) | ((i0 == i1) & (il0 <= il1))
    return bool(np.all(re_lt | (re_eq & im_le)))


def min_separation(z: np.ndarray) -> float:
    """Smallest pairwise distance (sort + window; exact)."""
    z = np.asarray(z, dtype=np.complex128)
    if z.size < 2:
        return float("inf")
    o = np.argsort(z.real)
    zs = z[o]
    best = np.inf
    w = 1
    while True:
        d = np.abs(zs[w:] - zs[:-w])
        best = min(best, float(d.min())) if d.size else best
        gap = zs.real[w:] - zs.real[:-w]
        if gap.size == 0 or gap.min() >= best:
            return best
        w += 1
