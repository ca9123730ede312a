"""Pins of the oracle's separation statistics (Sec. 6.3.2) to facts that do
not come from the oracle itself: closed forms on lattices, the bin edges of
Fig. separationHistogram, double-double digits below one ulp, and the
paper's law on the oracle's own roots of p_9 .. p_12 -- the minimal distance
within Hyp(n) is 118.4 / 4^n to 0.1 % for n >= 9, attained by the two
left-most real roots, and for even n the roots of p_n get closer still
through a centre of period n/2 next to a satellite of period n.

Each pin fails on a plausible slip: counting the root itself (all 0),
ignoring the mask (h instead of h sqrt 2), dropping the low parts (0
instead of 1e-20), a bin edge on the wrong side, or a transposed min axis
(the row count differs from the column count in every case)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import goldens

SEP = goldens.table("separation_law.txt")  # Sec. 6.3.2


def _lattice(nx, ny, h, rng):
    g = (np.arange(nx)[:, None] * h + 1j * np.arange(ny)[None, :] * h).ravel() - 1.0
    p = rng.permutation(g.size)
    return g[p], p


def test_lattice_spacing_is_every_distance():
    rng = np.random.default_rng(1)
    z, _ = _lattice(7, 9, 0.125, rng)
    nn = oracle.nearest_neighbours(z)
    assert np.all(nn == 0.125)  # multiples of a power of two: exact


def test_checkerboard_mask_gives_the_diagonal():
    rng = np.random.default_rng(2)
    nx, ny, h = 6, 11, 0.125
    z, p = _lattice(nx, ny, h, rng)
    i, j = np.divmod(p, ny)
    mask = ((i + j) % 2 == 0).astype(np.uint8)
    nn = oracle.nearest_neighbours(z, mask)
    assert np.all(nn[mask == 1] == np.hypot(h, h)) and np.all(nn[mask == 0] == 0)
    # the same rows asked one by one (idx) give the same values
    k = np.nonzero(mask)[0][:5]
    assert np.array_equal(oracle.nearest_neighbours(z, mask, idx=k), nn[k])


def test_alone_pair_and_duplicates():
    assert oracle.nearest_neighbours(np.array([0.3 + 0.1j]))[0] == np.inf
    nn = oracle.nearest_neighbours(np.array([-1.0, 0.25 + 0.5j]))
    assert np.all(nn == abs(1.25 + 0.5j))
    assert list(oracle.nearest_neighbours(np.array([-1.0, 0.0, -1.0]))) == [0.0, 1.0, 0.0]


def test_low_parts_resolve_below_one_ulp():
    """Two double-double roots with equal hi parts 1e-20 apart (lo parts):
    binary64 sees a duplicate, double-double the true gap."""
    z = np.array([-1.9 + 0.2j, -1.9 + 0.2j, -1.0 + 0.0j])
    lo = np.array([0.0, 1e-20, 0.0])
    nn = oracle.nearest_neighbours(z, z_lo=lo)
    assert nn[0] == nn[1] == 1e-20 and nn[2] == np.hypot(-1.0 - -1.9, 0.0 - 0.2)
    assert oracle.nearest_neighbours(z)[0] == 0.0


def test_bins_of_the_histogram():
    """I_k = (-2 + 4^-(k+1), -2 + 4^-k]: closed on the right."""
    b = oracle.separation_band
    assert b(-2 + 1.0) == 0 and b(0.25) == 0 and b(-2 + 0.3) == 0
    assert b(-2 + 0.25) == 1 and b(-2 + 0.25 + 1e-12) == 0
    assert b(-2 + 4.0 ** -5) == 5 and b(-2 + 4.0 ** -5 * 1.0000001) == 4
    assert b(-2.0) == 63 and b(-2 + 4.0 ** -70) == 63
    z = np.array([-2 + 0.25, -2 + 0.2, 0.1, -2 + 4.0 ** -3])
    bands = oracle.separation_bands(z, np.array([1.0, 2.0, 3.0, 4.0]))
    assert bands[0] == 3.0 and bands[1] == 1.0 and bands[3] == 4.0 and bands[2] == np.inf


@pytest.mark.parametrize("n", [9, 10, 11, 12])
def test_separation_law_on_oracle_roots(n):
    ref = oracle.split("hyp", n)
    z = ref["roots"]
    per = ref["type"][:, 1]
    hyp = per == n
    nn = oracle.nearest_neighbours(z, hyp)
    mn = nn[hyp].min()
    assert abs(mn * 4.0 ** n / SEP["hyp_constant"] - 1) < SEP["hyp_rel_error"], mn * 4.0 ** n  # n >= 9
    # attained by the two left-most real roots
    order = np.lexsort((z.imag, z.real))
    a, b = order[0], order[1]
    assert z[a].imag == 0 and z[b].imag == 0 and nn[a] == nn[b] == mn
    nn_all = oracle.nearest_neighbours(z)
    if n % 2:
        assert nn_all.min() == mn
    else:  # a centre of period n/2 next to a satellite of period n
        i = int(np.argmin(nn_all))
        d = np.abs(z - z[i])
        d[i] = np.inf
        j = int(np.argmin(d))
        assert nn_all.min() < 0.6 * mn and sorted((per[i], per[j])) == [n // 2, n]
