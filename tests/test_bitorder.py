"""The integer-order facts the device code relies on (CPU, no GPU).

The Newton kernels compare non-negative binary64 values through their bit
patterns read as signed 64-bit integers (ord_f64 in csrc/mt_common.cuh) and
carry the c-derivative scaled by powers of two.  These tests check, with
numpy on the host, the identities those shortcuts need, and that the
constants written in the header are the bit patterns they name."""
from __future__ import annotations

import os
import re
import struct

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2402_06083_gb300", "csrc", "mt_common.cuh")


def ord64(x):
    return np.asarray(x, dtype=np.float64).view(np.int64)


def header_constant(name: str) -> int:
    text = open(HEADER).read()
    m = re.search(r"constexpr long long %s = (0x[0-9a-fA-F]+|[0-9]+ll << [0-9]+|[0-9a-fx]+)" % name, text)
    assert m, name
    expr = m.group(1).replace("ll", "")
    return int(eval(expr, {}))  # a literal or a shift of literals


def test_header_constants_are_the_named_bit_patterns():
    assert header_constant("ORD_1E290") == struct.unpack("<q", struct.pack("<d", 1e290))[0]
    assert header_constant("ORD_1EM290") == struct.unpack("<q", struct.pack("<d", 1e-290))[0]
    assert header_constant("ORD_QUARTER") == 2 << 52


def _nonneg(rng, n):
    e = rng.uniform(-1074, 1023, n)
    x = 2.0 ** e * rng.uniform(1, 2, n)
    return np.concatenate([x, [0.0, np.inf, 5e-324, 2.2250738585072014e-308,
                               1.7976931348623157e308, 1e-26, 1e-300, 1e300]])


def test_nonnegative_values_order_as_their_bit_patterns():
    rng = np.random.default_rng(1)
    x = _nonneg(rng, 200_000)
    y = rng.permutation(x)
    assert np.array_equal(x < y, ord64(x) < ord64(y))
    assert np.array_equal(x <= y, ord64(x) <= ord64(y))
    assert np.array_equal(x == y, ord64(x) == ord64(y))


def test_quarter_by_bit_pattern_for_normal_prev():
    """s2 >= prev2 / 4  <=>  ord(s2) >= ord(prev2) - ORD_QUARTER, for prev2 >= 1e-300
    (the descent clamps tol2 there and prev2 never falls below tol2)."""
    rng = np.random.default_rng(2)
    x = _nonneg(rng, 200_000)
    s2 = x[x >= 1e-300]
    p2 = rng.permutation(s2)
    # plus pairs within an ulp of the boundary prev2 = 4 s2
    near = s2[s2 < 4e307] * 4
    near = near * (1 + rng.choice([-1.0, 0.0, 1.0], near.size) * 2.0 ** -52)
    s2 = np.concatenate([s2, s2[s2 < 4e307][: near.size]])
    p2 = np.concatenate([p2, near])
    q = 2 << 52
    assert np.array_equal(s2 >= 0.25 * p2, ord64(s2) >= ord64(p2) - q)


def test_division_range_guard_by_bit_pattern():
    """The quotient's guard !(1e-290 <= den <= 1e290) for den in [+0, +inf] or NaN of
    either sign gives the same answer on bit patterns."""
    rng = np.random.default_rng(3)
    den = np.concatenate([_nonneg(rng, 100_000), [np.nan, -np.nan]])
    lo = struct.unpack("<q", struct.pack("<d", 1e-290))[0]
    hi = struct.unpack("<q", struct.pack("<d", 1e290))[0]
    with np.errstate(invalid="ignore"):
        ref = ~((den <= 1e290) & (den >= 1e-290))
    got = ~((ord64(den) <= hi) & (ord64(den) >= lo))
    assert np.array_equal(ref, got)


def test_finite_by_exponent_field():
    rng = np.random.default_rng(4)
    x = _nonneg(rng, 50_000)
    z = np.concatenate([x, -x, [np.nan, -np.nan, -np.inf]])
    hiword = (ord64(z) >> 32) & 0xFFFFFFFF
    assert np.array_equal(np.isfinite(z), (hiword & 0x7FF00000) != 0x7FF00000)


def test_scaled_derivative_recurrence_matches_plain_one_bit_for_bit():
    """e_k = p'_k / 2^k, e_k = p_{k-1} e_{k-1} + 2^-k, reproduces the binary64 p'_m of
    p'_k = 2 p_{k-1} p'_{k-1} + 1 exactly (each rounding scales by a power of two).
    numpy has no fused multiply-add, so both sides use separate products here; the
    scaling argument is the same."""
    rng = np.random.default_rng(5)
    c = rng.uniform(-2, 0.5, 4000) + 1j * rng.uniform(-1.2, 1.2, 4000)
    cr, ci = c.real.copy(), c.imag.copy()
    m = 20
    zr = np.zeros_like(cr); zi = np.zeros_like(cr)
    dr = np.zeros_like(cr); di = np.zeros_like(cr)
    er = np.zeros_like(cr); ei = np.zeros_like(cr)
    with np.errstate(all="ignore"):
        for k in range(1, m + 1):
            tzr, tzi = zr + zr, zi + zi
            ndr = tzr * dr - tzi * di + 1.0
            ndi = tzr * di + tzi * dr
            h = 2.0 ** -k
            ner = zr * er - zi * ei + h
            nei = zr * ei + zi * er
            nzr = zr * zr - zi * zi + cr
            nzi = tzr * zi + ci
            zr, zi, dr, di, er, ei = nzr, nzi, ndr, ndi, ner, nei
        ok = np.isfinite(dr) & np.isfinite(di) & (np.abs(dr) < 1e300) & (np.abs(di) < 1e300)
    assert ok.sum() > 1000
    s = 2.0 ** m
    assert np.array_equal(er[ok] * s, dr[ok])
    assert np.array_equal(ei[ok] * s, di[ok])


def _twice_bits(x: np.ndarray) -> np.ndarray:
    """The integer-pipe doubling of twice_f64 (csrc/mt_common.cuh), restated
    on the two 32-bit halves with numpy."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    lo = (b & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    e = (hi >> np.uint32(20)) & np.uint32(0x7FF)
    sgn = hi & np.uint32(0x80000000)
    rh = hi + np.uint32(0x00100000)
    rl = lo.copy()
    z = e == 0
    rh[z] = sgn[z] | ((hi[z] << np.uint32(1)) & np.uint32(0x7FFFFFFF)) | (lo[z] >> np.uint32(31))
    rl[z] = lo[z] << np.uint32(1)
    o = e == 0x7FE
    rh[o] = sgn[o] | np.uint32(0x7FF00000)
    rl[o] = 0
    f = e == 0x7FF
    rh[f] = hi[f]
    return ((rh.astype(np.uint64) << np.uint64(32)) | rl.astype(np.uint64)).view(np.float64)


def test_twice_by_exponent_is_x_plus_x():
    """twice_f64 doubles on the integer pipe; it must equal x + x bit for bit
    for every finite and infinite binary64: normal, subnormal (becoming
    normal), zero of both signs, and overflow to inf."""
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2 ** 63, 2_000_000, dtype=np.int64).view(np.uint64)
    bits[::2] |= np.uint64(1) << np.uint64(63)
    x = bits.view(np.float64)
    x = x[~np.isnan(x)]
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308,
                        8.98846567431158e307, -8.98846567431158e307, 1.7976931348623157e308, np.inf, -np.inf,
                        1.0, -3.0, 1e-310])
    x = np.concatenate([x, special])
    with np.errstate(over="ignore"):
        want = x + x
    assert np.array_equal(_twice_bits(x).view(np.uint64), want.view(np.uint64))
