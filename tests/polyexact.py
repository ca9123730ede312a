"""Exact integer coefficients of p_n and s_{l,n}, written straight from their
definitions (eq. def:hyp_poly and eq. polySimple), for brute-force checks of
small cases with an independent root finder (mpmath's polyroots) and exact
real-root counts (sympy's Sturm sequences).  Test-only helper."""
from __future__ import annotations


def _square_plus_z(p: list[int]) -> list[int]:
    sq = [0] * (2 * len(p) - 1)
    for i, a in enumerate(p):
        if a:
            for j, b in enumerate(p):
                sq[i + j] += a * b
    if len(sq) < 2:
        sq += [0] * (2 - len(sq))
    sq[1] += 1
    while len(sq) > 1 and sq[-1] == 0:
        sq.pop()
    return sq


def p_coeffs(n: int) -> list[int]:
    """p_n in ascending powers: p_0 = 0, p_{k+1} = p_k^2 + z."""
    p = [0]
    for _ in range(n):
        p = _square_plus_z(p)
    return p


def s_coeffs(l: int, n: int) -> list[int]:
    """s_{l,n} = p_{l+n-1} + p_{l-1} in ascending powers."""
    a = p_coeffs(l + n - 1)
    b = p_coeffs(l - 1)
    out = a[:] + [0] * max(0, len(b) - len(a))
    for i, c in enumerate(b):
        out[i] += c
    return out


def eval_int_poly(coeffs: list[int], z):
    acc = 0
    for c in reversed(coeffs):
        acc = acc * z + c
    return acc
