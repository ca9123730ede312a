"""ORACLE -- test infrastructure only.  Closed-form counts from the paper.

* Thm countingHyp (eq. HypCount):   |Hyp(n)| = sum_{k | n} mu(n/k) 2^(k-1)
* eq. MisCount:                      |Mis(l,n)| = Phi(l,n) |Hyp(n)|
  with Phi(l,n) = 1 (l = 0), 2^(l-1) - 1 (l != 0 and n | l-1), 2^(l-1) otherwise
* eq. polyMisSimple: the roots of s_{l,n} are Hyp(k) for k | gcd(n, l-1) and
  Mis(l,k) for k | n, all simple; deg s_{l,n} = 2^(l+n-2).
* Thm fact_mis: q_{l,n} = prod_{k|n} h_k^eta_l(k) prod_{j=2..l} m_{j,k},
  eta_l(k) = floor((l-1)/k) + 2; deg q_{l,n} = 2^(l+n-1).
"""
from __future__ import annotations

import math


def divisors(n: int) -> list[int]:
    return [k for k in range(1, n + 1) if n % k == 0]


def mobius(n: int) -> int:
    """Moebius function (Thm countingHyp)."""
    if n < 1:
        raise ValueError(n)
    res, m, p = 1, n, 2
    while p * p <= m:
        if m % p == 0:
            m //= p
            if m % p == 0:
                return 0
            res = -res
        p += 1
    if m > 1:
        res = -res
    return res


def hyp_count(n: int) -> int:
    """|Hyp(n)|, eq. HypCount."""
    return sum(mobius(n // k) * 2 ** (k - 1) for k in divisors(n))


def phi(l: int, n: int) -> int:
    """Phi(l, n) of eq. MisCount."""
    if l == 0:
        return 1
    if (l - 1) % n == 0:
        return 2 ** (l - 1) - 1
    return 2 ** (l - 1)


def mis_count(l: int, n: int) -> int:
    """|Mis(l, n)|, eq. MisCount."""
    return phi(l, n) * hyp_count(n)


def deg_p(n: int) -> int:
    return 2 ** (n - 1)


def deg_s(l: int, n: int) -> int:
    """deg s_{l,n} = deg p_{l+n-1} = 2^(l+n-2)."""
    return 2 ** (l + n - 2)


def period_histogram(n: int) -> dict[int, int]:
    """Exact-period counts of the roots of p_n (eq. HypFactor: p_n = prod_{k|n} h_k)."""
    return {k: hyp_count(k) for k in divisors(n)}


def type_histogram_s(l: int, n: int) -> dict[tuple[int, int], int]:
    """Root types of s_{l,n} (eq. polyMisSimple): (0, k) for Hyp(k), (l, k) for Mis(l, k)."""
    h: dict[tuple[int, int], int] = {}
    for k in divisors(math.gcd(n, l - 1)):
        h[(0, k)] = hyp_count(k)
    for k in divisors(n):
        h[(l, k)] = mis_count(l, k)
    return h


def deg_q(l: int, n: int) -> int:
    """deg q_{l,n} = deg p_{l+n} = 2^(l+n-1)."""
    return 2 ** (l + n - 1)


def eta(l: int, k: int) -> int:
    """Multiplicity of Hyp(k) in q_{l,n}, k | n (Thm fact_mis, eq. defMultHyp)."""
    return (l - 1) // k + 2


def type_histogram_q(l: int, n: int) -> dict[tuple[int, int], int]:
    """Distinct roots of q_{l,n} by type (Thm fact_mis): (0, k) for Hyp(k),
    k | n, and (j, k) for Mis(j, k), 2 <= j <= l, k | n."""
    h: dict[tuple[int, int], int] = {}
    for k in divisors(n):
        h[(0, k)] = hyp_count(k)
        for j in range(2, l + 1):
            h[(j, k)] = mis_count(j, k)
    return h


def misiurewicz_pairs(max_order: int) -> list[tuple[int, int]]:
    """All (l, n) with l >= 2, n >= 1, l + n <= max_order."""
    return [(l, n) for l in range(2, max_order) for n in range(1, max_order - l + 1)]


def eps_dup_default(kind: str, n: int, l: int = 0, bits: int = 53) -> float:
    """Separation parameter of the root set (Chebyshev pixel half-side).

    Hyperbolic: min(1e-9, 0.05 * 118.4 / 4^n) -- a twentieth of the minimal
    separation law of Sec. 6.3.2 -- and at least 64 ulp(2) of the working
    precision.  Misiurewicz family: the paper gives no law; the left-tip
    separations of s_{l,n} measured with this oracle fall like ~6.4e3 / 8^(l+n)
    (consistent with the 4.86e-20 the paper reports at order 26), so the rule
    is min(1e-9, 128 / 8^(l+n)), a fiftieth of that."""
    ulp2 = 2.0 ** (2 - bits)
    if kind == "hyp":
        e = min(1e-9, 0.05 * 118.4 / 4.0 ** n)
    else:
        e = min(1e-9, 128.0 / 8.0 ** (l + n))
    return max(e, 64 * ulp2)
