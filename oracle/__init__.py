"""ORACLE -- test infrastructure only.

A plain, slow CPU implementation of the level-line Newton splitting of the
hyperbolic polynomials p_n and the simplified Misiurewicz polynomials
s_{l,n} = p_{l+n-1} + p_{l-1} (Mihalache & Vigneron, arXiv 2402.06083,
Sec. 4 and Sec. 6.3), plus the closed-form counts the paper gives and the separation statistics
of a root list (Sec. 6.3.2, by their definition, in numpy).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library under ``paper_2402_06083_gb300/`` and never imports it.

The arithmetic lives in ``mt_oracle.c`` (binary128 by default, binary64 for
the timed baseline); this module only loads it with ctypes and wraps the
results in numpy arrays.  ``counts.py`` holds the closed-form counts
(Thm countingHyp, eq. MisCount, eq. MisDeg).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

from . import counts  # noqa: F401  (re-export)
from .counts import (deg_s, divisors, eps_dup_default, hyp_count, mis_count,  # noqa: F401
                     mobius, period_histogram, phi, type_histogram_s)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.c")
_LOCK = threading.Lock()
_LIBS: dict[bool, ctypes.CDLL] = {}


def lib_path(fp64: bool) -> str:
    return os.path.join(_HERE, "_build", "liboracle_%s.so" % ("fp64" if fp64 else "q"))


def build(force: bool = False) -> None:
    """Compile both precisions of the oracle with gcc (no CUDA involved)."""
    os.makedirs(os.path.join(_HERE, "_build"), exist_ok=True)
    for fp64 in (False, True):
        out = lib_path(fp64)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-shared", "-fPIC", "-o", out + ".tmp", _SRC]
        if fp64:
            cmd.insert(1, "-DORACLE_FP64")
        if os.uname().machine in ("x86_64", "i686") and not fp64:
            cmd.append("-lquadmath")
        cmd.append("-lm")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_long) for name in (
        "degree", "n_roots", "n_real", "n_starts", "n_conv", "n_repeat", "n_diverge",
        "n_timeout", "walk_newton", "desc_newton", "walk_fail")] + [
        ("M", ctypes.c_int), ("cL", ctypes.c_int), ("retries", ctypes.c_int),
        ("endpoint_ok", ctypes.c_int), ("n_mult", ctypes.c_long)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def build_mutant(k: int, outdir: str) -> str:
    """Build a copy of the oracle with planted mistake number k (1..12) into
    outdir; used only by the test that shows the pins catch such mistakes."""
    out = os.path.join(outdir, "liboracle_mutant%d.so" % k)
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-DORACLE_MUTANT=%d" % k, "-o", out, _SRC]
    if os.uname().machine in ("x86_64", "i686"):
        cmd.append("-lquadmath")
    cmd.append("-lm")
    subprocess.check_call(cmd)
    return out


def _declare(L: ctypes.CDLL) -> ctypes.CDLL:
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.or_degree.restype = ctypes.c_long
    L.or_degree.argtypes = [ctypes.c_int] * 3
    L.or_eval.restype = ctypes.c_int
    L.or_eval.argtypes = [ctypes.c_int] * 3 + [dp, dp]
    L.or_eval_pk.restype = ctypes.c_int
    L.or_eval_pk.argtypes = [ctypes.c_int, dp, dp]
    L.or_real_endpoint.restype = ctypes.c_int
    L.or_real_endpoint.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, dp]
    L.or_split.restype = ctypes.c_long
    L.or_split.argtypes = ([ctypes.c_int] * 5 + [ctypes.c_double] * 3 + [ctypes.c_int, ctypes.c_double]
                           + [dp, ctypes.c_long, ip, ip, dp, ctypes.c_long, ctypes.POINTER(Stats)])
    L.or_polish.restype = ctypes.c_int
    L.or_polish.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int, dp, dp]
    L.or_polish_many.restype = ctypes.c_long
    L.or_polish_many.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_long, ctypes.c_int, dp, dp, dp]
    L.or_walk.restype = ctypes.c_long
    L.or_walk.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double, dp, ctypes.c_long, ctypes.POINTER(Stats)]
    L.or_lift_seed.restype = ctypes.c_int
    L.or_lift_seed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_int, dp]
    L.or_split_window.restype = ctypes.c_long
    L.or_split_window.argtypes = ([ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [ctypes.c_long] * 2
                                  + [ctypes.c_int, dp, ctypes.c_long, ctypes.POINTER(Stats)])
    L.or_split_q.restype = ctypes.c_long
    L.or_split_q.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 4 + [dp, ctypes.c_double, ctypes.c_int]
                             + [dp, ctypes.c_long, ip, ip, ip, ctypes.POINTER(ctypes.c_long),
                                ctypes.POINTER(Stats)])
    L.or_classify.restype = ctypes.c_int
    L.or_classify.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_double, ip, ip]
    L.or_count_in_disk.restype = ctypes.c_long
    L.or_count_in_disk.argtypes = [dp, ctypes.c_long, dp, ctypes.c_double]
    L.or_precision_bits.restype = ctypes.c_int
    return L


_OVERRIDE: list = []


class use_library:
    """Context manager that routes every call of this module through another
    build of the oracle (a planted-mistake copy in the mutant test)."""

    def __init__(self, path: str):
        self.L = _declare(ctypes.CDLL(path))

    def __enter__(self):
        _OVERRIDE.append(self.L)
        return self

    def __exit__(self, *exc):
        _OVERRIDE.pop()


def _lib(fp64: bool = False) -> ctypes.CDLL:
    if _OVERRIDE:
        return _OVERRIDE[-1]
    with _LOCK:
        if fp64 in _LIBS:
            return _LIBS[fp64]
        build()
        L = ctypes.CDLL(lib_path(fp64))
        _LIBS[fp64] = _declare(L)
        return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c4(c) -> np.ndarray:
    """A point as (Re hi, Re lo, Im hi, Im lo); accepts complex or a 4-vector."""
    if isinstance(c, (complex, float, int, np.complexfloating, np.floating)):
        c = complex(c)
        return np.array([c.real, 0.0, c.imag, 0.0], dtype=np.float64)
    a = np.ascontiguousarray(c, dtype=np.float64)
    assert a.shape == (4,)
    return a


def _kind_args(kind: str, l: int, n: int):
    if kind == "hyp":
        return 0, 0, n
    if kind == "mis":
        return 1, l, n
    if kind == "q":
        return 2, l, n
    raise ValueError(kind)


def degree(kind: str, n: int, l: int = 0) -> int:
    k, ll, nn = _kind_args(kind, l, n)
    return int(_lib().or_degree(k, ll, nn))


def default_lambda0(kind: str) -> float:
    """Outer level: 5 for p_n, 100 for the Misiurewicz family (Sec. 4.2)."""
    return 5.0 if kind == "hyp" else 100.0


def default_IN(kind: str) -> float:
    """Newton cap factor I_N: 1 for p_n, 2.6 for the Misiurewicz family (Sec. 4.2)."""
    return 1.0 if kind == "hyp" else 2.6


def split(kind: str, n: int, l: int = 0, *, M: int = 8, cL: int = 4, lambda0: float | None = None,
          I_N: float | None = None, eps_dup: float | None = None, max_retries: int = 2,
          frac: float = 1.0, fp64: bool = False, want_starts: bool = False,
          want_types: bool = True) -> dict:
    """Split P (p_n for kind 'hyp', s_{l,n} for kind 'mis', q_{l,n} for kind
    'q') with the oracle.

    Returns a dict with 'roots' (complex128, the rounded values), 'roots4'
    ([N, 4] Re hi, Re lo, Im hi, Im lo), 'type' ([N, 2] (preperiod, period)),
    'stats' and optionally 'starts4' (upper-half level-line starts).  For
    q_{l,n} (see split_q) the roots are distinct and 'mult' holds each one's
    multiplicity."""
    if kind == "q":
        if frac < 1.0 or want_starts:
            raise ValueError("q_{l,n}: whole splits only (level_line() gives its starts)")
        return split_q(l, n, M=M, cL=cL, eps_dup=eps_dup, max_retries=max_retries, fp64=fp64)
    k, ll, nn = _kind_args(kind, l, n)
    L = _lib(fp64)
    d = int(L.or_degree(k, ll, nn))
    if d <= 0:
        raise ValueError("bad polynomial")
    lam = default_lambda0(kind) if lambda0 is None else lambda0
    IN = default_IN(kind) if I_N is None else I_N
    eps = eps_dup_default(kind, n, l, bits=53 if fp64 else 113) if eps_dup is None else eps_dup
    cap = d
    roots4 = np.zeros((cap, 4), dtype=np.float64)
    ta = np.zeros(cap, dtype=np.int32)
    tb = np.zeros(cap, dtype=np.int32)
    scap = (cL << max_retries) * d // 2 + 2 if want_starts else 0
    starts4 = np.zeros((max(scap, 1), 4), dtype=np.float64)
    st = Stats()
    nr = L.or_split(k, ll, nn, M, cL, lam, IN, eps, max_retries, frac, _dp(roots4), cap,
                    _ip(ta) if want_types else None, _ip(tb) if want_types else None,
                    _dp(starts4) if want_starts else None, scap, ctypes.byref(st))
    if nr < 0:
        raise RuntimeError("oracle split failed (%d)" % nr)
    m = min(nr, cap)
    out = {
        "roots4": roots4[:m].copy(),
        "roots": roots4[:m, 0] + 1j * roots4[:m, 2],
        "n_roots": int(nr),
        "stats": st.as_dict(),
        "eps_dup": eps,
    }
    if want_types:
        out["type"] = np.stack([ta[:m], tb[:m]], axis=1)
    if want_starts:
        ns = min(int(st.n_starts), scap)
        out["starts4"] = starts4[:ns].copy()
        out["starts"] = starts4[:ns, 0] + 1j * starts4[:ns, 2]
    return out


def split_q(l: int, n: int, *, M: int = 8, cL: int = 4, eps_dup: float | None = None, max_retries: int = 2,
            fp64: bool = False) -> dict:
    """The distinct roots of q_{l,n} = p_{l+n} - p_l with their multiplicities
    and types, from eq. polySimple telescoped: q_{l,n} = p_n^2 prod_{j=2..l}
    s_{j,n} (s_{1,n} = p_n, eq. hypCase).  The factors are split by this
    oracle (p_n and every s_{j,n}, each with its own defaults); their roots
    are merged with the Chebyshev rule at the q_{l,n} separation eps_dup; a
    root's multiplicity is the number of factors it is a root of (p_n
    counted twice) and its type comes from its factor ((0, k) for Hyp(k),
    (j, k) for Mis(j, k)).  Returns the dict of split() with 'mult', and
    'n_conflict' (cluster members whose factor types disagree: 0)."""
    if l < 1 or n < 1 or l + n > 40:
        raise ValueError("bad polynomial")
    L = _lib(fp64)
    bits = 53 if fp64 else 113
    epsf = np.zeros(l, dtype=np.float64)
    epsf[0] = eps_dup_default("hyp", n, bits=bits)
    for j in range(2, l + 1):
        epsf[j - 1] = eps_dup_default("mis", n, j, bits=bits)
    eps = eps_dup_default("q", n, l, bits=bits) if eps_dup is None else eps_dup
    cap = 2 ** (l + n - 1)
    roots4 = np.zeros((cap, 4), dtype=np.float64)
    pre = np.zeros(cap, dtype=np.int32)
    per = np.zeros(cap, dtype=np.int32)
    mult = np.zeros(cap, dtype=np.int32)
    nconf = ctypes.c_long(0)
    st = Stats()
    nr = L.or_split_q(l, n, M, cL, default_lambda0("hyp"), default_lambda0("mis"), default_IN("hyp"),
                      default_IN("mis"), _dp(epsf), eps, max_retries, _dp(roots4), cap, _ip(pre), _ip(per),
                      _ip(mult), ctypes.byref(nconf), ctypes.byref(st))
    if nr < 0:
        raise RuntimeError("oracle split of q failed (%d)" % nr)
    m = min(nr, cap)
    return {
        "roots4": roots4[:m].copy(),
        "roots": roots4[:m, 0] + 1j * roots4[:m, 2],
        "n_roots": int(nr),
        "type": np.stack([pre[:m], per[:m]], axis=1),
        "mult": mult[:m].copy(),
        "n_conflict": int(nconf.value),
        "stats": st.as_dict(),
        "eps_dup": eps,
    }


def level_line(kind: str, n: int, l: int = 0, *, M: int = 8, cL: int = 4, lambda0: float | None = None,
               fp64: bool = False) -> dict:
    """The upper half of the discrete level line |P| = lambda0 walked
    sequentially from the real end point (no descents): 'starts4' / 'starts',
    start s with P = lambda0 e^{i pi s / 2} for c_L = 4 (kinds hyp, mis, q)."""
    k, ll, nn = _kind_args(kind, l, n)
    L = _lib(fp64)
    d = int(L.or_degree(k, ll, nn))
    if d <= 0:
        raise ValueError("bad polynomial")
    lam = default_lambda0(kind) if lambda0 is None else lambda0
    scap = cL * d // 2 + 2
    starts4 = np.zeros((scap, 4), dtype=np.float64)
    st = Stats()
    ns = L.or_walk(k, ll, nn, M, cL, lam, _dp(starts4), scap, ctypes.byref(st))
    if ns < 0:
        raise RuntimeError("oracle walk failed (%d)" % ns)
    ns = min(int(ns), scap)
    return {"starts4": starts4[:ns].copy(), "starts": starts4[:ns, 0] + 1j * starts4[:ns, 2],
            "stats": st.as_dict()}


def lift_seed(n: int, j: int, *, M: int = 8, lambda0: float = 5.0, shrink: int = 16, fp64: bool = False):
    """The point of index j of the level line of p_n (M points per turn),
    lifted through the nested family p_1 -> ... -> p_n (Sec. 4.2).  Returns
    (4-vector, number of solves that did not converge)."""
    out = np.zeros(4, dtype=np.float64)
    f = _lib(fp64).or_lift_seed(n, M, j, lambda0, shrink, _dp(out))
    if f < 0:
        raise ValueError("bad arguments")
    return out, int(f)


def split_window(n: int, jbeg: int, jend: int, *, M: int = 8, cL: int = 4, lambda0: float | None = None,
                 eps_dup: float | None = None, shrink: int = 16, fp64: bool = True,
                 want_roots: bool = False) -> dict:
    """One window of the split of p_n: sub-steps jbeg..jend of the upper half
    (M d / 2 in all, d = 2^(n-1)), walked from the lifted seed of index jbeg,
    with its descents and its own root set.  Returns 'n_roots' (distinct
    upper-half roots of the window), 'stats' and, with want_roots, 'roots4'."""
    L = _lib(fp64)
    lam = default_lambda0("hyp") if lambda0 is None else lambda0
    eps = eps_dup_default("hyp", n, bits=53 if fp64 else 113) if eps_dup is None else eps_dup
    st = Stats()
    cap = (jend - jbeg) // max(1, M // cL) + 2 if want_roots else 0
    r4 = np.zeros((max(cap, 1), 4), dtype=np.float64)
    nr = L.or_split_window(n, M, cL, lam, default_IN("hyp"), eps, jbeg, jend, shrink,
                           _dp(r4) if want_roots else None, cap, ctypes.byref(st))
    if nr < 0:
        raise ValueError("bad window")
    out = {"n_roots": int(nr), "stats": st.as_dict()}
    if want_roots:
        out["roots4"] = r4[:min(int(nr), cap)].copy()
    return out


def polish_many(kind: str, n: int, roots, l: int = 0, steps: int = 3, roots_lo=None, want_points: bool = False):
    """Binary128 Newton polish of every point of a list (or_polish in one C
    loop).  roots: complex array (hi parts), roots_lo: optional low parts.
    Returns (disp, last[, points4]): |polished - given| and the size of the
    last Newton step per point (+inf where the iterate left the finite
    numbers), and the polished points as 4-vectors."""
    k, ll, nn = _kind_args(kind, l, n)
    z = np.asarray(roots, dtype=np.complex128).ravel()
    c4 = np.zeros((z.size, 4), dtype=np.float64)
    c4[:, 0] = z.real
    c4[:, 2] = z.imag
    if roots_lo is not None:
        zl = np.asarray(roots_lo, dtype=np.complex128).ravel()
        c4[:, 1] = zl.real
        c4[:, 3] = zl.imag
    disp = np.zeros(z.size)
    last = np.zeros(z.size)
    out4 = np.zeros((z.size, 4)) if want_points else None
    rc = _lib().or_polish_many(k, ll, nn, _dp(c4), z.size, steps, _dp(out4) if want_points else None,
                               _dp(disp), _dp(last))
    if rc < 0:
        raise ValueError("bad polynomial")
    return (disp, last, out4) if want_points else (disp, last)


def evaluate(kind: str, n: int, c, l: int = 0, fp64: bool = False):
    """(P(c), P'(c)) as 4-vectors (hi/lo of Re and Im) each."""
    k, ll, nn = _kind_args(kind, l, n)
    out = np.zeros(8, dtype=np.float64)
    if _lib(fp64).or_eval(k, ll, nn, _dp(_c4(c)), _dp(out)) != 0:
        raise ValueError("bad polynomial")
    return out[:4].copy(), out[4:].copy()


def evaluate_pk(k: int, c, fp64: bool = False):
    out = np.zeros(8, dtype=np.float64)
    _lib(fp64).or_eval_pk(k, _dp(_c4(c)), _dp(out))
    return out[:4].copy(), out[4:].copy()


def real_endpoint(kind: str, n: int, l: int = 0, lambda0: float | None = None, fp64: bool = False):
    k, ll, nn = _kind_args(kind, l, n)
    out = np.zeros(2, dtype=np.float64)
    lam = default_lambda0(kind) if lambda0 is None else lambda0
    _lib(fp64).or_real_endpoint(k, ll, nn, lam, _dp(out))
    return out


def polish(kind: str, n: int, c, l: int = 0, steps: int = 3):
    """Newton-polish one point in binary128; returns (4-vector, displacement)."""
    k, ll, nn = _kind_args(kind, l, n)
    out = np.zeros(4, dtype=np.float64)
    disp = ctypes.c_double(0)
    rc = _lib().or_polish(k, ll, nn, _dp(_c4(c)), steps, _dp(out), ctypes.byref(disp))
    if rc != 0:
        raise FloatingPointError("polish diverged")
    return out, disp.value


def classify(kind: str, n: int, c, l: int = 0, tau: float = 0.0, fp64: bool = False):
    k, ll, nn = _kind_args(kind, l, n)
    a = ctypes.c_int(0)
    b = ctypes.c_int(0)
    _lib(fp64).or_classify(k, ll, nn, _dp(_c4(c)), tau, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def count_in_disk(roots4: np.ndarray, c, r: float) -> int:
    r4 = np.ascontiguousarray(roots4, dtype=np.float64)
    return int(_lib().or_count_in_disk(_dp(r4), r4.shape[0], _dp(_c4(c)), r))


def precision_bits(fp64: bool = False) -> int:
    return int(_lib(fp64).or_precision_bits())


def join4(a: np.ndarray):
    """4-vectors -> (Re, Im) as pairs of float64 hi + lo (for mpmath use)."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, 4)
    return a[:, 0], a[:, 1], a[:, 2], a[:, 3]


def _two_diff(a, b):
    """a - b = s + e exactly (Knuth's TwoSum applied to a and -b)."""
    s = a - b
    bb = s - a
    e = (a - (s - bb)) + (-b - bb)
    return s, e


def nearest_neighbours(z, mask=None, z_lo=None, idx=None, cells: int = 1 << 23) -> np.ndarray:
    """Separation (Sec. 6.3.2), by its definition.  For root i of the set
    S = {j : mask[j] != 0} (every root if mask is None),
        nn_i = min over j in S, j != i, of |c_j - c_i|,
    a minimum over all other roots of S (no index, no pruning), taken in
    blocks of at most `cells` pairs.  nn_i = +inf if i is alone in S.  With
    z_lo (double-double roots c = z + z_lo) each coordinate difference is
    (z_j - z_i) split exactly by TwoSum, plus (lo_j - lo_i).  Returns nn for
    every root (0 outside S) or, with idx, for the roots idx only."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    lo = None if z_lo is None else np.asarray(z_lo, dtype=np.complex128).ravel()
    sel = np.ones(z.size, bool) if mask is None else (np.asarray(mask).ravel() != 0)
    S = np.nonzero(sel)[0]
    rows = S if idx is None else np.asarray(idx, dtype=np.int64).ravel()
    res = np.zeros(rows.size)
    xs, ys = z.real[S], z.imag[S]
    xls = None if lo is None else lo.real[S]
    yls = None if lo is None else lo.imag[S]
    col = max(1, min(S.size, cells))
    rb = max(1, cells // col)
    for a in range(0, rows.size, rb):
        r = rows[a:a + rb]
        best = np.full(r.size, np.inf)
        for b in range(0, S.size, col):
            dx, ex = _two_diff(xs[None, b:b + col], z.real[r][:, None])
            dy, ey = _two_diff(ys[None, b:b + col], z.imag[r][:, None])
            if lo is not None:
                dx = dx + (ex + (xls[None, b:b + col] - lo.real[r][:, None]))
                dy = dy + (ey + (yls[None, b:b + col] - lo.imag[r][:, None]))
            d = np.hypot(dx, dy)
            d[S[None, b:b + col] == r[:, None]] = np.inf  # not the root itself
            best = np.minimum(best, d.min(axis=1))
        res[a:a + rb] = best
    if idx is not None:
        return np.where(sel[rows], res, 0.0)
    out = np.zeros(z.size)
    out[S] = res
    return out


def separation_band(x: float) -> int:
    """Fig. separationHistogram: the k >= 0 with Re c + 2 in the bin
    I_k = (4^-(k+1), 4^-k]; Re c + 2 > 1 counts in bin 0, Re c + 2 <= 4^-63
    (and c = -2 itself) in bin 63."""
    t = float(x) + 2.0
    for k in range(63):
        if t > 4.0 ** -(k + 1):
            return k
    return 63


def separation_bands(z, nn, mask=None) -> list:
    """Per bin I_k (k = 0..63) the minimal nn over the set's roots in it
    (+inf for an empty bin): the histogram of Fig. separationHistogram."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    sel = np.ones(z.size, bool) if mask is None else (np.asarray(mask).ravel() != 0)
    out = [np.inf] * 64
    for x, d, s in zip(z.real, np.asarray(nn).ravel(), sel):
        if s:
            k = separation_band(x)
            out[k] = min(out[k], float(d))
    return out


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print("oracle built:", lib_path(False), lib_path(True))
