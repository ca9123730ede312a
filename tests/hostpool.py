"""Binary128 checks of large GPU root lists on the host cores (test-only).

The oracle's Newton polish (3 binary128 steps, ``oracle.polish_many``) run
in one spawned process per host core: spawn, since the test process has
initialised CUDA and a forked child of it would hang.  No method arithmetic
here: chunking and result gathering only."""
from __future__ import annotations

import os

import numpy as np

_POOL = None


def cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def pool():
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        _POOL = mp.get_context("spawn").Pool(cores())
    return _POOL


def _polish(args):
    import oracle
    kind, l, n, z, zl, steps = args
    return oracle.polish_many(kind, n, z, l=l, roots_lo=zl, steps=steps, want_points=True)


def polish_all(kind: str, n: int, z, l: int = 0, zl=None, chunk: int = 0, steps: int = 4):
    """(disp, last, points4) for every point of z (+ low parts zl), each
    polished by 'steps' binary128 Newton steps (4: at the left tip of p_24,
    where roots lie 4.2e-13 apart, a binary64 root's third step is still
    ~1e-24)."""
    z = np.asarray(z, dtype=np.complex128).ravel()
    zl = None if zl is None else np.asarray(zl, dtype=np.complex128).ravel()
    if chunk <= 0:  # about four chunks per host core
        chunk = max(256, -(-z.size // (4 * cores())))
    parts = [(kind, l, n, z[a:a + chunk], None if zl is None else zl[a:a + chunk], steps)
             for a in range(0, z.size, chunk)]
    if not parts:
        return np.zeros(0), np.zeros(0), np.zeros((0, 4))
    res = pool().map(_polish, parts, chunksize=1)
    return (np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res]),
            np.concatenate([r[2] for r in res]))


def dd_sub(a4: np.ndarray, b4: np.ndarray) -> np.ndarray:
    """|a - b| for points given as (Re hi, Re lo, Im hi, Im lo), the parts
    subtracted separately so that differences below binary64 survive."""
    dre = (a4[:, 0] - b4[:, 0]) + (a4[:, 1] - b4[:, 1])
    dim = (a4[:, 2] - b4[:, 2]) + (a4[:, 3] - b4[:, 3])
    return np.hypot(dre, dim)


def min_gap(points4: np.ndarray) -> float:
    """Smallest distance between two of the points (4-vectors): nearest
    neighbours on the binary64 parts by a k-d tree, and exact ties of the
    binary64 parts measured on their low parts."""
    from scipy.spatial import cKDTree
    if points4.shape[0] < 2:
        return float("inf")
    xy = np.stack([points4[:, 0], points4[:, 2]], axis=1)
    d, j = cKDTree(xy).query(xy, k=2)
    gap = d[:, 1].copy()
    tie = gap == 0
    if tie.any():
        gap[tie] = dd_sub(points4[tie], points4[j[tie, 1]])
    return float(gap.min())


def _window(args):
    import oracle
    n, a, b = args
    return oracle.split_window(n, a, b, fp64=True, want_roots=True)["roots4"]


def oracle_windows(n: int, pieces: int):
    """The binary64 oracle's split of p_n as windows tiling the upper half of
    its level line (each walked from its lifted seed, with its descents and
    root set), one window per task on the host pool; the upper-half roots of
    all windows (a root found from two windows appears twice)."""
    J = 8 * 2 ** (n - 1) // 2
    cuts = [J * k // pieces // 8 * 8 for k in range(pieces)] + [J]
    res = pool().map(_window, [(n, a, b) for a, b in zip(cuts, cuts[1:])], chunksize=1)
    return np.concatenate(res)
