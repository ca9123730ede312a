"""The C-ABI library loads and exports every symbol include/mtsplit.h
declares (CPU only: no compute call needs a GPU here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mtsplit.h")


def declared_symbols() -> list[str]:
    text = open(HEADER).read()
    return sorted(set(re.findall(r"MT_API\s+[\w\s\*]*?\b(mt_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_06083_gb300 import build as b
    b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_api():
    syms = declared_symbols()
    for name in ("mt_split_hyperbolic", "mt_split_misiurewicz", "mt_split_misiurewicz_batch",
                 "mt_certify", "mt_workspace_bytes", "mt_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_declares_every_exported_symbol():
    from paper_2402_06083_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_symbols()


def test_host_only_entry_points(lib):
    """Entry points that touch no device memory run on the CPU machine too."""
    import paper_2402_06083_gb300 as mt
    L = mt.load()
    assert L.mt_degree_hyperbolic(20) == 2 ** 19
    assert L.mt_degree_hyperbolic(0) == -1 and L.mt_degree_hyperbolic(41) == -1
    assert L.mt_degree_misiurewicz(2, 14) == 2 ** 14
    assert L.mt_degree_misiurewicz(1, 3) == -1
    assert len(mt.misiurewicz_pairs(16)) == 105
    o = mt.options(stream=0)
    assert o.max_retries == 1 and o.prec == 0
    nb = L.mt_workspace_bytes(0, 0, 20, ctypes.byref(o))
    assert nb > 2 ** 19 * 16 * 4
    assert L.mt_workspace_bytes(0, 0, 0, ctypes.byref(o)) == 0  # invalid n
    assert L.mt_workspace_bytes(1, 1, 3, ctypes.byref(o)) == 0  # l < 2
    # q_{l,n} in MT_DD goes through its factors: room for the largest
    # factor's split (s_{l,n} or p_n) and the union list of the distinct roots
    od = mt.options("dd", stream=0)
    nq = L.mt_workspace_bytes(2, 6, 16, ctypes.byref(od))
    assert nq > L.mt_workspace_bytes(1, 6, 16, ctypes.byref(od)) + 2 ** 21 * 16
    assert L.mt_workspace_bytes(2, 30, 11, ctypes.byref(od)) == 0  # l + n <= 40
    assert mt.version().startswith("mtsplit")


def test_invalid_arguments_fail_cleanly(lib):
    """Domain errors are reported before any CUDA call."""
    import paper_2402_06083_gb300 as mt
    L = mt.load()
    o = mt.options(stream=0)
    n_out = ctypes.c_int64(0)
    rc = L.mt_split_hyperbolic(0, ctypes.byref(o), None, None, 0, None, 0, ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_EINVAL and b"out of range" in L.mt_last_error()
    rc = L.mt_split_hyperbolic(12, ctypes.byref(o), None, None, 0, None, 0, ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_ENOMEM  # no workspace
    o.prec = 7
    rc = L.mt_split_hyperbolic(12, ctypes.byref(o), None, None, 0, None, 0, ctypes.byref(n_out), None)
    assert rc == mt._lib.MT_EINVAL


def test_streamed_plans_fit_one_gb300():
    """Host-only planning: from p_32 on the split streams its level line
    (more than 2^31 starts), and p_32 in MT_DD -- workspace plus roots and
    low parts -- fits the GB300's HBM; stream_pieces must be a power of two."""
    from paper_2402_06083_gb300 import _lib
    L = _lib.load()

    def ws(n, prec, pieces=0):
        o = _lib.Options()
        L.mt_default_options(ctypes.byref(o))
        o.prec, o.max_retries, o.stream_pieces = prec, 0, pieces
        return int(L.mt_workspace_bytes(0, 0, n, ctypes.byref(o)))

    d32 = 2 ** 31
    total = ws(32, 2) + 2 * d32 * 16
    assert 0 < total < 250e9, total / 1e9
    assert ws(31, 2) > ws(32, 2) / 2  # p_31 still runs in one pass
    assert ws(20, 0, 4) > 0 and ws(20, 0, 3) == 0


def test_retries_stop_at_the_largest_plan():
    """(M, c_L) double per retry up to M = 64: a larger retry budget sizes the
    workspace for the largest plan instead of making the query fail."""
    from paper_2402_06083_gb300 import _lib
    L = _lib.load()

    def ws(n, prec, retries):
        o = _lib.Options()
        L.mt_default_options(ctypes.byref(o))
        o.prec, o.max_retries = prec, retries
        return int(L.mt_workspace_bytes(0, 0, n, ctypes.byref(o)))

    for prec in (0, 1):
        sizes = [ws(12, prec, r) for r in range(7)]
        assert all(s > 0 for s in sizes)
        assert sizes == sorted(sizes)                # more retries never need less
        assert sizes[3] == sizes[4] == sizes[6]      # M = 8 * 2^3 = 64 is the last plan
