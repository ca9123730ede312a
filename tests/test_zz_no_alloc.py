"""mt_certify_static -- the disk certificate for callers that cannot allocate
device memory (host callbacks, allocator hooks, plug-ins living in another
runtime's memory pool).  It keeps its scratch in a static device array, so
these callers pass only the roots and the output arrays.

Checked through the C ABI against mt_certify (the entry point with a
caller-provided workspace) on two calls in a row with different inputs, so
that state left in the shared static array by the first call would show in
the second.  This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2402_06083_gb300 as mt
    return torch, mt, mt.load()


def _static(torch, L, kind, l, n, roots_ri):
    count = roots_ri.shape[0]
    ok = torch.full((count,), 7, dtype=torch.uint8, device="cuda")
    rad = torch.full((count,), -1.0, dtype=torch.float64, device="cuda")
    npass = ctypes.c_int64(-1)
    rc = L.mt_certify_static(kind, l, n, roots_ri.data_ptr(), count, 0.0, ok.data_ptr(), rad.data_ptr(),
                             ctypes.byref(npass), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, L.mt_last_error()
    return ok, rad, npass.value


def test_certify_static_matches_certify(env):
    torch, mt, L = env
    # call 1: all roots of p_12; call 2: roots of s_{3,6} with every third
    # root moved off by 1e-8 (those must fail in both entry points)
    z1 = oracle.split("hyp", 12, want_types=False)["roots"]
    z2 = oracle.split("mis", 6, l=3, want_types=False)["roots"].copy()
    z2[::3] += 1e-8
    cases = [(0, 0, 12, z1), (1, 3, 6, z2)]
    for kind, l, n, z in cases:
        t = torch.as_tensor(z, device="cuda")
        ri = torch.view_as_real(t).contiguous()
        ok_s, rad_s, np_s = _static(torch, L, kind, l, n, ri)
        ok_w, rad_w, np_w = mt.certify("hyp" if kind == 0 else "mis", n, t, l=l)
        assert np_s == np_w
        assert torch.equal(ok_s, ok_w)
        assert torch.equal(rad_s, rad_w)  # same kernels, same order: bit-identical
        if kind == 0:
            assert np_s == z.size
        else:
            assert np_s == z.size - len(z[::3])


def test_certify_static_rejects_oversized_lists(env):
    torch, mt, L = env
    count = mt._lib.MT_CERTIFY_STATIC_MAX_ROOTS + 1
    npass = ctypes.c_int64(0)
    rc = L.mt_certify_static(0, 0, 20, ctypes.c_void_p(16), count, 0.0, ctypes.c_void_p(16), None,
                             ctypes.byref(npass), None)
    assert rc == mt._lib.MT_ECAPACITY
    assert b"MT_CERTIFY_STATIC_MAX_ROOTS" in L.mt_last_error()


def test_certify_static_at_its_limit(env):
    """Exactly MT_CERTIFY_STATIC_MAX_ROOTS roots -- all 131,072 roots of p_18
    -- where the carve of the static array (counters, keys, permutation,
    radix histograms) is at its largest: bit-identical to mt_certify, twice
    in a row, every root passing."""
    torch, mt, L = env
    n = 18
    count = mt._lib.MT_CERTIFY_STATIC_MAX_ROOTS
    assert 2 ** (n - 1) == count
    roots = mt.split_hyperbolic(n).roots
    ri = torch.view_as_real(roots).contiguous()
    ok_w, rad_w, np_w = mt.certify("hyp", n, roots)
    for _ in range(2):
        ok_s, rad_s, np_s = _static(torch, L, 0, 0, n, ri)
        assert np_s == np_w == count
        assert torch.equal(ok_s, ok_w) and torch.equal(rad_s, rad_w)


def test_certify_static_rejects_q(env):
    """q_{l,n} (kind 2) is certified by mt_certify only."""
    torch, mt, L = env
    npass = ctypes.c_int64(0)
    rc = L.mt_certify_static(2, 3, 4, ctypes.c_void_p(16), 4, 0.0, ctypes.c_void_p(16), None,
                             ctypes.byref(npass), None)
    assert rc == mt._lib.MT_EINVAL
