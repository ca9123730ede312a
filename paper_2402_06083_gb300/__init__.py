"""GB300-native level-line Newton splitting of the Mandelbrot polynomials.

Python binding of the C ABI in include/mtsplit.h (libmtsplit.so, built from
csrc/ for sm_103a).  PyTorch supplies device memory and the current stream;
every step of the computation -- level line, Newton descents, root set,
types, certificates -- runs in the library's CUDA kernels.  There is no CPU
fallback: without the built library every call raises.

Polynomials (Mihalache & Vigneron, arXiv 2402.06083):
  p_n      = f_c^n(0),            deg 2^(n-1)        (eq. def:hyp_poly)
  s_{l,n}  = p_{l+n-1} + p_{l-1}, deg 2^(l+n-2)      (eq. polySimple)
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import _lib
from ._lib import MtError, Options, Stats, check, load  # noqa: F401

KIND = {"hyp": 0, "mis": 1, "q": 2}


def _torch():
    import torch  # deferred: importing the package does not need a GPU
    return torch


def options(prec: str = "fp64", stream=None, **kw) -> Options:
    """An mt_options struct with library defaults, overridden by kw."""
    L = load()
    o = Options()
    L.mt_default_options(ctypes.byref(o))
    o.prec = _lib.PREC[prec] if isinstance(prec, str) else int(prec)
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError("unknown option %s" % k)
        setattr(o, k, v)
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
    o.stream = stream
    return o


def degree(kind: str, n: int, l: int = 0) -> int:
    L = load()
    if kind == "q":  # deg q_{l,n} = deg p_{l+n}
        d = L.mt_degree_hyperbolic(l + n) if l >= 1 else -1
    else:
        d = L.mt_degree_hyperbolic(n) if kind == "hyp" else L.mt_degree_misiurewicz(l, n)
    if d < 0:
        raise ValueError("polynomial out of range")
    return int(d)


def workspace_bytes(kind: str, n: int, l: int = 0, opts: Options | None = None) -> int:
    o = opts if opts is not None else options(stream=0)
    return int(load().mt_workspace_bytes(KIND[kind], l, n, ctypes.byref(o)))


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


@dataclass
class SplitResult:
    roots: "object"          # complex128 tensor [n_roots] on the device, sorted by (Re, Im)
    roots_lo: "object"       # low parts (double-double) or None
    is_mis: "object"         # uint8 tensor (Misiurewicz) or None
    stats: dict
    status: int


class Workspace:
    """A reusable device scratch buffer (torch uint8 tensor)."""

    def __init__(self, nbytes: int = 0, device="cuda"):
        self.device = device
        self.buf = None
        self.ensure(nbytes)

    def ensure(self, nbytes: int):
        torch = _torch()
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


def split_hyperbolic(n: int, prec: str = "fp64", *, work: Workspace | None = None, want_lo: bool = False,
                     check_status: bool = True, out=None, out_lo=None, **kw) -> SplitResult:
    """All 2^(n-1) roots of p_n (Algorithm S_par, Sec. 4.2).  out / out_lo:
    optional float64 [deg, 2] device buffers for the roots and low parts."""
    return _split("hyp", n, 0, prec, work, want_lo, check_status, out, out_lo, kw)


def split_misiurewicz(l: int, n: int, prec: str = "fp64", *, work: Workspace | None = None,
                      want_lo: bool = False, check_status: bool = True, out=None, out_lo=None,
                      **kw) -> SplitResult:
    """All 2^(l+n-2) roots of s_{l,n}, with the Mis(l,n) mask (eq. def:mis)."""
    return _split("mis", n, l, prec, work, want_lo, check_status, out, out_lo, kw)


@dataclass
class SplitResultQ:
    roots: "object"   # complex128 tensor [n_roots]: the distinct roots, sorted by (Re, Im)
    mult: "object"    # uint8 tensor: multiplicity in q_{l,n} (Thm fact_mis)
    pre: "object"     # uint8 tensor: preperiod j (0 for a hyperbolic centre)
    per: "object"     # uint8 tensor: period k
    stats: dict
    status: int


def split_misiurewicz_q(l: int, n: int, prec: str = "fp64", *, work: Workspace | None = None,
                        check_status: bool = True, **kw) -> SplitResultQ:
    """The distinct roots of q_{l,n} = p_{l+n} - p_l with their multiplicities
    and types (Thm fact_mis), mt_split_misiurewicz_q: "fp64" descends on q
    in binary64, "dd" splits its factors p_n, s_{j,n} (eq. polySimple) in
    double-double."""
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    d = degree("q", n, l)
    nbytes = int(L.mt_workspace_bytes(2, l, n, ctypes.byref(o)))
    if nbytes == 0:
        raise ValueError("invalid options for this polynomial")
    work = work or Workspace()
    buf = work.ensure(nbytes)
    roots = torch.empty((d, 2), dtype=torch.float64, device="cuda")
    mult = torch.empty(d, dtype=torch.uint8, device="cuda")
    pre = torch.empty(d, dtype=torch.uint8, device="cuda")
    per = torch.empty(d, dtype=torch.uint8, device="cuda")
    n_out = ctypes.c_int64(0)
    st = Stats()
    rc = L.mt_split_misiurewicz_q(l, n, ctypes.byref(o), roots.data_ptr(), d, mult.data_ptr(), pre.data_ptr(),
                                  per.data_ptr(), buf.data_ptr(), buf.numel(), ctypes.byref(n_out),
                                  ctypes.byref(st))
    if check_status:
        check(rc)
    torch.cuda.current_stream().synchronize()
    m = min(int(n_out.value), d)
    return SplitResultQ(torch.view_as_complex(roots[:m]), mult[:m], pre[:m], per[:m], st.as_dict(), rc)


def _split(kind, n, l, prec, work, want_lo, check_status, out, out_lo, kw) -> SplitResult:
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    d = degree(kind, n, l)
    nbytes = int(L.mt_workspace_bytes(KIND[kind], l, n, ctypes.byref(o)))
    if nbytes == 0:
        raise ValueError("invalid options for this polynomial")
    work = work or Workspace()
    buf = work.ensure(nbytes)
    roots = out if out is not None else torch.empty((d, 2), dtype=torch.float64, device="cuda")
    lo = out_lo if out_lo is not None else (
        torch.empty((d, 2), dtype=torch.float64, device="cuda") if want_lo else None)
    mis = torch.empty(d, dtype=torch.uint8, device="cuda") if kind == "mis" else None
    n_out = ctypes.c_int64(0)
    st = Stats()
    if kind == "hyp":
        rc = L.mt_split_hyperbolic(n, ctypes.byref(o), roots.data_ptr(), _ptr(lo), d, buf.data_ptr(),
                                   buf.numel(), ctypes.byref(n_out), ctypes.byref(st))
    else:
        rc = L.mt_split_misiurewicz(l, n, ctypes.byref(o), roots.data_ptr(), _ptr(lo), d, _ptr(mis),
                                    buf.data_ptr(), buf.numel(), ctypes.byref(n_out), ctypes.byref(st))
    if check_status:
        check(rc)
    m = min(int(n_out.value), d)
    r = torch.view_as_complex(roots[:m])
    return SplitResult(r, None if lo is None else torch.view_as_complex(lo[:m]),
                       None if mis is None else mis[:m], st.as_dict(), rc)


def misiurewicz_pairs(max_order: int) -> list[tuple[int, int]]:
    L = load()
    k = L.mt_misiurewicz_pairs(max_order, None, None, 0)
    ls = (ctypes.c_int * k)()
    ns = (ctypes.c_int * k)()
    L.mt_misiurewicz_pairs(max_order, ls, ns, k)
    return list(zip(ls, ns))


def split_misiurewicz_batch(max_order: int, prec: str = "fp64", *, work: Workspace | None = None,
                            check_status: bool = True, **kw):
    """Every s_{l,n} with l >= 2, n >= 1, l + n <= max_order in one call.
    Returns (roots complex128 [total], is_mis uint8 [total], offsets list, per-pair stats)."""
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    pairs = misiurewicz_pairs(max_order)
    total = sum(2 ** (l + n - 2) for l, n in pairs)
    nbytes = int(L.mt_workspace_bytes_misiurewicz_batch(max_order, ctypes.byref(o)))
    work = work or Workspace()
    buf = work.ensure(nbytes)
    roots = torch.empty((total, 2), dtype=torch.float64, device="cuda")
    mis = torch.empty(total, dtype=torch.uint8, device="cuda")
    offs = (ctypes.c_int64 * (len(pairs) + 1))()
    st = (Stats * len(pairs))()
    rc = L.mt_split_misiurewicz_batch(max_order, ctypes.byref(o), roots.data_ptr(), None, total,
                                      mis.data_ptr(), buf.data_ptr(), buf.numel(), offs, st)
    if check_status:
        check(rc)
    return torch.view_as_complex(roots), mis, list(offs), [s.as_dict() for s in st], pairs


def certify(kind: str, n: int, roots, l: int = 0, tol: float = 0.0, *, work: Workspace | None = None,
            roots_lo=None):
    """Disk certificate (Thm proofRoots) of each root of a complex128 tensor
    (roots_lo: low parts of double-double roots, certified in double-double).
    Returns (pass uint8 tensor, radius float64 tensor, n_pass)."""
    torch = _torch()
    L = load()
    r = torch.view_as_real(roots.contiguous()) if roots.is_complex() else roots.contiguous()
    rl = None
    if roots_lo is not None:
        rl = torch.view_as_real(roots_lo.contiguous()) if roots_lo.is_complex() else roots_lo.contiguous()
    count = r.shape[0]
    nbytes = int(L.mt_certify_workspace_bytes(count))
    work = work or Workspace()
    buf = work.ensure(nbytes)
    ok = torch.empty(count, dtype=torch.uint8, device=r.device)
    rad = torch.empty(count, dtype=torch.float64, device=r.device)
    npass = ctypes.c_int64(0)
    check(L.mt_certify(KIND[kind], l, n, r.data_ptr(), _ptr(rl), count, tol, ok.data_ptr(), rad.data_ptr(),
                       buf.data_ptr(), buf.numel(), ctypes.byref(npass),
                       torch.cuda.current_stream().cuda_stream))
    return ok, rad, int(npass.value)


def certify_basin(kind: str, n: int, roots, radius, l: int = 0, eps_max: float = 0.0, *,
                  work: Workspace | None = None, roots_lo=None):
    """Newton-basin radius of each root (Thm proofContract), given the proven
    radii of certify().  Returns (basin float64 tensor, n_pass)."""
    torch = _torch()
    L = load()
    r = torch.view_as_real(roots.contiguous()) if roots.is_complex() else roots.contiguous()
    rl = None
    if roots_lo is not None:
        rl = torch.view_as_real(roots_lo.contiguous()) if roots_lo.is_complex() else roots_lo.contiguous()
    count = r.shape[0]
    rad = radius.contiguous().to(torch.float64)
    work = work or Workspace()
    buf = work.ensure(int(L.mt_certify_workspace_bytes(count)))
    out = torch.empty(count, dtype=torch.float64, device=r.device)
    npass = ctypes.c_int64(0)
    check(L.mt_certify_basin(KIND[kind], l, n, r.data_ptr(), _ptr(rl), count, rad.data_ptr(), eps_max,
                             out.data_ptr(), buf.data_ptr(), buf.numel(), ctypes.byref(npass),
                             torch.cuda.current_stream().cuda_stream))
    return out, int(npass.value)


def separation(roots, *, roots_lo=None, mask=None, work: Workspace | None = None):
    """Nearest-neighbour distance of each root (Sec. 6.3.2 separation law).
    Returns (nn float64 tensor, band minima list of 64 floats, overall minimum)."""
    torch = _torch()
    L = load()
    r = torch.view_as_real(roots.contiguous()) if roots.is_complex() else roots.contiguous()
    rl = None
    if roots_lo is not None:
        rl = torch.view_as_real(roots_lo.contiguous()) if roots_lo.is_complex() else roots_lo.contiguous()
    m = None if mask is None else mask.contiguous().to(torch.uint8)
    count = r.shape[0]
    work = work or Workspace()
    buf = work.ensure(int(L.mt_separation_workspace_bytes(count)))
    nn = torch.empty(count, dtype=torch.float64, device=r.device)
    bands = (ctypes.c_double * 64)()
    mn = ctypes.c_double(0)
    check(L.mt_separation(count, r.data_ptr(), _ptr(rl), _ptr(m), nn.data_ptr(), bands, ctypes.byref(mn),
                          buf.data_ptr(), buf.numel(), torch.cuda.current_stream().cuda_stream))
    return nn, list(bands), mn.value


def evaluate(kind: str, n: int, c, l: int = 0):
    """P(c), P'(c) for a complex128 tensor c: returns complex128 [count, 2]."""
    torch = _torch()
    L = load()
    cr = torch.view_as_real(c.contiguous())
    out = torch.empty((c.shape[0], 4), dtype=torch.float64, device=c.device)
    check(L.mt_eval(KIND[kind], l, n, cr.data_ptr(), c.shape[0], out.data_ptr(),
                    torch.cuda.current_stream().cuda_stream))
    return torch.view_as_complex(out.view(-1, 2, 2))


def level_line(kind: str, n: int, l: int = 0, prec: str = "fp64", *, work: Workspace | None = None, **kw):
    """Upper-half starts of the discrete level line (steps a1-a3): complex128 tensor."""
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    nbytes = int(L.mt_workspace_bytes(KIND[kind], l, n, ctypes.byref(o)))
    work = work or Workspace()
    buf = work.ensure(nbytes)
    ns = ctypes.c_int64(0)
    st = Stats()
    L.mt_level_line(KIND[kind], l, n, ctypes.byref(o), None, 0, buf.data_ptr(), buf.numel(),
                    ctypes.byref(ns), None)
    starts = torch.empty((ns.value, 2), dtype=torch.float64, device="cuda")
    check(L.mt_level_line(KIND[kind], l, n, ctypes.byref(o), starts.data_ptr(), ns.value, buf.data_ptr(),
                          buf.numel(), ctypes.byref(ns), ctypes.byref(st)))
    return torch.view_as_complex(starts), st.as_dict()


def descend(kind: str, n: int, starts, l: int = 0, prec: str = "fp64", **kw):
    """Newton descents from given starts (step a4): (final iterates, status)."""
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    s = torch.view_as_real(starts.contiguous())
    count = s.shape[0]
    out = torch.empty((count, 2), dtype=torch.float64, device=s.device)
    status = torch.empty(count, dtype=torch.uint8, device=s.device)
    work = torch.empty(4096, dtype=torch.uint8, device=s.device)
    st = Stats()
    check(L.mt_descend(KIND[kind], l, n, ctypes.byref(o), s.data_ptr(), count, out.data_ptr(),
                       status.data_ptr(), work.data_ptr(), work.numel(), ctypes.byref(st)))
    return torch.view_as_complex(out), status, st.as_dict()


def classify(kind: str, n: int, roots, l: int = 0, tau: float = 0.0):
    """Type code of each root (step a6)."""
    torch = _torch()
    L = load()
    r = torch.view_as_real(roots.contiguous())
    t = torch.empty(r.shape[0], dtype=torch.uint8, device=r.device)
    check(L.mt_classify(KIND[kind], l, n, r.data_ptr(), r.shape[0], tau, t.data_ptr(),
                        torch.cuda.current_stream().cuda_stream))
    return t


def autotune(kind: str, n: int, l: int = 0, prec: str = "fp64", *, work: Workspace | None = None, **kw):
    """Pick the level-line chunk length and walk block size for P by timing
    complete splits (mt_autotune); later splits of P in this process use them.
    Returns (chunk_log2, block, device ms of the best candidate)."""
    torch = _torch()
    L = load()
    o = options(prec, **kw)
    d = degree(kind, n, l)
    # the largest workspace over the candidates (finer chunks need more seeds)
    nbytes = int(L.mt_workspace_bytes(KIND[kind], l, n, ctypes.byref(o)))
    for cl in range(3, 15):
        oc = options(prec, chunk_log2=cl, **kw)
        nbytes = max(nbytes, int(L.mt_workspace_bytes(KIND[kind], l, n, ctypes.byref(oc))))
    work = work or Workspace()
    buf = work.ensure(nbytes)
    roots = torch.empty((d, 2), dtype=torch.float64, device="cuda")
    c = ctypes.c_int(0)
    b = ctypes.c_int(0)
    ms = ctypes.c_float(0)
    check(L.mt_autotune(KIND[kind], l, n, ctypes.byref(o), roots.data_ptr(), d, buf.data_ptr(), buf.numel(),
                        ctypes.byref(c), ctypes.byref(b), ctypes.byref(ms)))
    return c.value, b.value, ms.value


def fma_peak(prec: str = "fp64") -> float:
    """FMA issue rate of the current GPU in TFLOP/s (mt_fma_peak): binary64
    for prec 'fp64', binary32 for 'fp32'."""
    torch = _torch()
    L = load()
    buf = torch.empty(int(L.mt_fma_peak_workspace_bytes()), dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    check(L.mt_fma_peak(0 if prec == "fp64" else 1, buf.data_ptr(), buf.numel(), ctypes.byref(out),
                        torch.cuda.current_stream().cuda_stream))
    return float(out.value)


def check_sqrt_up() -> tuple:
    """mt_check_sqrt_up: (failures, largest relative error) of the
    certificate's binary32 square-root upper bound over every normal
    binary32 on the current GPU."""
    torch = _torch()
    L = load()
    nf = ctypes.c_ulonglong(0)
    mr = ctypes.c_double(0.0)
    check(L.mt_check_sqrt_up(ctypes.byref(nf), ctypes.byref(mr), torch.cuda.current_stream().cuda_stream))
    return int(nf.value), float(mr.value)


def version() -> str:
    return load().mt_version().decode()
