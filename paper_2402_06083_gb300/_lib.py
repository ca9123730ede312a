"""ctypes declarations of the C ABI in include/mtsplit.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  If the library is missing or cannot be loaded this module raises;
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmtsplit.so")

MT_OK, MT_EINVAL, MT_ENOMEM, MT_ECAPACITY, MT_ECUDA, MT_EINCOMPLETE, MT_ETIMEOUT, MT_ECERT = range(8)
STATUS_NAMES = {0: "MT_OK", 1: "MT_EINVAL", 2: "MT_ENOMEM", 3: "MT_ECAPACITY", 4: "MT_ECUDA",
                5: "MT_EINCOMPLETE", 6: "MT_ETIMEOUT", 7: "MT_ECERT"}
PREC = {"fp64": 0, "mixed": 1, "dd": 2}
MT_MAX_TYPES = 64

# every symbol include/mtsplit.h declares
EXPORTS = (
    "mt_default_options", "mt_degree_hyperbolic", "mt_degree_misiurewicz", "mt_workspace_bytes",
    "mt_split_hyperbolic", "mt_split_misiurewicz", "mt_split_misiurewicz_q", "mt_misiurewicz_pairs",
    "mt_workspace_bytes_misiurewicz_batch", "mt_split_misiurewicz_batch",
    "mt_certify_workspace_bytes", "mt_certify", "mt_certify_basin", "mt_separation_workspace_bytes", "mt_separation",
    "mt_eval", "mt_level_line",
    "mt_descend",
    "mt_classify", "mt_certify_static", "mt_autotune", "mt_fma_peak_workspace_bytes", "mt_fma_peak",
    "mt_check_sqrt_up",
    "mt_last_error", "mt_version",
)
MT_CERTIFY_STATIC_MAX_ROOTS = 131072


class Options(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("lambda0", ctypes.c_double),
        ("M", ctypes.c_int),
        ("c_L", ctypes.c_int),
        ("chunk_log2", ctypes.c_int),
        ("block", ctypes.c_int),
        ("max_retries", ctypes.c_int),
        ("eps_dup", ctypes.c_double),
        ("cert_tol", ctypes.c_double),
        ("use_graph", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("dd_radius", ctypes.c_double),
        ("dd_all", ctypes.c_int),
        ("stream_pieces", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "degree", "n_roots", "n_real", "n_starts", "n_conv", "n_repeat", "n_diverge", "n_timeout",
        "walk_newton", "desc_newton", "steps_fp32", "steps_dd", "walk_fail", "n_cert_pass")] + [
        ("count_by_type", ctypes.c_int64 * MT_MAX_TYPES),
        ("M", ctypes.c_int32), ("c_L", ctypes.c_int32), ("retries", ctypes.c_int32),
        ("n_chunks", ctypes.c_int32), ("n_launches", ctypes.c_int64),
        ("max_cert_radius", ctypes.c_double), ("min_cert_radius", ctypes.c_double),
        ("eps_dup", ctypes.c_double),
        ("ms_total", ctypes.c_float), ("ms_walk", ctypes.c_float), ("ms_descend", ctypes.c_float),
        ("ms_dedup", ctypes.c_float), ("ms_certify", ctypes.c_float),
        ("prec_used", ctypes.c_int32), ("ms_dd", ctypes.c_float),
        ("n_zones", ctypes.c_int64), ("n_zone_roots", ctypes.c_int64), ("n_dd_pieces", ctypes.c_int64),
        ("seed_newton", ctypes.c_int64), ("desc_fp32", ctypes.c_int64), ("ms_seeds", ctypes.c_float),
        ("reserved", ctypes.c_int32), ("n_finish", ctypes.c_int64), ("n_mult", ctypes.c_int64),
        ("ms_k_walk", ctypes.c_float), ("ms_k_desc64", ctypes.c_float), ("ms_k_desc32", ctypes.c_float),
        ("ms_k_finish", ctypes.c_float), ("finish_newton", ctypes.c_int64), ("n_k_timed", ctypes.c_int32),
        ("n_tip64", ctypes.c_int32), ("desc_orbit_steps", ctypes.c_int64),
        ("first_n_roots", ctypes.c_int64), ("first_n_cert_pass", ctypes.c_int64),
        ("first_walk_fail", ctypes.c_int32), ("first_prec", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "count_by_type" else v
        return d


_LIB = None


def load() -> ctypes.CDLL:
    """Load libmtsplit.so; raise if it is not built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmtsplit.so is not built (run __graft_entry__.build() or "
                           "python paper_2402_06083_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    i64p = ctypes.POINTER(ctypes.c_int64)
    op = ctypes.POINTER(Options)
    sp = ctypes.POINTER(Stats)
    sig = {
        "mt_default_options": (None, [op]),
        "mt_degree_hyperbolic": (i64, [ctypes.c_int]),
        "mt_degree_misiurewicz": (i64, [ctypes.c_int, ctypes.c_int]),
        "mt_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, op]),
        "mt_split_hyperbolic": (ctypes.c_int, [ctypes.c_int, op, vp, vp, i64, vp, ctypes.c_size_t, i64p, sp]),
        "mt_split_misiurewicz": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, op, vp, vp, i64, vp, vp,
                                                ctypes.c_size_t, i64p, sp]),
        "mt_split_misiurewicz_q": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, op, vp, i64, vp, vp, vp, vp,
                                                  ctypes.c_size_t, i64p, sp]),
        "mt_misiurewicz_pairs": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
        "mt_workspace_bytes_misiurewicz_batch": (ctypes.c_size_t, [ctypes.c_int, op]),
        "mt_split_misiurewicz_batch": (ctypes.c_int, [ctypes.c_int, op, vp, vp, i64, vp, vp,
                                                      ctypes.c_size_t, i64p, sp]),
        "mt_certify_workspace_bytes": (ctypes.c_size_t, [i64]),
        "mt_certify": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, i64, ctypes.c_double,
                                      vp, vp, vp, ctypes.c_size_t, i64p, vp]),
        "mt_certify_basin": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, i64, vp,
                                            ctypes.c_double, vp, vp, ctypes.c_size_t, i64p, vp]),
        "mt_separation_workspace_bytes": (ctypes.c_size_t, [i64]),
        "mt_separation": (ctypes.c_int, [i64, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
        "mt_eval": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, i64, vp, vp]),
        "mt_level_line": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, op, vp, i64, vp,
                                         ctypes.c_size_t, i64p, sp]),
        "mt_descend": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, op, vp, i64, vp, vp, vp,
                                      ctypes.c_size_t, sp]),
        "mt_classify": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, i64, ctypes.c_double,
                                       vp, vp]),
        "mt_certify_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, i64, ctypes.c_double,
                                             vp, vp, i64p, vp]),
        "mt_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, op, vp, i64, vp, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_float)]),
        "mt_fma_peak_workspace_bytes": (ctypes.c_size_t, []),
        "mt_fma_peak": (ctypes.c_int, [ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double), vp]),
        "mt_check_sqrt_up": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_double), vp]),
        "mt_last_error": (ctypes.c_char_p, []),
        "mt_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


class MtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(rc: int) -> None:
    if rc != MT_OK:
        raise MtError(rc, load().mt_last_error().decode())
