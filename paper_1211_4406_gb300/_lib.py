"""ctypes binding of libtreepm_sr.so (argument marshalling only).

The library must be built in-tree first (``python -m paper_1211_4406_gb300.build``
or ``__graft_entry__.build()``).  There is no fallback: every entry point
raises when the library is missing or a call returns an error.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtreepm_sr.so")

TP_OK = 0
TP_FP64 = 0
TP_FP32 = 1
TP_FLAG_CHUNKED = 1
TP_FLAG_XI_SOFTENED = 2
TP_FLAG_RSQRT_REFINED = 4
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "device out of memory",
          -4: "capacity overflow", -5: "device wait timed out", -6: "non-finite position",
          -7: "no CUDA device"}


class TPParams(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("r_cut", C.c_double), ("theta", C.c_double),
                ("n_crit", C.c_int32), ("n_leaf", C.c_int32), ("precision", C.c_int32),
                ("flags", C.c_int32)]


class TPStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_nodes", C.c_int64), ("n_groups", C.c_int64),
                ("n_entries", C.c_int64), ("n_interactions", C.c_int64), ("n_useful", C.c_int64),
                ("n_ambiguous", C.c_int64),
                ("mean_ni", C.c_double), ("mean_nj", C.c_double), ("max_nj", C.c_int32),
                ("nbox", C.c_int32), ("n_windows", C.c_int64)]


class TreeSRError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} ({code})")
        self.code = code


_V = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_D = C.c_double

SIGNATURES = {
    "tp_build_tree": ([_V, _V, _I64, C.POINTER(TPParams), _V, C.POINTER(_V)], C.c_int),
    "tp_build_tree_batched": ([_V, _V, C.POINTER(_I64), _I32, C.POINTER(TPParams), _V, C.POINTER(_V)],
                              C.c_int),
    "tp_rebuild_tree": ([_V, _V, _V, _V], C.c_int),
    "tp_refit_tree": ([_V, _V, _V, _V], C.c_int),
    "tp_short_range_force": ([_V, _V, _V], C.c_int),
    "tp_short_range_vjp": ([_V, _V, _V, _V], C.c_int),
    "tp_short_range_force_vjp": ([_V, _V, _V, _V, _V], C.c_int),
    "tp_tree_status": ([_V], C.c_int),
    "tp_tree_stats": ([_V, C.POINTER(TPStats)], C.c_int),
    "tp_export_keys": ([_V, _V, _V], C.c_int),
    "tp_export_nodes": ([_V, _V, _V], C.c_int),
    "tp_export_groups": ([_V, _V, _V], C.c_int),
    "tp_export_lists": ([_V, _V, _V], C.c_int),
    "tp_tree_free": ([_V], C.c_int),
    "tp_tree_set_tile": ([_V, _I32, _I32], C.c_int),
    "tp_tree_set_walk_budget": ([_V, _I64], C.c_int),
    "tp_tree_set_kernel_timing": ([_V, _I32], C.c_int),
    "tp_tree_kernel_ms": ([_V, C.POINTER(_D), C.POINTER(_D)], C.c_int),
    "tp_axpy": ([_V, _V, _I32, _D, _I64, _V], C.c_int),
    "tp_scale": ([_V, _I32, _V, _D, _I64, _V], C.c_int),
    "tp_measure_peak": ([_I32, C.POINTER(_D), _V], C.c_int),
    "tp_short_range_force_noalloc": ([_V, _V, _I64, C.POINTER(TPParams), _V, _V], C.c_int),
    "tp_launch_count": ([], _I64),
    "tp_pm_create": ([_I32, _D, _D, _V, C.POINTER(_V)], C.c_int),
    "tp_pm_force": ([_V, _V, _V, _I64, _V, _I32, _V], C.c_int),
    "tp_pm_vjp": ([_V, _V, _V, _I64, _V, _V, _I32, _V], C.c_int),
    "tp_pm_force_vjp": ([_V, _V, _V, _I64, _V, _V, _V, _I32, _V], C.c_int),
    "tp_pm_export_mesh": ([_V, _I32, _V], C.c_int),
    "tp_pm_free": ([_V], C.c_int),
    "tp_status_string": ([C.c_int], C.c_char_p),
    "tp_halo_create": ([_I32, _I32, _I32, C.POINTER(_V)], C.c_int),
    "tp_halo_set_cuts": ([_V, _V, _V, _V], C.c_int),
    "tp_halo_select": ([_V, _V, _I64, _I32, _I32, _D, _V, _I64, _V, _V], C.c_int),
    "tp_halo_free": ([_V], C.c_int),
    "tp_gather_rows": ([_V, _I32, _V, _I64, _V, _V], C.c_int),
    "tp_scatter_add_rows": ([_V, _I32, _V, _V, _I64, _V], C.c_int),
}

_lib = None


def load():
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1211_4406_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(code: int, where: str) -> None:
    if code != TP_OK:
        raise TreeSRError(code, where)


def params(G=1.0, eps=0.0, r_cut=0.1, theta=0.5, n_crit=64, n_leaf=8, precision="fp32") -> TPParams:
    prec = {"fp32": TP_FP32, "fp64": TP_FP64}[precision]
    return TPParams(float(G), float(eps), float(r_cut), float(theta), int(n_crit), int(n_leaf), prec, 0)
