"""ctypes declarations of the C ABI in include/ttn.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttn.so")

TTN_FP64, TTN_TF32, TTN_TF32X3, TTN_BF16, TTN_BF16X3 = range(5)
TTN_ENOCONV_CODE = -4
TTN_ETIMEOUT_CODE = -5
STATUS = {0: "TTN_OK", -1: "TTN_EINVAL", -2: "TTN_ENOMEM", -3: "TTN_ECUDA",
          -4: "TTN_ENOCONV", -5: "TTN_ETIMEOUT", -6: "TTN_ENAN"}

_dp = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("d", ctypes.c_int),
                ("chi", ctypes.c_int), ("K", ctypes.c_int), ("per_node", ctypes.c_int),
                ("onesite", _dp), ("A", _dp), ("B", _dp)]


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("top_mode", ctypes.c_int),
                ("lanczos_tol", ctypes.c_double), ("lanczos_max", ctypes.c_int),
                ("lanczos_restarts", ctypes.c_int), ("shift", ctypes.c_double),
                ("polar_damping", ctypes.c_double), ("deterministic", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("persistent", ctypes.c_int),
                ("streams", ctypes.c_int), ("polar_blocks", ctypes.c_int),
                ("double_float", ctypes.c_int), ("tc_engine", ctypes.c_int),
                ("wait_polls", ctypes.c_int), ("stage_streams", ctypes.c_int),
                ("recompute_ops", ctypes.c_int),
                ("tiles", ctypes.c_void_p),
                ("tiles_bytes", ctypes.c_size_t)]


# Every symbol the header declares, with its signature.
SIGNATURES = {
    "ttn_default_options": (None, [ctypes.POINTER(Options)]),
    "ttn_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(Options)]),
    "ttn_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Problem), ctypes.c_int,
                                  ctypes.POINTER(Options), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ttn_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                 ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]),
    "ttn_chis": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ttn_set_isometries": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, _dp]),
    "ttn_get_isometries": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, _dp]),
    "ttn_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "ttn_sweep_until": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), _dp]),
    "ttn_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_int]),
    "ttn_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "ttn_value_and_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp,
                                          ctypes.c_void_p]),
    "ttn_ascend": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
    "ttn_rdm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
    "ttn_env": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "ttn_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "ttn_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "ttn_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "ttn_profile_sweep": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_int]),
    "ttn_selftest_bytes": (ctypes.c_size_t, []),
    "ttn_selftest_gemm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, _dp,
                                         ctypes.c_int, ctypes.c_void_p]),
    "ttn_selftest_df": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, _dp, ctypes.c_int,
                                       ctypes.c_void_p]),
    "ttn_close_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]),
    "ttn_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "ttn_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ttn_destroy": (None, [ctypes.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libttn.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                          "(there is no fallback implementation)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
