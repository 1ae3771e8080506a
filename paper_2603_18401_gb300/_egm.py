"""ctypes binding of libegm.so (declarations in include/egm.h).

Argument marshalling only: every step of the matching path runs in the CUDA
kernels of the shared library.  Loading fails loudly when the library has not
been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libegm.so")

EGM_OK = 0
EGM_ERR_ARG = -1
EGM_ERR_CUDA = -2
EGM_ERR_NOMEM = -3
EGM_ERR_CAPACITY = -4
EGM_ERR_DEGENERATE_F = -5
EGM_ERR_NAN = -6
EGM_ERR_TIMEOUT = -7
EGM_ERR_UNIMPLEMENTED = -8

EGM_DESC_U8_L2 = 0
EGM_DESC_F32_L2 = 1
EGM_DESC_BIN = 2

EGM_FLAG_HAS_BEST = 1
EGM_FLAG_RATIO_PASS = 2
EGM_FLAG_NO_SECOND = 4
EGM_FLAG_DEGENERATE_LINE = 8
EGM_FLAG_MUTUAL = 16
EGM_FLAG_GMS = 32
EGM_FLOAT_PASS_BF16 = 0
EGM_FLOAT_PASS_FP8 = 1

EGM_FORM_AUTO = 0
EGM_FORM_PLAIN = 1
EGM_FORM_BANDED = 2

EGM_MLP_PARAMS = 8769


class egm_pair(C.Structure):
    _fields_ = [
        ("xy1", C.c_void_p), ("xy2", C.c_void_p), ("F", C.c_void_p), ("eps2", C.c_void_p),
        ("desc1", C.c_void_p), ("desc2", C.c_void_p),
        ("m", C.c_int32), ("n", C.c_int32), ("eps_scalar", C.c_double),
        ("kind", C.c_int32), ("dim", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
    ]


class egm_out(C.Structure):
    _fields_ = [
        ("best", C.c_void_p), ("second", C.c_void_p), ("best_d", C.c_void_p),
        ("second_d", C.c_void_p), ("flags", C.c_void_p), ("cand_offsets", C.c_void_p),
        ("cand_idx", C.c_void_p), ("cand_capacity", C.c_int64), ("cand_total", C.c_void_p),
    ]


class egm_params(C.Structure):
    _fields_ = [("ratio_num", C.c_int32), ("ratio_den", C.c_int32), ("sync", C.c_int32),
                ("form", C.c_int32), ("band_tile", C.c_int32), ("float_pass", C.c_int32),
                ("timeout_check", C.c_int32), ("tune", C.c_int32), ("reserved", C.c_int32 * 8)]


class egm_stats(C.Structure):
    _fields_ = [("queries", C.c_int64), ("refs", C.c_int64), ("window_refs", C.c_int64),
                ("candidates", C.c_int64), ("fp64_rechecks", C.c_int64)]


class egm_timing(C.Structure):
    _fields_ = [("geometry_ms", C.c_double), ("prep_ms", C.c_double), ("sort_ms", C.c_double),
                ("post_sort_ms", C.c_double), ("stab_ms", C.c_double), ("csr_ms", C.c_double),
                ("calls", C.c_int64), ("banded_calls", C.c_int64)]


class egm_gms_pair(C.Structure):
    _fields_ = [("xy1", C.c_void_p), ("xy2", C.c_void_p), ("best", C.c_void_p), ("flags", C.c_void_p),
                ("m", C.c_int64), ("n", C.c_int64), ("width1", C.c_int32), ("height1", C.c_int32),
                ("width2", C.c_int32), ("height2", C.c_int32)]


# name -> (restype, argtypes); every symbol include/egm.h declares
SIGNATURES = {
    "egm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "egm_destroy": (C.c_int, [C.c_void_p]),
    "egm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "egm_set_params": (C.c_int, [C.c_void_p, C.POINTER(egm_params)]),
    "egm_get_params": (C.c_int, [C.c_void_p, C.POINTER(egm_params)]),
    "egm_default_params": (None, [C.POINTER(egm_params)]),
    "egm_reserve": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32]),
    "egm_match_pair": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.POINTER(egm_out)]),
    "egm_match_batch": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.c_int32, C.POINTER(egm_out)]),
    "egm_match_pair_host": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.POINTER(egm_out)]),
    "egm_match_pair_static": (C.c_int, [C.POINTER(egm_pair), C.POINTER(egm_out), C.POINTER(egm_params),
                                        C.c_void_p]),
    "egm_graph_create": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.c_int32, C.POINTER(egm_out),
                                   C.POINTER(C.c_void_p)]),
    "egm_graph_launch": (C.c_int, [C.c_void_p]),
    "egm_graph_destroy": (C.c_int, [C.c_void_p]),
    "egm_mlp_create": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "egm_mlp_destroy": (C.c_int, [C.c_void_p]),
    "egm_mlp_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "egm_mlp_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "egm_mlp_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "egm_mlp_set_fallback": (C.c_int, [C.c_void_p, C.c_double]),
    "egm_match_mutual_pair": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.c_void_p, C.c_double, C.c_int32, C.c_int32,
                                        C.POINTER(egm_out)]),
    "egm_tuner_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "egm_tuner_import": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "egm_mlp_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p,
                               C.c_void_p]),
    "egm_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float,
                                     C.c_void_p]),
    "egm_pair_residuals": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.c_void_p, C.c_void_p, C.c_int64,
                                     C.c_void_p]),
    "egm_match_mutual": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.POINTER(egm_pair), C.POINTER(egm_out)]),
    "egm_match_batch_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "egm_gms_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_uint32, C.c_int32, C.c_double]),
    "egm_gms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                          C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_int32, C.c_double]),
    "egm_compact_matches": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_uint32, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "egm_sync": (C.c_int, [C.c_void_p]),
    "egm_intervals": (C.c_int, [C.c_void_p, C.POINTER(egm_pair), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "egm_set_counters": (C.c_int, [C.c_void_p, C.c_int32]),
    "egm_get_stats": (C.c_int, [C.c_void_p, C.POINTER(egm_stats)]),
    "egm_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "egm_get_timing": (C.c_int, [C.c_void_p, C.POINTER(egm_timing)]),
    "egm_status_string": (C.c_char_p, [C.c_int]),
    "egm_version": (C.c_int32, []),
}

_lib = None


class EgmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = load().egm_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} ({status})")


def load():
    """Load libegm.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libegm.so not built at {LIB_PATH}; run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str) -> None:
    if status != EGM_OK:
        raise EgmError(status, where)
