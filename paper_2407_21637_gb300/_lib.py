"""ctypes declarations of the C ABI in include/hodlr.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhodlr.so")

PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "e4m3": 4, "e5m2": 5}
PREC_NAME = {v: k for k, v in PREC.items()}
MAX_DEPTH = 24

STATUS = {0: "HODLR_OK", 1: "HODLR_EINVAL", 2: "HODLR_ENOMEM", 3: "HODLR_ECUDA",
          4: "HODLR_ETIMEOUT", 5: "HODLR_ENOTFACTORED", 6: "HODLR_ESINGULAR",
          7: "HODLR_EACCURACY"}


class HodlrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("work", ctypes.c_int32),
                ("tier_mask", ctypes.c_uint32), ("per_block", ctypes.c_int32),
                ("max_nrhs", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("depth", ctypes.c_int32), ("work", ctypes.c_int32),
                ("per_block", ctypes.c_int32), ("max_rank", ctypes.c_int32),
                ("n_blocks", ctypes.c_int32), ("factor_bytes", ctypes.c_int64),
                ("u_bytes", ctypes.c_int64), ("v_bytes", ctypes.c_int64),
                ("leaf_bytes", ctypes.c_int64), ("scale_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("bytes_per_tier", ctypes.c_int64 * 6),
                ("norm2_all", ctypes.c_double), ("xi", ctypes.c_double * (MAX_DEPTH + 1)),
                ("u_prime", ctypes.c_double * (MAX_DEPTH + 1)),
                ("level_tier", ctypes.c_int32 * (MAX_DEPTH + 1))]


class Kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dim", ctypes.c_int32), ("c", ctypes.c_double),
                ("len2", ctypes.c_double), ("diag", ctypes.c_double)]


class BuildOpts(ctypes.Structure):
    _fields_ = [("sketch", ctypes.c_int32), ("max_sketch", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("node_sketch", ctypes.POINTER(ctypes.c_int32))]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("gmres_steps", ctypes.c_int32),
                ("backward_error", ctypes.c_double)]


# name -> (restype, argtypes); every symbol the header declares
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_DP = ctypes.POINTER(_D)
_I32P = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "hodlr_import": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _I32P, _DP, _DP, _DP,
                                    ctypes.POINTER(Opts), _P, ctypes.POINTER(_P)]),
    "hodlr_build": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(Kernel), _P,
                                   ctypes.POINTER(Opts), ctypes.POINTER(BuildOpts), _P,
                                   ctypes.POINTER(_P)]),
    "hodlr_export": (ctypes.c_int, [_P, _DP, _DP, _DP, _P]),
    "hodlr_matvec": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int64,
                                    ctypes.c_int32, _P]),
    "hodlr_matvec_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int64,
                                            ctypes.c_int32, _P]),
    "hodlr_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "hodlr_save": (ctypes.c_int, [_P, ctypes.c_char_p, _P]),
    "hodlr_load": (ctypes.c_int, [ctypes.c_char_p, _P, ctypes.POINTER(_P)]),
    "hodlr_sync_status": (ctypes.c_int, [_P, _P]),
    "hodlr_debug_stall_next": (ctypes.c_int, [_P]),
    "hodlr_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "hodlr_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "hodlr_block_tiers": (ctypes.c_int, [_P, _I32P, _I32P]),
    "hodlr_node_sizes": (ctypes.c_int, [_P, _I32P, _I32P]),
    "hodlr_build_stats": (ctypes.c_int, [_P, _I32P, _I32P, ctypes.POINTER(ctypes.c_int64)]),
    "hodlr_dense_kernel_matvec": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int32, _P, ctypes.c_int32, _P,
                                                 ctypes.c_int64, _P, ctypes.c_int64, _P]),
    "hodlr_lu": (ctypes.c_int, [_P, ctypes.c_double, _P]),
    "hodlr_lu_solve": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]),
    "hodlr_solve": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_int32, ctypes.POINTER(SolveStats), _P]),
    "hodlr_lu_export": (ctypes.c_int, [_P, _I32P, _I32P, _DP, _DP, _DP, _P]),
    "hodlr_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P), _I32P, ctypes.POINTER(_P),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_P),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.POINTER(_P)]),
    "hodlr_batch_run": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
    "hodlr_batch_tune": (ctypes.c_int, [_P, _P, _I32P, ctypes.POINTER(ctypes.c_float)]),
    "hodlr_batch_destroy": (None, [_P]),
    "hodlr_tree_order": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _I32P]),
    "hodlr_part_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "hodlr_part_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "hodlr_part_partial": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P]),
    "hodlr_part_finish": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, ctypes.c_int64, _P]),
    "hodlr_part_destroy": (None, [_P]),
    "hodlr_mlp_num_params": (ctypes.c_int32, []),
    "hodlr_mlp_features": (ctypes.c_int, [ctypes.POINTER(Kernel), _P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, _P, _P]),
    "hodlr_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "hodlr_mlp_loss": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P]),
    "hodlr_mlp_backward": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P]),
    "hodlr_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_float, _P]),
    "hodlr_destroy": (None, [_P]),
    "hodlr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hodlr_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libhodlr.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2407_21637_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != 0:
        detail = load().hodlr_last_error().decode()
        raise HodlrError(status, where, detail)
