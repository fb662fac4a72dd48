"""ctypes declarations for libmht (mirrors include/mht.h; argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmht.so")

MHT_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CALLBACK", 4: "NUMERIC", 5: "CUDA",
          6: "FORMAT", 7: "TIMEOUT", 8: "UNSUPPORTED", 9: "NOT_BOUND"}
REAL, COMPLEX = 0, 1
APPLY_FP64, APPLY_FP32, APPLY_3XTF32, APPLY_6XBF16 = 0, 1, 2, 3
TREE_AUTO, TREE_FIEDLER, TREE_RECT, TREE_PCA_MEDIAN, TREE_GIVEN, TREE_FIEDLER_MESH = 0, 1, 2, 3, 4, 5
EVAL_CALLBACK, EVAL_TORUS, EVAL_SPHERE, EVAL_DENSE = 0, 1, 2, 3

EVAL_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_int64), C.c_int64,
                      C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_double))


class Problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("field", C.c_int),
                ("eigenvalues", C.POINTER(C.c_double)), ("eval_kind", C.c_int),
                ("eval", EVAL_FN), ("eval_ctx", C.c_void_p),
                ("points", C.POINTER(C.c_double)), ("dim", C.c_int32),
                ("torus_modes", C.POINTER(C.c_int64)),
                ("dense", C.POINTER(C.c_double)), ("ld_dense", C.c_int64),
                ("space_perm", C.POINTER(C.c_int64)), ("space_offsets", C.POINTER(C.c_int64)),
                ("weights", C.POINTER(C.c_double)),
                ("tris", C.POINTER(C.c_int64)), ("ntris", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("eps", C.c_double), ("leaf_size", C.c_int64), ("levels", C.c_int32),
                ("mode", C.c_int), ("tree", C.c_int), ("seed", C.c_uint64),
                ("num_threads", C.c_int32), ("oversample", C.c_double), ("id_method", C.c_int)]


class Factors(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("levels", C.c_int32), ("field", C.c_int),
                ("space_perm", C.POINTER(C.c_int64)), ("space_offsets", C.POINTER(C.c_int64)),
                ("mode_perm", C.POINTER(C.c_int64)), ("mode_offsets", C.POINTER(C.c_int64)),
                ("ranks", C.POINTER(C.c_int32)), ("local_perm", C.POINTER(C.c_int32)),
                ("transfer", C.POINTER(C.c_double)), ("column_bases", C.POINTER(C.c_double)),
                ("weights", C.POINTER(C.c_double))]


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("levels", C.c_int32), ("field", C.c_int),
                ("mode", C.c_int), ("eps", C.c_double), ("blocks_per_level", C.c_int64),
                ("local_perm_entries", C.c_int64), ("transfer_entries", C.c_int64),
                ("column_basis_entries", C.c_int64), ("stored_entries", C.c_int64),
                ("max_rank", C.c_int64), ("workspace_entries_per_rhs", C.c_int64),
                ("factor_bytes", C.c_size_t), ("algorithmic_bytes", C.c_size_t),
                ("build_seconds", C.c_double)]


class LevelInfo(C.Structure):
    _fields_ = [("rank_min", C.c_int64), ("rank_median", C.c_int64), ("rank_max", C.c_int64),
                ("rank_sum", C.c_int64), ("transfer_entries", C.c_int64), ("bytes", C.c_size_t),
                ("algorithmic_bytes", C.c_size_t)]


# name -> (restype, argtypes); every entry point declared in include/mht.h
SIGNATURES = {
    "mht_build_plan": (C.c_int, [C.POINTER(Problem), C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "mht_problem_eval": (C.c_int, [C.POINTER(Problem), C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64),
                                   C.c_int64, C.POINTER(C.c_double)]),
    "mht_plan_import": (C.c_int, [C.POINTER(Factors), C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "mht_plan_export": (C.c_int, [C.c_void_p, C.POINTER(Factors)]),
    "mht_plan_info": (C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    "mht_plan_level_info": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(LevelInfo)]),
    "mht_plan_device_bytes": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "mht_plan_bind_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_int64,
                                       C.c_void_p]),
    "mht_synthesize": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]),
    "mht_synthesize_weighted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                          C.c_void_p]),
    "mht_synthesize_scaled": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64,
                                        C.c_int64, C.c_void_p]),
    "mht_filter": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                             C.c_int32, C.c_void_p]),
    "mht_lsqr_scratch_bytes": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t)]),
    "mht_inverse_lsqr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                   C.c_size_t, C.c_int32, C.c_double, C.c_void_p, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double)]),
    "mht_analyze": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                              C.c_void_p]),
    "mht_synthesize_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                                      C.c_void_p]),
    "mht_analyze_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                   C.c_void_p]),
    "mht_apply_launch_count": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "mht_plan_check": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "mht_synthesize_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mht_noalloc_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "mht_debug_host_alloc_limit": (C.c_int, [C.c_size_t]),
    "mht_noalloc_debug_hold": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "mht_plan_set_path": (C.c_int, [C.c_void_p, C.c_int32]),
    "mht_plan_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "mht_plan_clone": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mht_plan_autotune": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "mht_plan_tune_info": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "mht_plan_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "mht_plan_stage_times": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "mht_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_void_p)]),
    "mht_batch_device_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "mht_batch_bind_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]),
    "mht_batch_set_io": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_int64), C.c_void_p]),
    "mht_batch_synthesize": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mht_batch_analyze": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "mht_batch_set_graph": (C.c_int, [C.c_void_p, C.c_int32]),
    "mht_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "mht_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "mht_batch_check": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "mht_batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "mht_batch_debug_hold": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "mht_batch_destroy": (C.c_int, [C.c_void_p]),
    "mht_plan_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mht_plan_load": (C.c_int, [C.c_char_p, C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "mht_destroy": (C.c_int, [C.c_void_p]),
    "mht_last_error": (C.c_char_p, []),
    "mht_version": (C.c_char_p, []),
}

_lib = None


class MhtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Loads libmht.so (built in-tree by ``paper_2605_21828_gb300.build``); fails loudly."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libmht.so not built at {path}; run paper_2605_21828_gb300.build.build_library()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != MHT_OK:
        raise MhtError(status, load().mht_last_error().decode())
