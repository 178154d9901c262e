"""ctypes loader of libmrcqr.so (the C ABI declared in include/mrcqr.h).

There is no fallback: if the compiled library is missing or fails to load,
every call raises."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmrcqr.so")

PREC = {"fp16": 0, "bf16": 1, "fp32": 2, "fp64": 3, "auto": 4}
PREC_NAME = {v: k for k, v in PREC.items()}
STATUS = {0: "OK", 1: "INVALID", 2: "BREAKDOWN", 3: "NONFINITE", 4: "ORTHO", 5: "ALLOC", 6: "CUDA", 7: "TIMEOUT"}


class MrcqrError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"mrcqr error {code} ({STATUS.get(code, '?')}){': ' + what if what else ''}")


class Opts(ctypes.Structure):
    _fields_ = [("s_factor", ctypes.c_int32), ("check", ctypes.c_int32), ("escalate", ctypes.c_int32),
                ("sketch_variant", ctypes.c_int32), ("ortho_tol", ctypes.c_double), ("stats_device", ctypes.c_void_p),
                ("fp64_products", ctypes.c_int32), ("transform", ctypes.c_int32)]


class BatchedOpts(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int32), ("autotune", ctypes.c_int32), ("check", ctypes.c_int32),
                ("escalate", ctypes.c_int32), ("ortho_tol", ctypes.c_double), ("rows_per_split", ctypes.c_int64),
                ("rows_per_chunk", ctypes.c_int64), ("fp64_products", ctypes.c_int32), ("transform", ctypes.c_int32),
                ("oz_per_problem", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("prec_used", ctypes.c_int32), ("retries", ctypes.c_int32),
                ("prec_first", ctypes.c_int32), ("selector_choice", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3), ("ortho_fro", ctypes.c_double)]

    def as_dict(self):
        return {"status": STATUS.get(self.status, str(self.status)), "status_code": int(self.status),
                "prec_used": PREC_NAME.get(self.prec_used, str(self.prec_used)), "retries": int(self.retries),
                "prec_first": PREC_NAME.get(self.prec_first, str(self.prec_first)),
                "selector_choice": int(self.selector_choice), "ortho_fro": float(self.ortho_fro)}


_i64 = ctypes.c_int64
_i32 = ctypes.c_int
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p

SIGNATURES = {
    "mrcqr_version": ([], _i32),
    "mrcqr_status_string": ([_i32], ctypes.c_char_p),
    "mrcqr_factor": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i32, _u64, _vp], _i32),
    "mrcqr_factor_ex": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _u64, ctypes.POINTER(Opts), _vp], _i32),
    "mrcqr_get_last_status": ([_vp, ctypes.POINTER(Stats)], _i32),
    "mrcqr_factor_batched": ([_i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_vp),
                              ctypes.POINTER(_i64), ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_vp),
                              ctypes.POINTER(_i32), ctypes.POINTER(_u64), _vp, _vp], _i32),
    "mrcqr_batched_plan_create": ([_i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_i64), ctypes.POINTER(_vp), ctypes.POINTER(_i64),
                                   ctypes.POINTER(_vp), ctypes.POINTER(_i32), ctypes.POINTER(_u64), _vp,
                                   ctypes.POINTER(BatchedOpts), ctypes.POINTER(_vp)], _i32),
    "mrcqr_batched_plan_execute": ([_vp, _vp], _i32),
    "mrcqr_batched_plan_info": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(_i64)], _i32),
    "mrcqr_batched_plan_destroy": ([_vp], _i32),
    "mrcqr_signs": ([_i64, _u64, _vp, _vp], _i32),
    "mrcqr_sample_rows": ([_i64, _i64, _u64, _vp, _vp], _i32),
    "mrcqr_sample_transform_rows": ([_i64, _i64, _i32, _u64, _vp, _vp], _i32),
    "mrcqr_round": ([_i32, _i64, _vp, _vp, _vp], _i32),
    "mrcqr_sketch": ([_i64, _i64, _vp, _i64, _i64, _i32, _u64, _vp, _vp], _i32),
    "mrcqr_sketch_ex": ([_i64, _i64, _vp, _i64, _i64, _i32, _u64, _i32, _vp, _vp], _i32),
    "mrcqr_sketch_transform": ([_i64, _i64, _vp, _i64, _i64, _i32, _i32, _u64, _i32, _vp, _vp], _i32),
    "mrcqr_regime_estimate": ([_i64, _i64, _vp, _i64, _i32, _u64, _vp, _vp], _i32),
    "mrcqr_debug_wait_timeout": ([ctypes.c_uint32, _vp, _vp], _i32),
    "mrcqr_sketch_qr": ([_i64, _i64, _vp, _i32, _vp, _vp], _i32),
    "mrcqr_last_sketch_variant": ([], _i32),
    "mrcqr_cholqr_precond": ([_i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp], _i32),
    "mrcqr_finalize_q": ([_i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp], _i32),
    "mrcqr_gram": ([_i64, _i64, _vp, _i64, _vp, _i32, _vp], _i32),
    "mrcqr_cholqr2": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp], _i32),
    "mrcqr_trsm": ([_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp], _i32),
    "mrcqr_sketch_qr_noalloc": ([_i64, _i64, _vp, _i32, _vp, _vp], _i32),
    "mrcqr_selector_num_params": ([], _i32),
    "mrcqr_selector_set": ([_vp, _vp, _vp, _vp], _i32),
    "mrcqr_selector_load": ([ctypes.c_char_p], _i32),
    "mrcqr_selector_features": ([_i64, _i64, _vp, _vp, _vp], _i32),
    "mrcqr_mlp_forward": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "mrcqr_mlp_train_step": ([_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, ctypes.c_float, _i32, _i32, _vp, _vp, _vp], _i32),
    "mrcqr_launch_count": ([], ctypes.c_uint64),
    "mrcqr_stage_name": ([_i32], ctypes.c_char_p),
    "mrcqr_profile_begin": ([], _i32),
    "mrcqr_profile_end": ([_i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)], _i32),
    "mrcqr_shutdown": ([], _i32),
}

_LIB = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (once) and return the library with argument types set."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise MrcqrError(6, f"compiled library not found at {p}; run __graft_entry__.build() or "
                            f"python -m paper_2606_18411_gb300.build")
    lib = ctypes.CDLL(p)
    for name, (argt, rest) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = argt
        fn.restype = rest
    if path is None:
        _LIB = lib
    return lib


def check(rc: int, what: str = "") -> None:
    if rc != 0:
        raise MrcqrError(rc, what)
