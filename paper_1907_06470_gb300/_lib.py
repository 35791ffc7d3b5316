"""ctypes view of the C ABI declared in include/rsvd.h (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

c_i32, c_i64, c_u64, c_size, c_vp = C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_void_p

RSVD_OK = 0
STAGES = ["gaussian", "apass_fwd", "apass_trans", "orth", "small_svd", "lift", "h2d", "total", "quantize", "sweep"]
STATUS_NAMES = {
    0: "RSVD_OK", 1: "RSVD_ERR_INVALID_ARG", 2: "RSVD_ERR_OOM", 3: "RSVD_ERR_CAP_TOO_SMALL",
    4: "RSVD_ERR_CUDA", 5: "RSVD_ERR_NOT_SPD", 6: "RSVD_ERR_NO_CONVERGE", 7: "RSVD_ERR_TIMEOUT",
    8: "RSVD_ERR_UNSUPPORTED", 9: "RSVD_ERR_INTERRUPTED",
}
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16x3": 3, "fp8": 4}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
DENSE, CSR = 0, 1
ON_DEVICE, ON_HOST = 0, 1


class RsvdOpts(C.Structure):
    _fields_ = [("prec", c_i32), ("refine", c_i32), ("mb", c_i64), ("nb", c_i64),
                ("n_slots", c_i32), ("dtype", c_i32), ("kind", c_i32), ("auto_q", c_i32),
                ("auto_q_tol", C.c_double), ("fused", c_i32), ("reserved", c_i32)]


class RsvdMatrix(C.Structure):
    _fields_ = [("kind", c_i32), ("dtype", c_i32), ("location", c_i32), ("reserved", c_i32),
                ("m", c_i64), ("n", c_i64), ("data", c_vp), ("ld", c_i64),
                ("rowptr", c_vp), ("colidx", c_vp), ("val", c_vp), ("nnz", c_i64),
                ("t_rowptr", c_vp), ("t_colidx", c_vp), ("t_val", c_vp)]


class RsvdTile(C.Structure):
    _fields_ = [(f, c_i64) for f in ("t", "I", "J", "row0", "row1", "col0", "col1", "slot")]


class RsvdPlanInfo(C.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("k", c_i32), ("p", c_i32), ("q", c_i32), ("r", c_i32),
                ("prec", c_i32), ("dtype", c_i32), ("mb", c_i64), ("nb", c_i64),
                ("tiles_m", c_i64), ("tiles_n", c_i64), ("n_slots", c_i32), ("resident", c_i32),
                ("workspace_bytes", c_size), ("min_cap_bytes", c_size), ("seed", c_u64), ("q_used", c_i32),
                ("resumed_from", c_i32),
                ("bf16_copy", c_i32)]


class RsvdCheckpointInfo(C.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("k", c_i32), ("p", c_i32), ("q", c_i32), ("r", c_i32),
                ("prec", c_i32), ("dtype", c_i32), ("kind", c_i32), ("seed", c_u64), ("fingerprint", c_u64),
                ("step", c_i32), ("panel_rows", c_i64), ("panel_bytes", c_u64)]


# Every function the header declares, with its ctypes signature.
SIGNATURES = {
    "rsvd_plan": (c_i32, [c_i64, c_i64, C.c_int, C.c_int, C.c_int, c_u64, c_size, C.POINTER(RsvdOpts), C.POINTER(c_vp)]),
    "rsvd_plan_min_cap": (c_i32, [c_i64, c_i64, C.c_int, C.c_int, C.POINTER(RsvdOpts), C.POINTER(c_size)]),
    "rsvd_plan_info": (c_i32, [c_vp, C.POINTER(RsvdPlanInfo)]),
    "rsvd_run": (c_i32, [c_vp, C.POINTER(RsvdMatrix), c_vp, c_vp, c_vp, c_vp]),
    "rsvd_plan_prefetch": (c_i32, [c_vp, C.POINTER(RsvdMatrix)]),
    "rsvd_full": (c_i32, [C.POINTER(RsvdMatrix), c_vp, c_vp, c_vp, c_vp]),
    "rsvd_destroy": (None, [c_vp]),
    "rsvd_backward": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "rsvd_status_str": (C.c_char_p, [c_i32]),
    "rsvd_last_error": (C.c_char_p, []),
    "rsvd_plan_set_profiling": (c_i32, [c_vp, c_i32]),
    "rsvd_plan_stage_ms": (c_i32, [c_vp, C.POINTER(C.c_double), C.POINTER(c_i32)]),
    "rsvd_kernel_launches": (C.c_ulonglong, []),
    "rsvd_plan_stream_stats": (c_i32, [c_vp, C.POINTER(c_u64), C.POINTER(c_i64), C.POINTER(c_i64)]),
    "rsvd_gaussian": (c_i32, [c_u64, c_i64, c_i64, c_i32, c_i32, c_vp, c_i64, c_vp]),
    "rsvd_tile_map": (c_i32, [c_i64, c_i64, c_i64, c_i64, c_i32, C.POINTER(RsvdTile), c_i64, C.POINTER(c_i64)]),
    "rsvd_apass_workspace": (c_size, [c_i64, c_i64, c_i32, c_i32, c_i32, c_i64, c_i64]),
    "rsvd_apass": (c_i32, [C.POINTER(RsvdMatrix), c_i32, c_i32, c_i32, c_vp, c_i64, c_vp, c_i64, c_i64, c_i64,
                           c_vp, c_size, c_vp]),
    "rsvd_orth_workspace": (c_size, [c_i64, c_i32]),
    "rsvd_orth": (c_i32, [c_i32, c_i64, c_i32, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_size, c_vp]),
    "rsvd_small_svd_workspace": (c_size, [c_i32]),
    "rsvd_small_svd": (c_i32, [c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "rsvd_small_svd_noalloc": (c_i32, [c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "rsvd_csr_transpose": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "rsvd_csr_tile": (c_i32, [c_i64, c_i64, c_vp, c_vp, c_vp, c_i64, c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_i64,
                              C.POINTER(c_i64)]),
    "rsvd_coo_to_csr": (c_i32, [c_i64, c_i64, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "rsvd_spmm_workspace": (c_size, [c_i64, c_i32]),
    "rsvd_csr_apass_workspace": (c_size, [c_i64, c_i64, c_i32, c_i32]),
    "rsvd_plan_set_checkpoint": (c_i32, [c_vp, C.c_char_p, c_i32]),
    "rsvd_checkpoint_info": (c_i32, [C.c_char_p, C.POINTER(RsvdCheckpointInfo)]),
    "rsvd_fp8_quantize": (c_i32, [C.POINTER(RsvdMatrix), c_i64, c_i64, c_vp, c_i64, c_vp, c_vp]),
}
NOALLOC_MAX_R = 256

_lock = threading.Lock()
_lib = None


class RsvdError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {detail}")
        self.status = status
        self.detail = detail


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load librsvd_gb300.so (building it in-tree first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"librsvd_gb300.so missing at {_build.LIB}; run build()")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int):
    if status != RSVD_OK:
        lib = load(build_if_needed=False)
        raise RsvdError(status, lib.rsvd_last_error().decode(errors="replace"))
