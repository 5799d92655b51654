"""ctypes declarations of the C ABI in ``include/cossin.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

_lock = threading.Lock()
_lib = None

CS_OK, CS_EINVAL, CS_ENOMEM, CS_ENONFINITE, CS_ERANGE, CS_ECUDA, CS_ETIMEOUT = range(7)
STATUS_NAMES = {0: "CS_OK", 1: "CS_EINVAL", 2: "CS_ENOMEM", 3: "CS_ENONFINITE", 4: "CS_ERANGE",
                5: "CS_ECUDA", 6: "CS_ETIMEOUT"}
CS_FP64, CS_FP32, CS_SPLIT_TF32, CS_FP64_EMU, CS_SPLIT_EMU, CS_SPLIT_BF16 = 0, 1, 2, 3, 4, 5
KERNEL_KINDS = {"norm1": 0, "gemm_f64": 1, "gemm_tf32": 2, "batched": 3, "adjoint": 4, "other": 5, "gemm_emu": 6}


class CsInfo(ctypes.Structure):
    _fields_ = [("norm1", ctypes.c_double), ("m", ctypes.c_int32), ("s", ctypes.c_int32),
                ("products", ctypes.c_int32), ("table", ctypes.c_int32), ("flops", ctypes.c_double)]

    def as_dict(self):
        return {"norm1": self.norm1, "m": self.m, "s": self.s, "products": self.products,
                "table": self.table, "flops": self.flops}


class CossinError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_sz = ctypes.c_size_t

SIGNATURES = {
    "cossin_workspace_size": (ctypes.c_int, [_i64, ctypes.c_int, ctypes.POINTER(_sz)]),
    "cossin_norm1": (ctypes.c_int, [_vp, _i64, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    "cossin_norm1_noalloc": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp, _vp]),
    "cossin_select": (ctypes.c_int, [ctypes.c_double, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cossin": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp, _vp, _vp]),
    "cossin_ex": (ctypes.c_int, [_vp, _i64, ctypes.c_int, _vp, _vp, _vp, _sz, _i32, _i32,
                                 ctypes.POINTER(CsInfo), _vp]),
    "cossin_cs_select": (ctypes.c_int, [ctypes.c_double, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cossin_cs": (ctypes.c_int, [_vp, _i64, ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _sz, _i32, _i32,
                                 ctypes.POINTER(CsInfo), _vp]),
    "cossin_matmul": (ctypes.c_int, [_vp, _vp, _i64, ctypes.c_int, _vp, _vp]),
    "cossin_backward": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "cossin_backward_ex": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_int, _vp,
                                          _vp]),
    "cossin_unitary_workspace_size": (ctypes.c_int, [_i64, ctypes.c_int, ctypes.POINTER(_sz)]),
    "cossin_unitary": (ctypes.c_int, [_vp, _i64, ctypes.c_double, ctypes.c_int, _vp, _vp, _sz, _i32, _i32,
                                      ctypes.POINTER(CsInfo), _vp]),
    "cossin_unitary_backward": (ctypes.c_int, [_i64, _i64, ctypes.c_double, _vp, _vp, _vp, _vp, _i32, _i32, _vp,
                                               _vp]),
    "cossin_batched_workspace_size": (ctypes.c_int, [_i64, _vp, ctypes.POINTER(_sz)]),
    "cossin_batched": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp, _vp]),
    "cossin_batched_plan_create": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp, _i32, _vp,
                                                  ctypes.POINTER(_vp)]),
    "cossin_batched_plan_launch": (ctypes.c_int, [_vp, _vp]),
    "cossin_batched_plan_info": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "cossin_batched_plan_destroy": (ctypes.c_int, [_vp]),
    "cossin_selftest_wait_timeout": (ctypes.c_int, [_vp]),
    "cossin_selftest_fail_next_alloc": (None, [_i32]),
    "cossin_fp64_fma_rate": (ctypes.c_int, [_i64, ctypes.POINTER(ctypes.c_double), _vp]),
    "cossin_fp64_product_launches": (ctypes.c_int, [_i64, _i64, _i64, ctypes.POINTER(ctypes.c_int32)]),
    "cossin_backward_workspace_size": (ctypes.c_int, [_i64, _i64, ctypes.c_int, _i32, ctypes.POINTER(_sz)]),
    "cossin_backward_ws": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_int, _vp, _sz,
                                          _vp, _vp]),
    "cossin_last_error": (ctypes.c_char_p, []),
    "cossin_device_status": (ctypes.c_int, [_vp]),
    "cossin_prof_enable": (None, [_i32]),
    "cossin_prof_reset": (None, []),
    "cossin_prof_read": (ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64),
                                        ctypes.POINTER(ctypes.c_double)]),
}


def lib():
    """The loaded library.  Raises if it has not been built: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError("libcossin.so is not built (%s); run "
                                   "`python -m paper_2010_00465_gb300.build`" % LIB)
            L = ctypes.CDLL(LIB)
            for name, (res, args) in SIGNATURES.items():
                if not hasattr(L, name):
                    continue
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != CS_OK:
        msg = lib().cossin_last_error()
        raise CossinError(status, msg.decode() if msg else "")
