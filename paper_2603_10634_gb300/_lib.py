"""ctypes loader for libozk2.so (the C ABI of include/ozk2.h).

Loading fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libozk2.so")

c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_void_p = ctypes.c_void_p
c_size_t = ctypes.c_size_t

# name -> (restype, argtypes); mirrors include/ozk2.h
SIGNATURES = {
    "ozk2_dgemm": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int, c_void_p]),
    "ozk2_workspace_size": (c_size_t, [c_i64, c_i64, c_i64, c_int]),
    "ozk2_dgemm_ws": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int,
                              c_void_p, c_size_t, c_void_p]),
    "ozk2_dgemm_noalloc": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int,
                                   c_void_p]),
    "ozk2_dgemm_ex": (c_int, [c_int, c_int, c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64,
                              c_int, c_int, c_i64, c_i64, c_void_p, c_size_t, c_void_p]),
    "ozk2_workspace_size_ex": (c_size_t, [c_i64, c_i64, c_i64, c_int, c_int, c_i64, c_i64]),
    "ozk2_dgemm_host": (c_int, [c_int, c_int, c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64,
                                c_int, c_int, c_void_p, c_size_t, c_void_p]),
    "ozk2_dgemm_host_ex": (c_int, [c_int, c_int, c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p,
                                   c_i64, c_int, c_int, ctypes.c_uint, c_void_p, c_size_t, c_void_p]),
    "ozk2_workspace_size_host": (c_size_t, [c_i64, c_i64, c_i64, c_int, c_int]),
    "ozk2_debug_scales_ex": (c_int, [c_int, c_int, c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int, c_int,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
    "ozk2_workspace_size_batched": (c_size_t, [c_int, c_void_p, c_void_p, c_void_p, c_int, c_int]),
    "ozk2_batch_plan_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p, c_size_t, c_void_p]),
    "ozk2_batch_plan_execute": (c_int, [c_void_p, c_void_p]),
    "ozk2_batch_plan_workspace": (c_void_p, [c_void_p]),
    "ozk2_batch_plan_destroy": (None, [c_void_p]),
    "ozk2_dgemm_batched": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_int, c_int, c_void_p, c_size_t, c_void_p]),
    "ozk2_debug_timeline": (c_int, [c_void_p, c_int]),
    "ozk2_noalloc_device_status": (c_int, [c_void_p]),
    "ozk2_dgemm_backward": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64,
                                    c_void_p, c_i64, c_void_p, c_i64, c_int, c_void_p, c_size_t, c_void_p,
                                    c_size_t, c_void_p]),
    "ozk2_workspace_size_backward": (c_size_t, [c_i64, c_i64, c_i64, c_int]),
    "ozk2_debug_backward_exponents": (c_int, [c_i64, c_i64, c_i64, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ozk2_set_wait_limit": (ctypes.c_uint64, [ctypes.c_uint64]),
    "ozk2_set_tile_n": (c_int, [c_int]),
    "ozk2_batch_plan_tile_n": (c_int, [c_void_p]),
    "ozk2_set_square_split": (c_i64, [c_i64]),
    "ozk2_debug_inject_fault": (c_int, [c_int]),
    "ozk2_status_string": (ctypes.c_char_p, [c_int]),
    "ozk2_device_status": (c_int, [c_void_p, c_void_p]),
    "ozk2_moduli": (c_int, [c_int, ctypes.POINTER(ctypes.c_int32)]),
    "ozk2_set_timing": (None, [c_int]),
    "ozk2_get_timing": (c_int, [ctypes.POINTER(ctypes.c_float), c_int]),
    "ozk2_last_launch_count": (c_int, []),
    "ozk2_debug_fp8_gemm": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_void_p, c_i64,
                                    c_void_p]),
    "ozk2_debug_scales": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p]),
    "ozk2_debug_residue_planes": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ozk2_debug_residue_products": (c_int, [c_i64, c_i64, c_i64, c_void_p, c_i64, c_void_p, c_i64, c_int,
                                            c_void_p, c_void_p, c_void_p, c_void_p]),
    "ozk2_debug_crt": (c_int, [c_i64, c_i64, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_i64, c_void_p]),
}

STATUS = {
    0: "OZK2_OK", 1: "OZK2_ERR_INVALID_VALUE", 2: "OZK2_ERR_UNSUPPORTED", 3: "OZK2_ERR_ALLOC",
    4: "OZK2_ERR_CUDA", 5: "OZK2_ERR_INTERNAL", 6: "OZK2_ERR_TIMEOUT", 7: "OZK2_ERR_NONFINITE",
    8: "OZK2_ERR_RANGE",
}

_lib = None


class Ozk2Error(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where} failed: {STATUS.get(status, status)}")


def load(path: str | None = None):
    """Load libozk2.so once and attach the C signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libozk2.so not found at {p}; build it with "
                          f"`python -m paper_2603_10634_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status, where):
    if status != 0:
        raise Ozk2Error(status, where)
