"""ctypes binding of ``libntt_gb300.so`` (the C ABI in include/ntt_gb300.h).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing -- there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libntt_gb300.so")

_lock = threading.Lock()
_lib = None

c_u64 = ctypes.c_uint64
c_size = ctypes.c_size_t
c_int = ctypes.c_int
c_void_p = ctypes.c_void_p


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("p", c_u64), ("omega", c_u64), ("omega_inv", c_u64), ("L", c_u64), ("L_inv", c_u64),
        ("log_L", c_int), ("word_bytes", c_int), ("variant", c_int), ("n_passes", c_int),
        ("log_r", c_int * 4),
        ("table_bytes", c_u64),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("p", c_u64), ("max_coeffs", c_size), ("mem_budget_bytes", c_size), ("n_streams", c_int),
                ("max_batch", c_int), ("variant", c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", c_u64), ("refused", c_u64), ("cancelled", c_u64), ("failed", c_u64),
                ("batches", c_u64), ("butterflies", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("direct_batches", c_u64)]


class Desc(ctypes.Structure):
    _fields_ = [("plan", c_void_p), ("d_data", c_void_p), ("inverse", c_int)]


_SIGNATURES = {
    "ntt_version": (c_int, []),
    "ntt_strerror": (ctypes.c_char_p, [c_int]),
    "ntt_last_cuda_error": (ctypes.c_char_p, []),
    "ntt_is_prime": (c_int, [c_u64, ctypes.POINTER(c_int)]),
    "ntt_root_of_unity": (c_int, [c_u64, c_u64, ctypes.POINTER(c_u64)]),
    "ntt_find_prime": (c_int, [c_u64, c_int, ctypes.POINTER(c_u64)]),
    "ntt_plan": (c_int, [ctypes.POINTER(c_void_p), c_u64, c_u64, c_u64]),
    "ntt_plan_words": (c_int, [ctypes.POINTER(c_void_p), c_u64, c_u64, c_u64, c_int]),
    "ntt_plan_destroy": (c_int, [c_void_p]),
    "ntt_plan_set_variant": (c_int, [c_void_p, c_int]),
    "ntt_plan_set_checked": (c_int, [c_void_p, c_int]),
    "ntt_plan_set_warp_rows": (c_int, [c_void_p, c_int]),
    "ntt_selftest_geometry": (c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.c_char_p, c_int]),
    "ntt_check_input": (c_int, [c_void_p, c_int, c_void_p, c_size, c_size, c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "ntt_plan_get_info": (c_int, [c_void_p, ctypes.POINTER(PlanInfo)]),
    "ntt_plan_set_split": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "ntt_plan_autotune": (c_int, [c_void_p, c_size, c_int, ctypes.POINTER(c_int)]),
    "ntt_forward_batch": (c_int, [c_void_p, c_void_p, c_size, c_size, c_void_p]),
    "ntt_forward_dit_batch": (c_int, [c_void_p, c_void_p, c_size, c_size, c_void_p]),
    "ntt_inverse_dif_batch": (c_int, [c_void_p, c_void_p, c_size, c_size, c_void_p]),
    "ntt_inverse_batch": (c_int, [c_void_p, c_void_p, c_size, c_size, c_void_p]),
    "ntt_execute_step": (c_int, [c_void_p, c_int, c_int, c_void_p, c_size, c_size, c_void_p]),
    "ntt_transform_host": (c_int, [c_void_p, c_int, c_void_p, c_size, c_size, c_void_p]),
    "polymul_mod_p": (c_int, [c_u64, c_void_p, c_size, c_void_p, c_size, c_void_p, c_void_p]),
    "bigint_mul": (c_int, [c_void_p, c_size, c_void_p, c_size, c_void_p, c_void_p]),
    "polymul_mod_p_noalloc": (c_int, [c_void_p, c_void_p, c_size, c_void_p, c_size, c_void_p, c_void_p]),
    "ntt_execute_uneven": (c_int, [ctypes.POINTER(Desc), c_size, c_void_p]),
    "ntt_uneven_autotune": (c_int, [ctypes.POINTER(Desc), c_size, c_int, c_void_p]),
    "ntt_uneven_release": (c_int, []),
    "ntt_uneven_status": (c_int, [ctypes.POINTER(c_int)]),
    "ntt_uneven_set_wait_budget": (c_int, [ctypes.c_longlong, c_int]),
    "ntt_pass_status": (c_int, [c_int, ctypes.POINTER(c_int)]),
    "ntt_pass_set_wait_budget": (c_int, [ctypes.c_longlong, ctypes.c_uint]),
    "ntt_server_create": (c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(c_void_p)]),
    "ntt_server_submit": (c_int, [c_void_p, c_void_p, c_size, c_void_p, c_size, c_void_p,
                                  ctypes.POINTER(c_u64)]),
    "ntt_server_poll": (c_int, [c_void_p, c_u64, ctypes.POINTER(c_int)]),
    "ntt_server_wait": (c_int, [c_void_p, c_u64, c_int, ctypes.POINTER(c_int)]),
    "ntt_server_cancel": (c_int, [c_void_p, c_u64]),
    "ntt_server_drain": (c_int, [c_void_p, c_int]),
    "ntt_server_stats": (c_int, [c_void_p, ctypes.POINTER(ServerStats)]),
    "ntt_server_reset_stats": (c_int, [c_void_p]),
    "ntt_server_inject_failures": (c_int, [c_void_p, c_int]),
    "ntt_server_destroy": (c_int, [c_void_p]),
}


def exported_symbols():
    """Names the C ABI declares (used by the export test)."""
    return list(_SIGNATURES)


def load(path: str | None = None):
    """Load the library (once).  Raises OSError if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"{p} not found: build it with paper_1205_2926_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class NTTError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.ntt_strerror(code).decode()
        if code == -5:
            msg += " (" + lib.ntt_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg} [{code}]")
        self.code = code


def check(code: int, where: str) -> None:
    if code != 0:
        raise NTTError(code, where)
