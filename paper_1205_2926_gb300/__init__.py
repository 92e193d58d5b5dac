"""GB300-native batched number-theoretic transform (Harvey, arXiv:1205.2926).

Thin Python layer over the C ABI of ``libntt_gb300.so``: it passes device
pointers (from torch tensors or raw integers), sizes and CUDA streams to the
library and turns status codes into exceptions.  Every transform step runs in
the library's CUDA kernels; importing this package does not load the library,
the first call does (and fails loudly if it is missing).

Names follow the C ABI: ``ntt_plan``, ``ntt_forward_batch``,
``ntt_inverse_batch``, ``ntt_transform_host``, ``polymul_mod_p``,
``ntt_execute_uneven``.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import NTTError, check

VARIANT_LAZY = 0
VARIANT_NTL = 1
VARIANT_MONT = 2
VARIANT_MOLLER = 3
P_MAX_W32 = 2654435769  # floor(2^32 / phi): Moeller's bound for 32-bit words
P_MAX_W64 = 11400714819323198485  # floor(2^64 / phi)


def _ptr(x) -> int:
    """Device address of a torch tensor (contiguous) or an int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"expected a device pointer or tensor, got {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def is_prime(n: int) -> bool:
    r = ctypes.c_int()
    check(_lib.load().ntt_is_prime(n, ctypes.byref(r)), "ntt_is_prime")
    return bool(r.value)


def root_of_unity(p: int, L: int) -> int:
    w = ctypes.c_uint64()
    check(_lib.load().ntt_root_of_unity(p, L, ctypes.byref(w)), "ntt_root_of_unity")
    return w.value


def find_prime(lo: int, k: int) -> int:
    q = ctypes.c_uint64()
    check(_lib.load().ntt_find_prime(lo, k, ctypes.byref(q)), "ntt_find_prime")
    return q.value


class Plan:
    """A device-resident plan for length-L transforms over F_p (ntt_plan, or
    ntt_plan_words when the word size is given)."""

    def __init__(self, p: int, omega: int, L: int, word_bytes: int | None = None):
        lib = _lib.load()
        h = ctypes.c_void_p()
        if word_bytes is None:
            check(lib.ntt_plan(ctypes.byref(h), p, omega, L), "ntt_plan")
        else:
            check(lib.ntt_plan_words(ctypes.byref(h), p, omega, L, word_bytes), "ntt_plan_words")
        self.handle = h.value
        self.p, self.omega, self.L = p, omega, L
        self.word_bytes = self.info().word_bytes

    def info(self) -> _lib.PlanInfo:
        info = _lib.PlanInfo()
        check(_lib.load().ntt_plan_get_info(self.handle, ctypes.byref(info)), "ntt_plan_get_info")
        return info

    def set_variant(self, variant: int) -> None:
        check(_lib.load().ntt_plan_set_variant(self.handle, variant), "ntt_plan_set_variant")

    def set_warp_rows(self, on: bool) -> None:
        """Row passes of 2^5..2^10 words: one warp per row (register blocks, shuffles)."""
        check(_lib.load().ntt_plan_set_warp_rows(self.handle, 1 if on else 0), "ntt_plan_set_warp_rows")

    def set_checked(self, on: bool) -> None:
        """Checked mode: transforms validate their input range first (NTT_ERR_INPUT)."""
        check(_lib.load().ntt_plan_set_checked(self.handle, 1 if on else 0), "ntt_plan_set_checked")

    def set_split(self, log_r) -> None:
        arr = (ctypes.c_int * len(log_r))(*log_r)
        check(_lib.load().ntt_plan_set_split(self.handle, len(log_r), arr), "ntt_plan_set_split")

    def autotune(self, batch: int, use_cache: bool = True) -> list:
        """Time every allowed pass split for this batch size, keep the fastest,
        then the row pass's body (CTA rows or one warp per row) for that split
        (both cached per GPU model and shape); returns the chosen split."""
        out = (ctypes.c_int * 4)()
        check(_lib.load().ntt_plan_autotune(self.handle, batch, int(use_cache), out), "ntt_plan_autotune")
        return [v for v in out if v][: self.info().n_passes]

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            check(_lib.load().ntt_plan_destroy(self.handle), "ntt_plan_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def ntt_plan(p: int, omega: int, L: int, word_bytes: int | None = None) -> Plan:
    return Plan(p, omega, L, word_bytes)


def ntt_forward_batch(plan: Plan, data, batch: int, stride_words: int | None = None, stream=None) -> None:
    stride = plan.L if stride_words is None else stride_words
    check(_lib.load().ntt_forward_batch(plan.handle, _ptr(data), batch, stride, _stream(stream)),
          "ntt_forward_batch")


def ntt_inverse_batch(plan: Plan, data, batch: int, stride_words: int | None = None, stream=None) -> None:
    stride = plan.L if stride_words is None else stride_words
    check(_lib.load().ntt_inverse_batch(plan.handle, _ptr(data), batch, stride, _stream(stream)),
          "ntt_inverse_batch")


def ntt_forward_dit_batch(plan: Plan, data, batch: int, stride_words: int | None = None, stream=None) -> None:
    """Forward transform, bit-reversed input to natural-order output."""
    stride = plan.L if stride_words is None else stride_words
    check(_lib.load().ntt_forward_dit_batch(plan.handle, _ptr(data), batch, stride, _stream(stream)),
          "ntt_forward_dit_batch")


def ntt_inverse_dif_batch(plan: Plan, data, batch: int, stride_words: int | None = None, stream=None) -> None:
    """Inverse transform (unnormalised), natural-order input to bit-reversed output."""
    stride = plan.L if stride_words is None else stride_words
    check(_lib.load().ntt_inverse_dif_batch(plan.handle, _ptr(data), batch, stride, _stream(stream)),
          "ntt_inverse_dif_batch")


def ntt_check_input(plan: Plan, inverse: bool, data, batch: int, stride_words: int | None = None,
                    stream=None) -> int:
    """First flat index of an input word outside the accepted range, or -1 (synchronous)."""
    stride = plan.L if stride_words is None else stride_words
    bad = ctypes.c_longlong()
    check(_lib.load().ntt_check_input(plan.handle, int(bool(inverse)), _ptr(data), batch, stride, _stream(stream),
                                      ctypes.byref(bad)), "ntt_check_input")
    return bad.value


def ntt_execute_step(plan: Plan, inverse: bool, step: int, data, batch: int, stride_words: int | None = None,
                     stream=None) -> None:
    """One pass (one kernel launch) of a transform; see the C header."""
    stride = plan.L if stride_words is None else stride_words
    check(_lib.load().ntt_execute_step(plan.handle, int(bool(inverse)), step, _ptr(data), batch, stride,
                                       _stream(stream)), "ntt_execute_step")


def ntt_transform_host(plan: Plan, inverse: bool, host_array, batch: int, stride_words: int | None = None,
                       stream=None) -> None:
    """Transform a host numpy array (or pinned torch tensor) in place."""
    stride = plan.L if stride_words is None else stride_words
    if hasattr(host_array, "ctypes"):
        addr = host_array.ctypes.data
    else:
        addr = host_array.data_ptr()
    check(_lib.load().ntt_transform_host(plan.handle, int(bool(inverse)), addr, batch, stride, _stream(stream)),
          "ntt_transform_host")


def polymul_mod_p(p: int, a, na: int, b, nb: int, c, stream=None) -> None:
    check(_lib.load().polymul_mod_p(p, _ptr(a), na, _ptr(b), nb, _ptr(c), _stream(stream)), "polymul_mod_p")


def bigint_mul(a, na: int, b, nb: int, c, stream=None) -> None:
    """c = a * b for integers as little-endian 32-bit limb arrays on the device
    (c has na + nb limbs); see the C header for the limits."""
    check(_lib.load().bigint_mul(_ptr(a), na, _ptr(b), nb, _ptr(c), _stream(stream)), "bigint_mul")


def polymul_mod_p_noalloc(plan: Plan, a, na: int, b, nb: int, c, stream=None) -> None:
    """polymul_mod_p with a plan made beforehand and the library's fixed device
    scratch: allocates nothing (see the C header for the limits)."""
    check(_lib.load().polymul_mod_p_noalloc(plan.handle, _ptr(a), na, _ptr(b), nb, _ptr(c), _stream(stream)),
          "polymul_mod_p_noalloc")


def _desc_array(descs):
    n = len(descs)
    arr = (_lib.Desc * n)()
    for i, (plan, data, inv) in enumerate(descs):
        arr[i].plan = plan.handle
        arr[i].d_data = _ptr(data)
        arr[i].inverse = int(bool(inv))
    return arr, n


def ntt_execute_uneven(descs, stream=None) -> None:
    """descs: sequence of (plan, device tensor or pointer, inverse flag)."""
    arr, n = _desc_array(descs)
    check(_lib.load().ntt_execute_uneven(arr, n, _stream(stream)), "ntt_execute_uneven")


def ntt_uneven_autotune(descs, use_cache: bool = True, stream=None) -> None:
    """Tune the pass split of each multi-pass length class of an uneven batch
    inside the persistent launch (applied to the plans, cached); see the C header."""
    arr, n = _desc_array(descs)
    check(_lib.load().ntt_uneven_autotune(arr, n, int(use_cache), _stream(stream)), "ntt_uneven_autotune")


def ntt_uneven_release() -> None:
    """Free every prepared uneven batch of the current device (see the C header)."""
    check(_lib.load().ntt_uneven_release(), "ntt_uneven_release")


def ntt_uneven_status() -> int:
    s = ctypes.c_int()
    check(_lib.load().ntt_uneven_status(ctypes.byref(s)), "ntt_uneven_status")
    return s.value


def ntt_uneven_set_wait_budget(cycles: int, stall_stage: int = -1) -> None:
    check(_lib.load().ntt_uneven_set_wait_budget(cycles, stall_stage), "ntt_uneven_set_wait_budget")


def ntt_pass_status(reset: bool = False) -> int:
    """Status word of the pass kernels on the current device (NTT_OK or NTT_ERR_TIMEOUT)."""
    s = ctypes.c_int()
    check(_lib.load().ntt_pass_status(1 if reset else 0, ctypes.byref(s)), "ntt_pass_status")
    return s.value


def ntt_pass_set_wait_budget(cycles: int, stall_bytes: int = 0) -> None:
    check(_lib.load().ntt_pass_set_wait_budget(cycles, stall_bytes), "ntt_pass_set_wait_budget")


class Server:
    """Continuous-batching polymul server (ntt_server_*); host arrays in and out."""

    def __init__(self, p: int, max_coeffs: int, mem_budget_bytes: int, n_streams: int = 4, max_batch: int = 256,
                 variant: int = 0):
        cfg = _lib.ServerConfig(p, max_coeffs, mem_budget_bytes, n_streams, max_batch, variant)
        h = ctypes.c_void_p()
        check(_lib.load().ntt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "ntt_server_create")
        self.handle = h.value
        self.p = p

    def submit(self, a_addr: int, na: int, b_addr: int, nb: int, c_addr: int) -> tuple[int, int]:
        """Queue c = a*b (host addresses); returns (status, request id)."""
        rid = ctypes.c_uint64()
        rc = _lib.load().ntt_server_submit(self.handle, a_addr, na, b_addr, nb, c_addr, ctypes.byref(rid))
        if rc not in (0, -10):
            check(rc, "ntt_server_submit")
        return rc, rid.value

    def poll(self, rid: int) -> int:
        s = ctypes.c_int()
        check(_lib.load().ntt_server_poll(self.handle, rid, ctypes.byref(s)), "ntt_server_poll")
        return s.value

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        s = ctypes.c_int()
        check(_lib.load().ntt_server_wait(self.handle, rid, timeout_ms, ctypes.byref(s)), "ntt_server_wait")
        return s.value

    def cancel(self, rid: int) -> int:
        return _lib.load().ntt_server_cancel(self.handle, rid)

    def drain(self, timeout_ms: int = -1) -> int:
        return _lib.load().ntt_server_drain(self.handle, timeout_ms)

    def stats(self) -> _lib.ServerStats:
        st = _lib.ServerStats()
        check(_lib.load().ntt_server_stats(self.handle, ctypes.byref(st)), "ntt_server_stats")
        return st

    def reset_stats(self) -> None:
        check(_lib.load().ntt_server_reset_stats(self.handle), "ntt_server_reset_stats")

    def inject_failures(self, n_batches: int) -> None:
        check(_lib.load().ntt_server_inject_failures(self.handle, n_batches), "ntt_server_inject_failures")

    def destroy(self) -> None:
        if getattr(self, "handle", None):
            check(_lib.load().ntt_server_destroy(self.handle), "ntt_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
