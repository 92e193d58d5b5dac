"""CPU oracle for the number-theoretic transform over F_p.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library under
``paper_1205_2926_gb300`` never does, and this package never imports it.

The arithmetic lives in ``ntt_oracle.c`` (plain C, fully reduced ``%`` on
128-bit products, no lazy reduction).  This module compiles it with gcc on
first use and wraps it for numpy ``uint64`` arrays.

Functions and the passages they follow (Harvey, arXiv:1205.2926):

* ``dft_naive`` / ``idft_naive``  -- Section 1 definition of the NTT, placed in
  Algorithm 1's bit-reversed order; the inverse of Section 4 (unnormalised).
* ``dft_at`` -- one output position from the definition (O(L)).
* ``ntt_ref`` / ``intt_ref``      -- Algorithm 1, and Algorithm 1 run backwards.
* ``polymul_schoolbook`` / ``polymul_ntt`` -- the polynomial-multiplication
  application of Section 1 (definition, and the convolution theorem).
* ``is_prime``, ``smallest_qnr``, ``find_prime_above``, ``root_of_unity`` --
  number theory that names the primes p = 1 mod L and the roots omega.
* ``bigint_mul`` -- the large-integer application of Section 1: the product
  of two integers given as little-endian 32-bit limbs, by Python's exact
  integer arithmetic (the definition; no transform involved).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ntt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}

_u64 = ctypes.c_uint64
_p64 = ctypes.POINTER(ctypes.c_uint64)


def so_path(mutant: int = 0) -> str:
    name = "libntt_oracle.so" if mutant == 0 else f"libntt_oracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or a planted-mistake variant) with gcc; return the .so path."""
    out = so_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        lib = _libs.get(mutant)
        if lib is not None:
            return lib
        lib = ctypes.CDLL(build(mutant))
        for name, res, args in [
            ("or_powmod", _u64, [_u64, _u64, _u64]),
            ("or_invmod", _u64, [_u64, _u64]),
            ("or_bitrev", _u64, [_u64, ctypes.c_int]),
            ("or_is_prime", ctypes.c_int, [_u64]),
            ("or_smallest_qnr", _u64, [_u64]),
            ("or_find_prime_above", _u64, [_u64, ctypes.c_int]),
            ("or_root_of_unity", _u64, [_u64, _u64]),
            ("or_dft_naive", None, [_u64, _u64, _u64, _p64, _p64]),
            ("or_idft_naive", None, [_u64, _u64, _u64, _p64, _p64]),
            ("or_ntt_ref", None, [_u64, _u64, _u64, _p64]),
            ("or_intt_ref", None, [_u64, _u64, _u64, _p64]),
            ("or_ntt_ref_batch", None, [_u64, _u64, _u64, _p64, _u64, _u64]),
            ("or_intt_ref_batch", None, [_u64, _u64, _u64, _p64, _u64, _u64]),
            ("or_polymul_schoolbook", None, [_u64, _p64, _u64, _p64, _u64, _p64]),
            ("or_polymul_ntt", ctypes.c_int, [_u64, _p64, _u64, _p64, _u64, _p64]),
            ("or_dft_at", _u64, [_u64, _u64, _u64, _p64, _u64]),
        ]:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[mutant] = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_p64)


def _as_u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


class Oracle:
    """Bound view of one oracle build (``mutant=0`` is the real oracle)."""

    def __init__(self, mutant: int = 0):
        self.mutant = mutant
        self.lib = _load(mutant)

    # number theory -------------------------------------------------------
    def powmod(self, a: int, e: int, p: int) -> int:
        return int(self.lib.or_powmod(a, e, p))

    def invmod(self, a: int, p: int) -> int:
        return int(self.lib.or_invmod(a, p))

    def bitrev(self, k: int, l: int) -> int:
        return int(self.lib.or_bitrev(k, l))

    def is_prime(self, n: int) -> bool:
        return bool(self.lib.or_is_prime(n))

    def smallest_qnr(self, p: int) -> int:
        return int(self.lib.or_smallest_qnr(p))

    def find_prime_above(self, lo: int, k: int) -> int:
        return int(self.lib.or_find_prime_above(lo, k))

    def root_of_unity(self, p: int, L: int) -> int:
        return int(self.lib.or_root_of_unity(p, L))

    # transforms ----------------------------------------------------------
    def dft_naive(self, p: int, w: int, a) -> np.ndarray:
        a = _as_u64(a)
        out = np.empty_like(a)
        self.lib.or_dft_naive(p, w, a.size, _ptr(a), _ptr(out))
        return out

    def idft_naive(self, p: int, w: int, y) -> np.ndarray:
        y = _as_u64(y)
        out = np.empty_like(y)
        self.lib.or_idft_naive(p, w, y.size, _ptr(y), _ptr(out))
        return out

    def ntt_ref(self, p: int, w: int, a) -> np.ndarray:
        """Algorithm 1 on each row of ``a`` (1-D or 2-D); returns a new array."""
        x = _as_u64(a).copy()
        if x.ndim == 1:
            self.lib.or_ntt_ref(p, w, x.size, _ptr(x))
        else:
            self.lib.or_ntt_ref_batch(p, w, x.shape[1], _ptr(x), x.shape[0], x.shape[1])
        return x

    def intt_ref(self, p: int, w: int, y) -> np.ndarray:
        """Algorithm 1 run backwards (unnormalised) on each row of ``y``."""
        x = _as_u64(y).copy()
        if x.ndim == 1:
            self.lib.or_intt_ref(p, w, x.size, _ptr(x))
        else:
            self.lib.or_intt_ref_batch(p, w, x.shape[1], _ptr(x), x.shape[0], x.shape[1])
        return x

    def dft_at(self, p: int, w: int, a, k: int) -> int:
        """Output position k of the forward transform (definition, O(L))."""
        a = _as_u64(a)
        return int(self.lib.or_dft_at(p, w, a.size, _ptr(a), k))

    def polymul_schoolbook(self, p: int, a, b) -> np.ndarray:
        a, b = _as_u64(a), _as_u64(b)
        n = a.size + b.size - 1 if a.size and b.size else 0
        c = np.zeros(n, dtype=np.uint64)
        if n:
            self.lib.or_polymul_schoolbook(p, _ptr(a), a.size, _ptr(b), b.size, _ptr(c))
        return c

    def polymul_ntt(self, p: int, a, b) -> np.ndarray:
        a, b = _as_u64(a), _as_u64(b)
        n = a.size + b.size - 1 if a.size and b.size else 0
        c = np.zeros(n, dtype=np.uint64)
        if n:
            rc = self.lib.or_polymul_ntt(p, _ptr(a), a.size, _ptr(b), b.size, _ptr(c))
            if rc != 0:
                raise ValueError(f"no root of unity of length nextpow2({n}) mod {p}")
        return c


_default: Oracle | None = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(0)
    return _default


def dft_naive(p, w, a):
    return get().dft_naive(p, w, a)


def idft_naive(p, w, y):
    return get().idft_naive(p, w, y)


def ntt_ref(p, w, a):
    return get().ntt_ref(p, w, a)


def intt_ref(p, w, y):
    return get().intt_ref(p, w, y)


def polymul_schoolbook(p, a, b):
    return get().polymul_schoolbook(p, a, b)


def polymul_ntt(p, a, b):
    return get().polymul_ntt(p, a, b)


def root_of_unity(p, L):
    return get().root_of_unity(p, L)


def limbs_to_int(limbs) -> int:
    """Little-endian 32-bit limbs -> Python integer."""
    return int.from_bytes(np.asarray(limbs, dtype="<u4").tobytes(), "little")


def int_to_limbs(v: int, n: int) -> np.ndarray:
    """Python integer (0 <= v < 2^(32 n)) -> n little-endian 32-bit limbs."""
    return np.frombuffer(v.to_bytes(4 * n, "little"), dtype="<u4").astype(np.uint32)


def bigint_mul(a, b) -> np.ndarray:
    """Product of two integers given as little-endian 32-bit limb arrays, as
    len(a) + len(b) limbs (Section 1's large-integer application, computed
    from the definition with exact integers)."""
    na, nb = len(a), len(b)
    return int_to_limbs(limbs_to_int(a) * limbs_to_int(b), na + nb)
