"""The C-ABI library loads without a GPU and exports every function that
include/ntt_gb300.h declares (no compute calls)."""
import os
import re

import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return names


def test_library_exports_declared_symbols():
    b.build()
    lib = ntt._lib.load()
    names = declared_functions()
    assert "ntt_plan" in names and "polymul_mod_p" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert lib.ntt_version() >= 100
    assert lib.ntt_strerror(-3).decode().startswith("omega")


def test_binding_covers_declared_symbols():
    names = set(declared_functions())
    assert names <= set(ntt._lib.exported_symbols()), names - set(ntt._lib.exported_symbols())


def test_wait_hooks_validate_arguments_without_a_gpu():
    """The failure-detection hooks are host-only setters: they validate their
    arguments and need no device (the GPU tests use them to make a wait run out)."""
    b.build()
    lib = ntt._lib.load()
    assert lib.ntt_pass_set_wait_budget(0, 0) == -4          # budget must be positive
    assert lib.ntt_pass_set_wait_budget(1000, 8) == -4       # stall bytes: multiples of 16
    assert lib.ntt_pass_set_wait_budget(1000, 1 << 17) == -4  # at most 65536
    assert lib.ntt_pass_set_wait_budget(1000, 16) == 0
    assert lib.ntt_pass_set_wait_budget(2_000_000_000, 0) == 0  # back to normal waits
    assert lib.ntt_uneven_set_wait_budget(0, -1) == -4
    assert lib.ntt_uneven_set_wait_budget(2_000_000_000, -1) == 0


def test_launch_geometry_self_test_without_a_gpu():
    """The library's host-side geometry self-test: every allowed split of every
    length 2^3..2^26, both word sizes, batches 1..16384 -- tiles cover the data
    exactly once, sub-tiles are contiguous thread blocks, shared buffers match
    the kernels' layout and fit, tensor-copy boxes are well formed."""
    import ctypes
    b.build()
    lib = ntt._lib.load()
    n = ctypes.c_longlong()
    msg = ctypes.create_string_buffer(256)
    rc = lib.ntt_selftest_geometry(ctypes.byref(n), msg, 256)
    assert rc == 0, msg.value.decode()
    assert n.value > 10_000
    assert lib.ntt_selftest_geometry(None, None, 0) == -4
