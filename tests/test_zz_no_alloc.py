"""polymul_mod_p_noalloc: the polynomial product for callers that cannot
allocate device memory while they run (their memory belongs to another
allocator, or the call sits on a latency-critical path where an allocation
could block or fail).  It works in a fixed device scratch array and must give
exactly what polymul_mod_p gives.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, uniform_residues, word_dtype
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _next_pow2(n):
    L = 2
    while L < n:
        L <<= 1
    return L


def _zeros(n, dt, torch):
    return torch.zeros(n, dtype=torch.int32 if dt == np.uint32 else torch.int64, device="cuda")


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
def test_noalloc_matches_polymul_on_two_calls_in_a_row(p):
    torch = require_gpu()
    lib = ntt._lib.load()
    dt = word_dtype(p)
    # A large product first, then a small one: the second call must not see
    # anything the first one left in the shared scratch array.
    for call, (na, nb) in enumerate([(150_000, 200_001), (97, 31)]):
        L = _next_pow2(na + nb - 1)
        plan = ntt.ntt_plan(p, ntt.root_of_unity(p, L), L)
        a = uniform_residues(1000 + call, na, p).astype(dt)
        b = uniform_residues(2000 + call, nb, p).astype(dt)
        da, db = to_dev(a, torch), to_dev(b, torch)
        want = _zeros(na + nb - 1, dt, torch)
        ntt.polymul_mod_p(p, da, na, db, nb, want)
        got = _zeros(na + nb - 1, dt, torch)
        rc = lib.polymul_mod_p_noalloc(plan.handle, da.data_ptr(), na, db.data_ptr(), nb, got.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
        assert rc == 0, lib.ntt_strerror(rc)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(got, dt), from_dev(want, dt)), f"call {call}: differs from polymul_mod_p"
        plan.destroy()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = require_gpu()
    lib = ntt._lib.load()
    p = P_NTT30
    L = 1 << 21  # 2 * L * 4 bytes = 16 MiB > 8 MiB of scratch
    plan = ntt.ntt_plan(p, ntt.root_of_unity(p, L), L)
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = lib.polymul_mod_p_noalloc(plan.handle, d.data_ptr(), 4, d.data_ptr(), 4, d.data_ptr(), None)
    assert rc == -9  # NTT_ERR_RANGE
    small = ntt.ntt_plan(p, ntt.root_of_unity(p, 8), 8)
    rc = lib.polymul_mod_p_noalloc(small.handle, d.data_ptr(), 5, d.data_ptr(), 5, d.data_ptr(), None)
    assert rc == -2  # NTT_ERR_LENGTH: 9 coefficients do not fit a length-8 plan
    plan.destroy()
    small.destroy()


# Run in a fresh process with eager module loading, so that the library's
# code and its __device__ arrays are in device memory once the runtime starts
# (before the measurement), and without torch, whose allocator would reserve
# memory of its own.  Buffers come from cudaMalloc of the test itself; the
# library is called only through its C ABI.
_FRESH = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1205_2926_gb300 import _lib
from paper_1205_2926_gb300.inputs import uniform_residues, word_dtype
lib = _lib.load()
rt = None
for name in ("libcudart.so.13", "libcudart.so"):
    try:
        rt = ctypes.CDLL(name)
        break
    except OSError:
        pass
assert rt is not None, "libcudart not found"
vp, sz = ctypes.c_void_p, ctypes.c_size_t
rt.cudaMalloc.argtypes = [ctypes.POINTER(vp), sz]
rt.cudaMemcpy.argtypes = [vp, vp, sz, ctypes.c_int]
rt.cudaMemGetInfo.argtypes = [ctypes.POINTER(sz), ctypes.POINTER(sz)]
def ok(e, what):
    assert e == 0, f"{what}: CUDA error {e}"
def free_bytes():
    f, t = sz(), sz()
    ok(rt.cudaDeviceSynchronize(), "sync")
    ok(rt.cudaMemGetInfo(ctypes.byref(f), ctypes.byref(t)), "cudaMemGetInfo")
    return f.value
def dev_array(host):
    d = vp()
    ok(rt.cudaMalloc(ctypes.byref(d), max(host.nbytes, 16)), "cudaMalloc")
    ok(rt.cudaMemcpy(d, host.ctypes.data, host.nbytes, 1), "H2D")
    return d
def to_host(d, n, dt):
    h = np.zeros(n, dtype=dt)
    ok(rt.cudaMemcpy(h.ctypes.data, d, h.nbytes, 2), "D2H")
    return h
p = int(sys.argv[2])
dt = word_dtype(p)
ok(rt.cudaSetDevice(0), "cudaSetDevice")
report = {"calls": []}
for call, (na, nb) in enumerate([(3000, 5001), (97, 31)]):
    a = uniform_residues(7000 + call, na, p).astype(dt)
    b = uniform_residues(8000 + call, nb, p).astype(dt)
    n = na + nb - 1
    L = 2
    while L < n:
        L *= 2
    da, db = dev_array(a), dev_array(b)
    dc, dref = dev_array(np.zeros(n, dtype=dt)), dev_array(np.zeros(n, dtype=dt))
    w = ctypes.c_uint64()
    ok(lib.ntt_root_of_unity(p, L, ctypes.byref(w)), "root")
    plan = vp()
    rc = lib.ntt_plan(ctypes.byref(plan), p, w.value, L)  # set-up: may allocate (its tables)
    assert rc == 0, rc
    before = free_bytes()
    rc = lib.polymul_mod_p_noalloc(plan, da, na, db, nb, dc, None)
    after = free_bytes()
    assert rc == 0, lib.ntt_strerror(rc)
    got = to_host(dc, n, dt)
    rc = lib.polymul_mod_p(p, da, na, db, nb, dref, None)  # the existing entry point, afterwards
    assert rc == 0, rc
    want = to_host(dref, n, dt)
    report["calls"].append({"na": na, "nb": nb, "free_before": before, "free_after": after,
                            "equal": bool(np.array_equal(got, want)),
                            "got": [int(x) for x in got[:8]], "want": [int(x) for x in want[:8]]})
    lib.ntt_plan_destroy(plan)
print(json.dumps(report))
"""


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
def test_noalloc_first_call_in_a_fresh_process_allocates_nothing(p):
    """The first transform work a process ever does is a polymul_mod_p_noalloc
    call (after its plan was made at set-up): the device's free memory is the
    same before and after each of two calls in a row, and the results equal
    polymul_mod_p's (called afterwards)."""
    require_gpu()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, root, str(p)], capture_output=True, text=True, env=env,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    report = json.loads(r.stdout.strip().splitlines()[-1])
    for i, c in enumerate(report["calls"]):
        assert c["equal"], f"call {i}: differs from polymul_mod_p ({c['got']} vs {c['want']})"
        assert c["free_after"] == c["free_before"], \
            f"call {i} changed the device's free memory by {c['free_before'] - c['free_after']} bytes"
