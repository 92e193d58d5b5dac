"""polymul_mod_p_noalloc: the polynomial product for callers that cannot
allocate device memory while they run (their memory belongs to another
allocator, or the call sits on a latency-critical path where an allocation
could block or fail).  It works in a fixed device scratch array and must give
exactly what polymul_mod_p gives.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test."""
import ctypes

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
