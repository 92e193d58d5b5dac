"""The continuous-batching polymul server: every result equals the oracle's
product, and is the same when the request runs alone and inside a mix of
concurrent requests of other sizes; admission by memory, refusal,
cancellation of queued requests and host-injected batch failures."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, uniform_residues, serving_trace
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def make_requests(n, seed, dmax_log=14.0):
    tr = serving_trace(seed=seed, n=n, dmin_log=6.0, dmax_log=dmax_log)
    reqs = []
    for r in tr:
        a = uniform_residues(seed * 7919 + 2 * r["id"], r["na"], P_NTT30).astype(np.uint32)
        b = uniform_residues(seed * 7919 + 2 * r["id"] + 1, r["nb"], P_NTT30).astype(np.uint32)
        reqs.append((a, b))
    return reqs


def expected(a, b):
    o = oracle.get()
    if a.size * b.size <= 4_000_000:
        return o.polymul_schoolbook(P_NTT30, a, b)
    return o.polymul_ntt(P_NTT30, a, b)


def test_mix_equals_alone_equals_oracle():
    require_gpu()
    reqs = make_requests(60, seed=21)
    sv = ntt.Server(P_NTT30, max_coeffs=1 << 15, mem_budget_bytes=256 << 20, n_streams=4)
    try:
        # all at once: batches of mixed lengths overlap on the device
        outs_mix = [np.zeros(a.size + b.size - 1, dtype=np.uint32) for a, b in reqs]
        ids = []
        for (a, b), c in zip(reqs, outs_mix):
            rc, rid = sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)
            assert rc == 0
            ids.append(rid)
        assert sv.drain(60_000) == 0
        assert all(sv.poll(r) == 0 for r in ids)
        st = sv.stats()
        assert st.completed == len(reqs) and st.failed == 0
        assert st.batches < len(reqs), "requests were not batched"
        assert 0 < st.p50_us <= st.p99_us
        # one at a time
        for (a, b), cm in zip(reqs, outs_mix):
            c = np.zeros_like(cm)
            rc, rid = sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)
            assert rc == 0 and sv.wait(rid, 60_000) == 0
            assert np.array_equal(c, cm), "result differs alone and in the mix"
            assert np.array_equal(c.astype(np.uint64), expected(a, b))
    finally:
        sv.destroy()


def test_admission_by_memory_and_refusal():
    require_gpu()
    reqs = make_requests(40, seed=22, dmax_log=12.0)
    # budget for about two of the largest requests at a time
    sv = ntt.Server(P_NTT30, max_coeffs=1 << 13, mem_budget_bytes=2 * 2 * (1 << 14) * 4, n_streams=2)
    try:
        outs = [np.zeros(a.size + b.size - 1, dtype=np.uint32) for a, b in reqs]
        ids = [sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)[1]
               for (a, b), c in zip(reqs, outs)]
        big = np.ones(1 << 14, dtype=np.uint32)
        cbig = np.zeros(2 * big.size - 1, dtype=np.uint32)
        rc, rid_big = sv.submit(big.ctypes.data, big.size, big.ctypes.data, big.size, cbig.ctypes.data)
        assert rc == -10 and sv.poll(rid_big) == -10  # larger than max_coeffs and the budget
        assert sv.drain(60_000) == 0
        for (a, b), c, rid in zip(reqs, outs, ids):
            assert sv.poll(rid) == 0
            assert np.array_equal(c.astype(np.uint64), expected(a, b))
        assert sv.stats().refused == 1
    finally:
        sv.destroy()


def test_cancel_queued_and_injected_failure():
    require_gpu()
    reqs = make_requests(30, seed=23, dmax_log=12.0)
    sv = ntt.Server(P_NTT30, max_coeffs=1 << 13, mem_budget_bytes=2 * (1 << 14) * 4, n_streams=1, max_batch=1)
    try:
        sv.inject_failures(1)
        outs = [np.zeros(a.size + b.size - 1, dtype=np.uint32) for a, b in reqs]
        ids = [sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)[1]
               for (a, b), c in zip(reqs, outs)]
        cancelled = []
        for rid in ids[-5:]:
            if sv.cancel(rid) == 0:
                cancelled.append(rid)
        assert sv.drain(60_000) == 0
        statuses = [sv.poll(r) for r in ids]
        assert statuses.count(-13) == 1, statuses  # exactly the injected batch (max_batch = 1)
        assert statuses[0] == -13
        for (a, b), c, rid, s in zip(reqs, outs, ids, statuses):
            if rid in cancelled:
                assert s == -11
            elif s == 0:
                assert np.array_equal(c.astype(np.uint64), expected(a, b))
        assert sum(s == 0 for s in statuses) == len(ids) - 1 - len(cancelled)
    finally:
        sv.destroy()


def test_page_locked_buffers_gathered_by_kernels():
    """Operands and results in page-locked host memory are gathered into the
    slab and scattered back by kernels (no per-request copy calls); each result
    equals the oracle's product and the one from pageable buffers, and a batch
    that mixes page-locked and pageable requests takes the copy path."""
    torch = require_gpu()
    reqs = make_requests(40, seed=33)
    sv = ntt.Server(P_NTT30, max_coeffs=1 << 15, mem_budget_bytes=256 << 20, n_streams=4)
    try:
        pinned = []
        for a, b in reqs:
            ta = torch.from_numpy(a.view(np.int32)).pin_memory()
            tb = torch.from_numpy(b.view(np.int32)).pin_memory()
            tc = torch.zeros(a.size + b.size - 1, dtype=torch.int32).pin_memory()
            pinned.append((ta, tb, tc))
        ids = []
        for ta, tb, tc in pinned:
            rc, rid = sv.submit(ta.data_ptr(), ta.numel(), tb.data_ptr(), tb.numel(), tc.data_ptr())
            assert rc == 0
            ids.append(rid)
        assert sv.drain(60_000) == 0
        st = sv.stats()
        assert st.completed == len(reqs) and st.failed == 0
        assert st.direct_batches == st.batches > 0
        for (a, b), (_, _, tc) in zip(reqs, pinned):
            assert np.array_equal(tc.numpy().view(np.uint32).astype(np.uint64), expected(a, b))
        # the same requests from pageable memory: copy path, identical results
        sv.reset_stats()
        outs = [np.zeros(a.size + b.size - 1, dtype=np.uint32) for a, b in reqs]
        for (a, b), c in zip(reqs, outs):
            assert sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)[0] == 0
        assert sv.drain(60_000) == 0
        st = sv.stats()
        assert st.direct_batches == 0 and st.completed == len(reqs)
        for c, (_, _, tc) in zip(outs, pinned):
            assert np.array_equal(c, tc.numpy().view(np.uint32))
        # page-locked operands with a pageable result buffer: copy path
        sv.reset_stats()
        ta, tb, _ = pinned[0]
        c = np.zeros(ta.numel() + tb.numel() - 1, dtype=np.uint32)
        rc, rid = sv.submit(ta.data_ptr(), ta.numel(), tb.data_ptr(), tb.numel(), c.ctypes.data)
        assert rc == 0 and sv.wait(rid, 60_000) == 0
        assert sv.stats().direct_batches == 0
        assert np.array_equal(c, outs[0])
    finally:
        sv.destroy()


def test_full_degree_range_through_the_gather_scatter_path():
    """The serving workload's whole degree range (up to 2^20, i.e. 2^21-point
    products) through the page-locked gather/scatter path, mixed with small
    requests: every result equals the oracle's product."""
    torch = require_gpu()
    rng = np.random.default_rng(44)
    sizes = [((1 << 20) + 1, (1 << 20) + 1), ((1 << 19) + 1, (1 << 18) + 1), ((1 << 17) + 3, 65),
             (1000, (1 << 20) + 1)] + [(int(rng.integers(64, 4096)), int(rng.integers(64, 4096))) for _ in range(12)]
    reqs = []
    for i, (na, nb) in enumerate(sizes):
        a = uniform_residues(7700 + 2 * i, na, P_NTT30).astype(np.uint32)
        b = uniform_residues(7701 + 2 * i, nb, P_NTT30).astype(np.uint32)
        if i == 0:
            a[:] = P_NTT30 - 1  # the top of the input range, every coefficient
            b[:] = P_NTT30 - 1
        reqs.append((a, b))
    sv = ntt.Server(P_NTT30, max_coeffs=(1 << 20) + 1, mem_budget_bytes=1 << 30, n_streams=4)
    try:
        pinned = []
        for a, b in reqs:
            ta = torch.from_numpy(a.view(np.int32)).pin_memory()
            tb = torch.from_numpy(b.view(np.int32)).pin_memory()
            tc = torch.zeros(a.size + b.size - 1, dtype=torch.int32).pin_memory()
            pinned.append((ta, tb, tc))
        for ta, tb, tc in pinned:
            assert sv.submit(ta.data_ptr(), ta.numel(), tb.data_ptr(), tb.numel(), tc.data_ptr())[0] == 0
        assert sv.drain(120_000) == 0
        st = sv.stats()
        assert st.completed == len(reqs) and st.failed == 0 and st.direct_batches == st.batches
        o = oracle.get()
        for (a, b), (_, _, tc) in zip(reqs, pinned):
            want = o.polymul_ntt(P_NTT30, a, b) if a.size * b.size > 4_000_000 else o.polymul_schoolbook(P_NTT30, a, b)
            assert np.array_equal(tc.numpy().view(np.uint32).astype(np.uint64), want), (a.size, b.size)
    finally:
        sv.destroy()


def test_ntl_variant_server_matches_oracle():
    """A server whose transforms use the NTL-style butterflies (Algorithm 2):
    every product equals the oracle's, including operands of all p - 1 (the
    top of that butterfly's input interval); a variant it does not carry is
    refused at creation."""
    require_gpu()
    reqs = make_requests(40, seed=23)
    reqs[0] = (np.full(reqs[0][0].size, P_NTT30 - 1, dtype=np.uint32), np.full(reqs[0][1].size, P_NTT30 - 1, dtype=np.uint32))
    sv = ntt.Server(P_NTT30, max_coeffs=1 << 15, mem_budget_bytes=256 << 20, n_streams=4, variant=ntt.VARIANT_NTL)
    try:
        outs = [np.zeros(a.size + b.size - 1, dtype=np.uint32) for a, b in reqs]
        ids = []
        for (a, b), c in zip(reqs, outs):
            rc, rid = sv.submit(a.ctypes.data, a.size, b.ctypes.data, b.size, c.ctypes.data)
            assert rc == 0
            ids.append(rid)
        assert sv.drain(60_000) == 0
        assert all(sv.poll(r) == 0 for r in ids)
        for (a, b), c in zip(reqs, outs):
            assert np.array_equal(c.astype(np.uint64), expected(a, b))
    finally:
        sv.destroy()
    with pytest.raises(ntt.NTTError) as e:
        ntt.Server(P_NTT30, max_coeffs=1 << 10, mem_budget_bytes=64 << 20, variant=ntt.VARIANT_MONT)
    assert e.value.code == -4
