"""Row passes with one warp per row (ntt_plan_set_warp_rows: register blocks of
R/32 words per thread, one warp-private transpose, lane exchanges by
shuffles) give Algorithm 1's results bit for bit: every row length 2^5..2^10,
alone (single-pass transforms) and as the last pass of longer transforms
(several splits), every variant, both word sizes, padded strides whose padding
must stay untouched, inputs at the top of each butterfly's interval, DIT/DIF."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, batch_inputs, uniform_residues, word_dtype
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

P32M = 2649751553  # Moeller's range, 32-bit words (ntt_plan_words)


def run(plan, rows, inverse, torch, dt):
    batch, L = rows.shape
    per16 = 16 // np.dtype(dt).itemsize
    stride = L + per16
    buf = np.full((batch, stride), np.iinfo(dt).max, dtype=dt)
    buf[:, :L] = rows.astype(dt)
    d = to_dev(buf, torch)
    (ntt.ntt_inverse_batch if inverse else ntt.ntt_forward_batch)(plan, d, batch, stride)
    torch.cuda.synchronize()
    out = from_dev(d, dt).reshape(batch, stride)
    assert np.all(out[:, L:] == np.iinfo(dt).max), "wrote into the padding"
    return out[:, :L].astype(np.uint64)


def variants_for(p, wb):
    if p == P32M:
        return [3]
    return [0, 1, 2, 3]


@pytest.mark.parametrize("p,wb", [(P_NTT30, None), (P_NTT62, None), (P32M, 4)])
@pytest.mark.parametrize("logL,split", [(5, None), (6, None), (7, None), (8, None), (9, None), (10, None),
                                        (11, [6, 5]), (12, [6, 6]), (13, [6, 7]), (14, [6, 8]), (15, [6, 9]),
                                        (16, [6, 10]), (16, [8, 8]), (17, [7, 10]), (20, [6, 6, 8])])
def test_warp_rows_match_oracle(p, wb, logL, split):
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    if (p - 1) % L:
        pytest.skip("L does not divide p-1")
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L, word_bytes=wb)
    if split is not None:
        plan.set_split(split)
    plan.set_warp_rows(True)
    dt = np.uint32 if plan.word_bytes == 4 else np.uint64
    batch = 5 if logL <= 14 else 2
    try:
        for v in variants_for(p, wb):
            plan.set_variant(v)
            top_f = p - 1 if v in (1, 3) else 2 * p - 1
            top_i = p - 1 if v in (1, 3) else 4 * p - 1
            a = batch_inputs(2100 + logL, batch, L, p).astype(np.uint64)
            a[0, :] = top_f
            got = run(plan, a, False, torch, dt)
            assert np.array_equal(got, o.ntt_ref(p, w, a % np.uint64(p))), f"forward variant {v}"
            y = batch_inputs(2200 + logL, batch, L, p).astype(np.uint64)
            y[0, :] = top_i
            got = run(plan, y, True, torch, dt)
            assert np.array_equal(got, o.intt_ref(p, w, y % np.uint64(p))), f"inverse variant {v}"
    finally:
        plan.destroy()


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
@pytest.mark.parametrize("logL", [7, 10, 14])
def test_warp_rows_dit_dif_and_setting_off(p, logL):
    """The orders-swapped transforms with warp rows, and switching back to the
    radix-8 rows gives the same results."""
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    w = o.root_of_unity(p, L)
    wi = o.invmod(w, p)
    dt = word_dtype(p)
    plan = ntt.ntt_plan(p, w, L)
    x = batch_inputs(2300 + logL, 3, L, p)
    outs = []
    for on in (True, False):
        plan.set_warp_rows(on)
        d = to_dev(x, torch)
        ntt.ntt_forward_dit_batch(plan, d, 3)
        torch.cuda.synchronize()
        got = from_dev(d, dt).reshape(3, L).astype(np.uint64)
        assert np.array_equal(got, o.intt_ref(p, wi, x.astype(np.uint64))), "DIT forward"
        d = to_dev(x, torch)
        ntt.ntt_inverse_dif_batch(plan, d, 3)
        torch.cuda.synchronize()
        got2 = from_dev(d, dt).reshape(3, L).astype(np.uint64)
        assert np.array_equal(got2, o.ntt_ref(p, wi, x.astype(np.uint64))), "DIF inverse"
        outs.append((got, got2))
    plan.destroy()


def group_rows(wb, logR):
    """Rows per warp of the batched warp-row kernel (several rows once a pass has
    at least that many times 2 x 8 x 152 rows): up to 32 (32-bit) or 16 (64-bit)
    words per thread, at most 8 rows."""
    n = (1 << logR) // 32
    words = 32 if wb == 4 else 16
    return 1 if n >= words else min(8, words // n)


@pytest.mark.parametrize("p,wb", [(P_NTT30, None), (P_NTT62, None), (P32M, 4)])
@pytest.mark.parametrize("logR", [5, 6, 7, 8, 9])
@pytest.mark.parametrize("last_of", [0, 6])
def test_warp_rows_many_rows_per_warp(p, wb, logR, last_of):
    """Passes with enough rows for several rows per warp (shared twiddle loads,
    lane stages paired across rows), every variant: alone (last_of = 0), with a
    ragged number of rows (a multiple of neither the rows per warp nor the warps
    per CTA), and as the last pass of a [6, log R] split."""
    torch = require_gpu()
    o = oracle.get()
    logL = logR + last_of
    L = 1 << logL
    if (p - 1) % L:
        pytest.skip("L does not divide p-1")
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L, word_bytes=wb)
    if last_of:
        plan.set_split([last_of, logR])
    plan.set_warp_rows(True)
    dt = np.uint32 if plan.word_bytes == 4 else np.uint64
    g = group_rows(plan.word_bytes, logR)
    if g == 1:
        plan.destroy()
        pytest.skip("one row per warp at this length and word size")
    rows_needed = g * 2 * 8 * 152 + 3
    batch = -(-rows_needed // (L >> logR))
    if (batch * (L >> logR)) % g == 0:
        batch += 1
    try:
        for v in variants_for(p, wb):
            plan.set_variant(v)
            top_f = p - 1 if v in (1, 3) else 2 * p - 1
            top_i = p - 1 if v in (1, 3) else 4 * p - 1
            a = batch_inputs(2400 + logL, batch, L, p).astype(np.uint64)
            a[1, :] = top_f
            a[-1, :] = top_f
            got = run(plan, a, False, torch, dt)
            assert np.array_equal(got, o.ntt_ref(p, w, a % np.uint64(p))), f"forward variant {v}"
            y = batch_inputs(2500 + logL, batch, L, p).astype(np.uint64)
            y[0, :] = top_i
            y[-1, :] = top_i
            got = run(plan, y, True, torch, dt)
            assert np.array_equal(got, o.intt_ref(p, w, y % np.uint64(p))), f"inverse variant {v}"
    finally:
        plan.destroy()
