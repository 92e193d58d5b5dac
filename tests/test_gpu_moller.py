"""Moeller's form of Algorithm 2 (end of Section 2): the fully reduced
butterfly for any p < beta/phi, on the GPU, bit-exact against the oracle.

The primes sit in the range the refinement opens, beta/2 < p < beta/phi,
where Algorithm 2 as printed overflows the word (X + Y >= beta) and the
redundant-residue variants do not apply (p >= beta/4):

* 2649751553 = 0x9DF00001 < 2^32/phi, 1 mod 2^20, on 32-bit words
  (ntt_plan_words); the largest such prime that is 1 mod 2^20;
* 11400714819167322113 = 0x9E3779B976000001 < 2^64/phi, 1 mod 2^25, on
  64-bit words; the largest such prime that is 1 mod 2^24.

Also: the variant on a small prime equals Algorithm 2's results, every
variant's modulus bound is enforced, and the word-size choice of ntt_plan."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, batch_inputs, uniform_residues
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

P32M = 2649751553
P64M = 11400714819167322113
CASES = [(P32M, 4), (P64M, 8)]


def make_plan(p, L, wb):
    o = oracle.get()
    plan = ntt.ntt_plan(p, o.root_of_unity(p, L), L, word_bytes=wb)
    assert plan.word_bytes == wb
    return plan


def run(plan, rows, inverse, torch, stride_extra=True):
    """Transform (batch, L) rows in a padded-stride batch; padding must stay."""
    batch, L = rows.shape
    dt = np.uint32 if plan.word_bytes == 4 else np.uint64
    per16 = 16 // plan.word_bytes
    stride = L + per16 if stride_extra else L
    stride = (stride + per16 - 1) // per16 * per16  # rows start on 16-byte boundaries
    buf = np.full((batch, stride), np.iinfo(dt).max, dtype=dt)
    buf[:, :L] = rows.astype(dt)
    d = to_dev(buf, torch)
    (ntt.ntt_inverse_batch if inverse else ntt.ntt_forward_batch)(plan, d, batch, stride)
    torch.cuda.synchronize()
    out = from_dev(d, dt).reshape(batch, stride)
    assert np.all(out[:, L:] == np.iinfo(dt).max), "wrote into the padding"
    return out[:, :L].astype(np.uint64)


@pytest.mark.parametrize("p,wb", CASES)
@pytest.mark.parametrize("logL", list(range(1, 17)) + [18, 20])
def test_moller_forward_inverse(p, wb, logL):
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    plan = make_plan(p, L, wb)
    assert plan.info().variant == ntt.VARIANT_MOLLER
    w = o.root_of_unity(p, L)
    batch = 3 if logL <= 16 else 2
    a = batch_inputs(1700 + logL, batch, L, p)
    got = run(plan, a, False, torch)
    assert np.array_equal(got, o.ntt_ref(p, w, a.astype(np.uint64))), f"forward p={p} L=2^{logL}"
    y = batch_inputs(1800 + logL, batch, L, p)
    got = run(plan, y, True, torch)
    assert np.array_equal(got, o.intt_ref(p, w, y.astype(np.uint64))), f"inverse p={p} L=2^{logL}"
    plan.destroy()


@pytest.mark.parametrize("p,wb,logL,split", [
    (P32M, 4, 14, [7, 7]), (P32M, 4, 14, [4, 4, 6]), (P32M, 4, 17, [6, 6, 5]), (P32M, 4, 20, [10, 10]),
    (P32M, 4, 20, [6, 6, 8]), (P64M, 8, 14, [3, 11]), (P64M, 8, 17, [9, 8]), (P64M, 8, 20, [6, 6, 8]),
    (P64M, 8, 22, [7, 6, 9]),
])
def test_moller_splits_and_edges(p, wb, logL, split):
    """Every split's column passes (middle twiddle fused with the W = 1 stage)
    at the top of the input interval: all p - 1, beside zero, delta and
    uniform rows."""
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    plan = make_plan(p, L, wb)
    plan.set_split(split)
    w = o.root_of_unity(p, L)
    rows = np.zeros((4, L), dtype=np.uint64)
    rows[0, :] = p - 1
    rows[2, 1] = 1
    rows[3] = uniform_residues(1900 + logL, L, p)
    for inverse in (False, True):
        got = run(plan, rows, inverse, torch)
        want = (o.intt_ref if inverse else o.ntt_ref)(p, w, rows)
        assert np.array_equal(got, want), f"{'inverse' if inverse else 'forward'} split {split}"
    plan.destroy()


@pytest.mark.parametrize("p,wb", CASES)
def test_moller_dit_dif(p, wb):
    torch = require_gpu()
    o = oracle.get()
    L = 1 << 11
    plan = make_plan(p, L, wb)
    w = o.root_of_unity(p, L)
    wi = o.invmod(w, p)
    dt = np.uint32 if wb == 4 else np.uint64
    x = batch_inputs(1950, 2, L, p).astype(dt)
    x[0, :] = p - 1
    d = to_dev(x, torch)
    ntt.ntt_forward_dit_batch(plan, d, 2)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, dt).reshape(2, L).astype(np.uint64), o.intt_ref(p, wi, x.astype(np.uint64)))
    d = to_dev(x, torch)
    ntt.ntt_inverse_dif_batch(plan, d, 2)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, dt).reshape(2, L).astype(np.uint64), o.ntt_ref(p, wi, x.astype(np.uint64)))
    plan.destroy()


@pytest.mark.parametrize("p,logL", [(P_NTT30, 11), (P_NTT30, 16), (P_NTT62, 13)])
def test_moller_equals_algorithm2_below_half_beta(p, logL):
    """For p < beta/2 both fully reduced variants give the oracle's result."""
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    plan = ntt.ntt_plan(p, o.root_of_unity(p, L), L)
    a = batch_inputs(1990 + logL, 3, L, p)
    w = o.root_of_unity(p, L)
    want = o.ntt_ref(p, w, a.astype(np.uint64))
    for v in (ntt.VARIANT_NTL, ntt.VARIANT_MOLLER):
        plan.set_variant(v)
        assert np.array_equal(run(plan, a, False, torch), want), f"variant {v}"
    plan.destroy()


def test_variant_bounds_and_word_choice():
    """LAZY/MONT need p < beta/4, NTL p < beta/2, MOLLER p < beta/phi; ntt_plan
    picks 64-bit words from 2^30 on, ntt_plan_words keeps 32-bit words up to
    floor(2^32/phi)."""
    torch = require_gpu()
    o = oracle.get()
    L = 1 << 10
    p32 = ntt.ntt_plan(P32M, o.root_of_unity(P32M, L), L, word_bytes=4)
    assert p32.info().variant == ntt.VARIANT_MOLLER
    for v in (ntt.VARIANT_LAZY, ntt.VARIANT_MONT, ntt.VARIANT_NTL):  # P32M > 2^31
        with pytest.raises(ntt.NTTError) as e:
            p32.set_variant(v)
        assert e.value.code == -1
    auto = ntt.ntt_plan(P32M, o.root_of_unity(P32M, L), L)  # default choice: 64-bit words, lazy
    assert auto.word_bytes == 8 and auto.info().variant == ntt.VARIANT_LAZY
    p64 = ntt.ntt_plan(P64M, o.root_of_unity(P64M, L), L)
    assert p64.word_bytes == 8 and p64.info().variant == ntt.VARIANT_MOLLER
    with pytest.raises(ntt.NTTError) as e:
        p64.set_variant(ntt.VARIANT_NTL)  # P64M > 2^63
    assert e.value.code == -1
    # a prime in [2^62, 2^63): Algorithm 2 fits, the lazy variants do not
    q = ntt.find_prime((1 << 62) + (1 << 40), 20)
    pq = ntt.ntt_plan(q, o.root_of_unity(q, L), L)
    assert pq.info().variant == ntt.VARIANT_NTL
    with pytest.raises(ntt.NTTError) as e:
        pq.set_variant(ntt.VARIANT_LAZY)
    assert e.value.code == -1
    pq.set_variant(ntt.VARIANT_MOLLER)
    # beyond the bounds
    bad32 = ntt.find_prime(ntt.P_MAX_W32, 10)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(bad32, o.root_of_unity(bad32, L), L, word_bytes=4)
    assert e.value.code == -1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(P_NTT30, o.root_of_unity(P_NTT30, L), L, word_bytes=3)
    assert e.value.code == -4
    # checked mode bounds the inputs of a fully reduced variant at p
    d = torch.zeros(L, dtype=torch.int32, device="cuda")
    d[5] = P32M - (1 << 32)  # the word P32M (as a signed 32-bit value)
    assert ntt.ntt_check_input(p32, False, d, 1) == 5
    for pl in (p32, auto, p64, pq):
        pl.destroy()
