"""Parity of the CUDA transforms with the CPU oracle, bit-exact after the final
reduction (Section 3), through the C ABI.  Every input is seeded.

Covered: every length 2^1 .. 2^16 (single and multi-pass schedules) with a
ragged batch and padded stride; the 32-bit and 64-bit word paths; the lazy
(Algorithms 3/4), NTL-style (Algorithm 2) and Montgomery (Algorithm 5)
variants; forward and inverse
(Section 4); redundant inputs in [0,2p) / [0,4p); every allowed pass split at
selected lengths; the full-size workloads (64 x 2^16, 2^20, 2^22 at 32 bits;
16 x 2^20 and 2^24 at 64 bits) compared in full; argument errors."""
import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, P_UNEVEN, batch_inputs, uniform_residues, word_dtype
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

O = None


def orc():
    global O
    if O is None:
        O = oracle.get()
    return O


def run(plan, a_np, inverse, stride=None, variant=0, torch=None):
    """Transform rows of a_np (batch, L) on the GPU; returns (batch, L) numpy."""
    batch, L = a_np.shape
    stride = stride or L
    buf = np.zeros((batch, stride), dtype=a_np.dtype)
    buf[:, :L] = a_np
    if stride > L:
        buf[:, L:] = np.iinfo(a_np.dtype).max  # padding must stay untouched
    d = to_dev(buf, torch)
    plan.set_variant(variant)
    if inverse:
        ntt.ntt_inverse_batch(plan, d, batch, stride)
    else:
        ntt.ntt_forward_batch(plan, d, batch, stride)
    torch.cuda.synchronize()
    out = from_dev(d, a_np.dtype).reshape(batch, stride)
    if stride > L:
        assert np.all(out[:, L:] == np.iinfo(a_np.dtype).max), "wrote outside the transform"
    return out[:, :L]


def pad_stride(L, wbytes, extra):
    per16 = 16 // wbytes
    return ((L + extra + per16 - 1) // per16) * per16


@pytest.mark.parametrize("p", [P_NTT30, P_UNEVEN[0], P_NTT62])
@pytest.mark.parametrize("logL", list(range(1, 17)))
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_forward_inverse_all_lengths(p, logL, variant):
    torch = require_gpu()
    L = 1 << logL
    if (p - 1) % L:
        pytest.skip("L does not divide p-1")
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    batch = 3
    a = batch_inputs(100 + logL, batch, L, p)
    stride = pad_stride(L, plan.word_bytes, 5)
    got = run(plan, a, False, stride, variant, torch)
    want = o.ntt_ref(p, w, a.astype(np.uint64))
    assert np.array_equal(got.astype(np.uint64), want), f"forward p={p} L={L} variant={variant}"
    y = batch_inputs(200 + logL, batch, L, p)
    got = run(plan, y, True, stride, variant, torch)
    want = o.intt_ref(p, w, y.astype(np.uint64))
    assert np.array_equal(got.astype(np.uint64), want), f"inverse p={p} L={L} variant={variant}"
    plan.destroy()


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
@pytest.mark.parametrize("logL", [3, 9, 13, 16])
@pytest.mark.parametrize("variant", [0, 2])
def test_redundant_inputs(p, logL, variant):
    """Algorithms 3 and 5 accept [0,2p), Algorithm 4 and its Montgomery
    counterpart [0,4p) on input."""
    torch = require_gpu()
    L = 1 << logL
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    dt = word_dtype(p)
    a = uniform_residues(300 + logL, 2 * L, 2 * p).astype(dt).reshape(2, L)
    got = run(plan, a, False, None, variant, torch)
    assert np.array_equal(got.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64) % np.uint64(p)))
    y = uniform_residues(400 + logL, 2 * L, 4 * p).astype(dt).reshape(2, L)
    got = run(plan, y, True, None, variant, torch)
    assert np.array_equal(got.astype(np.uint64), o.intt_ref(p, w, y.astype(np.uint64) % np.uint64(p)))
    plan.destroy()


SPLITS = {
    11: [[11], [3, 8], [6, 5], [3, 3, 5]],
    14: [[7, 7], [3, 11], [9, 5], [4, 4, 6], [3, 3, 3, 5], [10, 4]],
    17: [[5, 12], [9, 8], [10, 7], [6, 11], [11, 6], [4, 5, 8], [6, 6, 5]],
    22: [[11, 11], [10, 12], [6, 5, 11]],
}


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
@pytest.mark.parametrize("logL,split", [(k, s) for k, v in SPLITS.items() for s in v])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_split(p, logL, split, variant):
    torch = require_gpu()
    L = 1 << logL
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    min_after = 5 if plan.word_bytes == 4 else 4  # a column pass needs >= 128 bytes per tile row
    valid = all(logL - sum(split[:i + 1]) >= min_after for i in range(len(split) - 1)) and \
        all(3 <= r <= 11 for r in split)
    if not valid:
        with pytest.raises(ntt.NTTError) as e:
            plan.set_split(split)
        assert e.value.code == -4
        return
    plan.set_split(split)
    assert list(plan.info().log_r)[:len(split)] == split
    a = batch_inputs(500 + logL, 2, L, p)
    got = run(plan, a, False, None, variant, torch)
    assert np.array_equal(got.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    got = run(plan, a, True, None, variant, torch)
    assert np.array_equal(got.astype(np.uint64), o.intt_ref(p, w, a.astype(np.uint64)))
    plan.destroy()


FULL = [
    (P_NTT30, 16, 64),
    (P_NTT30, 20, 1),
    (P_NTT30, 22, 1),
    (P_NTT62, 20, 16),
    (P_NTT62, 24, 1),
]


@pytest.mark.parametrize("p,logL,batch", FULL)
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_full_size_workloads(p, logL, batch, variant):
    torch = require_gpu()
    L = 1 << logL
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    a = batch_inputs(600 + logL, batch, L, p)
    fwd = run(plan, a, False, None, variant, torch)
    assert np.array_equal(fwd.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    back = run(plan, fwd, True, None, variant, torch)
    want = (a.astype(object) * L % p).astype(np.uint64)
    assert np.array_equal(back.astype(np.uint64), want), "inverse(forward(a)) != L a"
    plan.destroy()


def test_sampled_definition_c1():
    """L = 2^10, p = 998244353: every output against the stored golden file and
    sampled positions against the definition."""
    torch = require_gpu()
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "forward_p998244353_L1024_seed1.txt")
    g = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        g[k] = [int(x) for x in v]
    p, L, w = g["p"][0], g["L"][0], g["omega"][0]
    assert ntt.root_of_unity(p, L) == w
    plan = ntt.ntt_plan(p, w, L)
    a = np.array(g["input"], dtype=np.uint32).reshape(1, L)
    got = run(plan, a, False, None, 0, torch)
    assert [int(v) for v in got[0]] == g["output"]
    for k in (0, 1, 2, 511, 1023):
        assert int(got[0, k]) == orc().dft_at(p, w, a[0], k)


def test_transform_host_roundtrip():
    require_gpu()
    p, L = P_NTT30, 1 << 12
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    a = batch_inputs(700, 4, L, p)
    h = a.copy()
    ntt.ntt_transform_host(plan, False, h, 4)
    assert np.array_equal(h.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    ntt.ntt_transform_host(plan, True, h, 4)
    assert np.array_equal(h.astype(np.uint64), (a.astype(object) * L % p).astype(np.uint64))


@pytest.mark.parametrize("p,logL,batch,pad", [(P_NTT30, 15, 50, 4), (P_NTT62, 16, 9, 2), (P_NTT30, 11, 1100, 0)])
def test_transform_host_chunked(p, logL, batch, pad):
    """Batches above the chunk size go through the copy/transform pipeline in
    uneven chunks; strided rows keep their padding words untouched."""
    require_gpu()
    L = 1 << logL
    o = orc()
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    a = batch_inputs(710 + logL, batch, L, p)
    h = np.zeros((batch, L + pad), dtype=a.dtype)
    h[:, :L] = a
    if pad:
        h[:, L:] = 12345
    ntt.ntt_transform_host(plan, False, h, batch, L + pad)
    want = o.ntt_ref(p, w, a.astype(np.uint64))
    assert np.array_equal(h[:, :L].astype(np.uint64), want)
    if pad:
        assert (h[:, L:] == 12345).all()
    ntt.ntt_transform_host(plan, True, h, batch, L + pad)
    assert np.array_equal(h[:, :L].astype(np.uint64), (a.astype(object) * L % p).astype(np.uint64))


def test_transform_host_threads():
    """Calls on different plans from different threads overlap and stay exact."""
    torch = require_gpu()
    import threading
    o = orc()
    jobs = []
    for i, (p, logL, batch) in enumerate([(P_NTT30, 16, 24), (P_NTT30, 20, 1), (P_NTT62, 14, 40)]):
        L = 1 << logL
        w = o.root_of_unity(p, L)
        a = batch_inputs(720 + i, batch, L, p)
        jobs.append((ntt.ntt_plan(p, w, L), a, a.copy(), batch, torch.cuda.Stream(), p, w))
    errs = []

    def run(j):
        plan, a, h, batch, s, p, w = j
        try:
            for _ in range(3):
                ntt.ntt_transform_host(plan, False, h, batch, stream=s)
                ntt.ntt_transform_host(plan, True, h, batch, stream=s)
        except Exception as e:  # pragma: no cover - reported below
            errs.append(e)

    ts = [threading.Thread(target=run, args=(j,)) for j in jobs]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs
    for plan, a, h, batch, s, p, w in jobs:
        # three round trips multiply by L^3 (unnormalised inverse)
        want = (a.astype(object) * pow(plan.L, 3, p) % p).astype(np.uint64)
        assert np.array_equal(h.astype(np.uint64), want)


def test_argument_errors():
    torch = require_gpu()
    p = P_NTT30
    w = ntt.root_of_unity(p, 1024)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(p + 2, w, 1024)  # composite
    assert e.value.code == -1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(p, w, 1000)
    assert e.value.code == -2
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(p, w, 1 << 24)  # 2^24 does not divide p-1
    assert e.value.code == -2
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(p, (w * w) % p, 1024)  # order 512
    assert e.value.code == -3
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan(11400714819323198549, 3, 2)  # the first prime above floor(2^64/phi): no word fits it
    assert e.value.code == -1
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_plan((1 << 62) + 135, 3, 2)  # a prime in Moeller's range, but 3 is not -1 mod p
    assert e.value.code == -3
    plan = ntt.ntt_plan(p, w, 1024)
    d = torch.zeros(4096, dtype=torch.int32, device="cuda")
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_forward_batch(plan, d.data_ptr() + 4, 1)
    assert e.value.code == -8
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_forward_batch(plan, d, 1, 1000)
    assert e.value.code == -4
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_forward_batch(plan, d, 0)
    assert e.value.code == -4
    for bad in ([5, 4], [2, 8], [11, 3], [3, 3, 2, 2], [4, 2, 4]):  # wrong sum / too short / tail < 2^5
        with pytest.raises(ntt.NTTError) as e:
            plan.set_split(bad)
        assert e.value.code == -4
    plan.destroy()


def test_library_number_theory_matches_oracle():
    require_gpu()
    o = orc()
    for p in (P_NTT30, P_NTT62) + P_UNEVEN:
        for L in (2, 1024, 1 << 16):
            assert ntt.root_of_unity(p, L) == o.root_of_unity(p, L)
    assert ntt.find_prime(1 << 61, 24) == P_NTT62


TMA_REF = {}


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("split,extra", [([8, 8], 0), ([6, 10], 0), ([7, 5, 4], 2)])
def test_tensor_copy_column_tiles(split, extra, variant):
    """64-bit column passes with 128-byte tile rows fetch their tiles by tensor
    copies (cp.async.bulk.tensor); 40 transforms keep those tiles at full
    width, and a padded stride exercises the map's transform dimension."""
    torch = require_gpu()
    o = orc()
    p, L, batch = P_NTT62, 1 << 16, 40
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    plan.set_split(split)
    a = batch_inputs(902, batch, L, p)  # one input for every split: the oracle runs once
    if "ref" not in TMA_REF:
        TMA_REF["ref"] = (o.ntt_ref(p, w, a.astype(np.uint64)), o.intt_ref(p, w, a.astype(np.uint64)))
    fwd, inv = TMA_REF["ref"]
    stride = pad_stride(L, 8, extra) if extra else None
    assert ntt.ntt_pass_status(reset=True) == 0
    assert np.array_equal(run(plan, a, False, stride, variant, torch).astype(np.uint64), fwd)
    assert np.array_equal(run(plan, a, True, stride, variant, torch).astype(np.uint64), inv)
    assert ntt.ntt_pass_status() == 0
    plan.destroy()


def test_tile_copy_wait_times_out_and_recovers():
    """Tile copies that never complete (the test hook makes each expect 16 bytes
    that never arrive) end the pass with NTT_ERR_TIMEOUT after the wait budget
    instead of hanging; the next launch with normal waits is exact."""
    torch = require_gpu()
    o = orc()
    p, L, batch = P_NTT62, 1 << 16, 40
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    plan.set_split([8, 8])
    a = batch_inputs(911, batch, L, p)
    ntt.ntt_pass_status(reset=True)
    try:
        ntt.ntt_pass_set_wait_budget(2_000_000, stall_bytes=16)  # about 1 ms per wait
        run(plan, a, False, None, 0, torch)
        assert ntt.ntt_pass_status(reset=True) == -7
    finally:
        ntt.ntt_pass_set_wait_budget(2_000_000_000, 0)
    got = run(plan, a, False, None, 0, torch)
    assert ntt.ntt_pass_status() == 0
    assert np.array_equal(got.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_pass_set_wait_budget(0, 0)
    assert e.value.code == -4
    plan.destroy()


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
def test_checked_mode_input_ranges(p):
    """Checked mode: the input-range check finds the first word outside the
    interval the variant accepts (Algorithm 3: [0, 2p), Algorithm 4: [0, 4p),
    Algorithm 2: [0, p)), and a checked transform refuses such a batch with
    NTT_ERR_INPUT and leaves it untouched; in-range batches transform exactly."""
    torch = require_gpu()
    o = orc()
    L, batch = 1 << 12, 3
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    dt = word_dtype(p)
    a = batch_inputs(950, batch, L, p)
    stride = pad_stride(L, plan.word_bytes, 3)
    buf = np.zeros((batch, stride), dtype=dt)
    buf[:, :L] = a
    buf[:, L:] = np.iinfo(dt).max  # padding is outside the transforms and never checked
    d = to_dev(buf, torch)
    assert ntt.ntt_check_input(plan, False, d, batch, stride) == -1
    # a word in [2p, 4p): out of range forward, in range inverse (lazy), out of range for NTL
    bad = buf.copy()
    bad[1, 777] = dt(3 * p)
    bad[2, 5] = dt(2 * p)
    db = to_dev(bad, torch)
    assert ntt.ntt_check_input(plan, False, db, batch, stride) == 1 * L + 777
    assert ntt.ntt_check_input(plan, True, db, batch, stride) == -1
    plan.set_variant(1)
    assert ntt.ntt_check_input(plan, True, db, batch, stride) == 1 * L + 777
    assert ntt.ntt_check_input(plan, False, d, batch, stride) == -1
    plan.set_variant(0)
    bad[0, 9] = dt(4 * p)
    db = to_dev(bad, torch)
    assert ntt.ntt_check_input(plan, True, db, batch, stride) == 9
    # checked transforms
    plan.set_checked(True)
    with pytest.raises(ntt.NTTError) as e:
        ntt.ntt_forward_batch(plan, db, batch, stride)
    assert e.value.code == -14
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(db, dt).reshape(batch, stride), bad), "a refused batch was modified"
    ntt.ntt_forward_batch(plan, d, batch, stride)
    torch.cuda.synchronize()
    got = from_dev(d, dt).reshape(batch, stride)[:, :L]
    assert np.array_equal(got.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    plan.set_checked(False)
    plan.destroy()


def _times_pow2_mod(x: np.ndarray, k: int, p: int) -> np.ndarray:
    """x * 2^k mod p for residues x < p < 2^62, by k modular doublings (exact in uint64)."""
    x = x.astype(np.uint64).copy()
    pp = np.uint64(p)
    for _ in range(k):
        x = x + x
        x = np.where(x >= pp, x - pp, x)
    return x


def test_largest_transforms():
    """Maximum sizes: the 32-bit prime's largest length 2^23 against the oracle
    element by element, and the plans' largest length 2^26 (64-bit words, the
    smallest prime above 2^61 that is 1 mod 2^26) on sampled outputs of the
    definition plus inverse(forward(a)) = L a on every element."""
    torch = require_gpu()
    o = orc()
    # 2^23, 32-bit words: the whole transform both ways
    p, L = P_NTT30, 1 << 23
    w = o.root_of_unity(p, L)
    plan = ntt.ntt_plan(p, w, L)
    a = batch_inputs(960, 1, L, p)
    fwd = run(plan, a, False, None, 0, torch)
    assert np.array_equal(fwd.astype(np.uint64), o.ntt_ref(p, w, a.astype(np.uint64)))
    back = run(plan, fwd, True, None, 0, torch)
    assert np.array_equal(back[0].astype(np.uint64), _times_pow2_mod(a[0], 23, p))
    plan.destroy()
    # 2^26, 64-bit words
    q = o.find_prime_above(1 << 61, 26)
    assert q == ntt.find_prime(1 << 61, 26) and o.is_prime(q) and (q - 1) % (1 << 26) == 0
    L = 1 << 26
    w = o.root_of_unity(q, L)
    plan = ntt.ntt_plan(q, w, L)
    a = batch_inputs(961, 1, L, q)
    fwd = run(plan, a, False, None, 0, torch)
    rng = np.random.default_rng(5)
    for k in [0, 1, L - 1, L // 2] + [int(x) for x in rng.integers(0, L, size=4)]:
        assert int(fwd[0, k]) == o.dft_at(q, w, a[0], k), f"output {k}"
    back = run(plan, fwd, True, None, 0, torch)
    assert np.array_equal(back[0].astype(np.uint64), _times_pow2_mod(a[0], 26, q))
    plan.destroy()


@pytest.mark.parametrize("p", [P_NTT30, P_NTT62])
@pytest.mark.parametrize("logL", [2, 3, 10, 16, 20])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_dit_forward_and_dif_inverse(p, logL, variant):
    """The schedules with the roots exchanged: the forward transform from
    bit-reversed to natural order is the oracle's backwards Algorithm 1 with
    root omega^-1 inverted, i.e. sum_j omega^(ij) x[rev j]; the inverse from
    natural to bit-reversed order is Algorithm 1 with root omega^-1."""
    torch = require_gpu()
    o = orc()
    L, batch = 1 << logL, 2
    w = o.root_of_unity(p, L)
    wi = o.invmod(w, p)
    plan = ntt.ntt_plan(p, w, L)
    plan.set_variant(variant)
    dt = word_dtype(p)
    x = batch_inputs(970 + logL, batch, L, p)
    d = to_dev(x, torch)
    ntt.ntt_forward_dit_batch(plan, d, batch)
    torch.cuda.synchronize()
    got = from_dev(d, dt).reshape(batch, L).astype(np.uint64)
    assert np.array_equal(got, o.intt_ref(p, wi, x.astype(np.uint64))), "DIT forward"
    # applied to the bit-reversal of a: the DFT of a in natural order
    rev = np.array([o.bitrev(k, logL) for k in range(L)]) if logL <= 10 else None
    if rev is not None:
        nat = o.ntt_ref(p, w, x.astype(np.uint64))[:, rev]  # undo the bit-reversed placement
        d = to_dev(x[:, rev].copy(), torch)
        ntt.ntt_forward_dit_batch(plan, d, batch)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(d, dt).reshape(batch, L).astype(np.uint64), nat)
    d = to_dev(x, torch)
    ntt.ntt_inverse_dif_batch(plan, d, batch)
    torch.cuda.synchronize()
    got = from_dev(d, dt).reshape(batch, L).astype(np.uint64)
    assert np.array_equal(got, o.ntt_ref(p, wi, x.astype(np.uint64))), "DIF inverse"
    plan.destroy()
