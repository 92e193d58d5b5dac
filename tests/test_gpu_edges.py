"""Parity at the edges of the butterflies' input intervals, on the GPU.

Algorithm 3 (and Algorithm 5) accept forward inputs in [0, 2p), Algorithm 4
(and its Montgomery counterpart) inverse inputs in [0, 4p), and Algorithm 2
fully reduced inputs in [0, p); Theorems 1-4 bound the outputs for every input
in those intervals.  The fused steps of the pass kernels (the distance-1 stage
merged with the middle twiddle, unreduced X + Y and X - Y + 2p before a
product) are only safe if those bounds hold at the very top of the interval,
which uniform inputs almost never reach.  So every row here is an extreme:

* the top of the accepted interval in every word (2p - 1 forward and 4p - 1
  inverse for the lazy and Montgomery variants, p - 1 for the NTL-style one);
* all p - 1, all zero, delta at 0, delta at 1, a constant;
* one uniform row,

mixed row by row in one ragged batch (7 rows, padded stride whose padding
must stay untouched), for all three variants, both word sizes, and the
default and other pass splits at each length.  Expected values come from the
oracle on the inputs reduced mod p, element by element.  At the largest
64-bit length (2^24) the oracle's O(L log L) reference is too slow for every
row, so there the rows are checked against properties that hold at any size
(closed forms of constant and delta inputs, pinned on the CPU against the
oracle and Horner evaluation), the oracle's single-position evaluation at
sampled outputs, and inverse(forward(a)) = L a on every element."""
import functools

import numpy as np
import pytest

import oracle
import paper_1205_2926_gb300 as ntt
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, P_UNEVEN, uniform_residues, word_dtype
from tests.gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

ROWS = ("top", "p-1", "zero", "delta0", "delta1", "const", "uniform")

# (p, log2 L): pass splits to run (None = the plan's default)
CASES = {
    (P_NTT30, 3): [None],
    (P_NTT30, 11): [None, [3, 8], [6, 5]],
    (P_NTT30, 14): [None, [7, 7], [4, 4, 6]],
    (P_NTT30, 17): [None, [9, 8], [6, 6, 5]],
    (P_NTT30, 20): [None, [6, 6, 8], [10, 10]],
    (P_NTT30, 22): [None, [7, 6, 9], [11, 11]],
    (P_UNEVEN[0], 16): [None, [8, 8]],
    (P_NTT62, 3): [None],
    (P_NTT62, 11): [None, [5, 6]],
    (P_NTT62, 14): [None, [4, 4, 6]],
    (P_NTT62, 17): [None, [9, 8]],
    (P_NTT62, 20): [None, [9, 11], [6, 6, 8]],
    (P_NTT62, 24): [None, [8, 8, 8], [7, 6, 11]],
}
FULL_ORACLE_MAX_LOG = 22  # above this, sampled outputs and properties (see the module docstring)


def _const(p):
    return (p - 1) // 3 + 1


def edge_rows(p, L, top):
    """The seven rows of ROWS, as Python-int-valued uint64 arrays (unreduced)."""
    rows = []
    for name in ROWS:
        r = np.zeros(L, dtype=np.uint64)
        if name == "top":
            r[:] = top
        elif name == "p-1":
            r[:] = p - 1
        elif name == "delta0":
            r[0] = 1
        elif name == "delta1":
            r[1] = 1
        elif name == "const":
            r[:] = _const(p)
        elif name == "uniform":
            r[:] = uniform_residues(31337 + L, L, p)
        rows.append(r)
    return np.stack(rows)


@functools.lru_cache(maxsize=None)
def oracle_rows(p, logL, inverse):
    """Oracle transform of the seven rows reduced mod p (the top row reduces
    to p - 1 for every variant, so one result serves all three)."""
    o = oracle.get()
    L = 1 << logL
    w = o.root_of_unity(p, L)
    rows = edge_rows(p, L, p - 1)
    return (o.intt_ref if inverse else o.ntt_ref)(p, w, rows)


def top_of_interval(p, variant, inverse):
    if variant == 1:  # Algorithm 2: fully reduced inputs
        return p - 1
    return 4 * p - 1 if inverse else 2 * p - 1


def run_rows(plan, rows, inverse, torch, dt):
    batch, L = rows.shape
    per16 = 16 // np.dtype(dt).itemsize
    stride = L + per16  # one 16-byte chunk of padding per row
    buf = np.full((batch, stride), np.iinfo(dt).max, dtype=dt)
    buf[:, :L] = rows.astype(dt)
    d = to_dev(buf, torch)
    if inverse:
        ntt.ntt_inverse_batch(plan, d, batch, stride)
    else:
        ntt.ntt_forward_batch(plan, d, batch, stride)
    torch.cuda.synchronize()
    out = from_dev(d, dt).reshape(batch, stride)
    assert np.all(out[:, L:] == np.iinfo(dt).max), "wrote into the padding between rows"
    del d
    return out[:, :L].astype(np.uint64)


def times_L(a, p, logL):
    """(a mod p) * 2^logL mod p, elementwise, by logL doublings (no overflow for p < 2^62)."""
    x = a % np.uint64(p)
    for _ in range(logL):
        x = x * np.uint64(2)
        x = np.where(x >= np.uint64(p), x - np.uint64(p), x)
    return x


@functools.lru_cache(maxsize=None)
def sampled_definition(p, logL, name):
    """Oracle single-position evaluations (Section 1 definition) of one row at
    sampled output positions: {k: value}."""
    o = oracle.get()
    L = 1 << logL
    w = o.root_of_unity(p, L)
    a = edge_rows(p, L, p - 1)[ROWS.index(name)] % np.uint64(p)
    rng = np.random.default_rng(logL)
    ks = np.unique(np.concatenate([[0, 1, 2, L // 2, L - 1], rng.integers(0, L, size=11)]))
    return {int(k): o.dft_at(p, w, a, int(k)) for k in ks}


def check_properties(p, logL, got, inverse):
    """Checks that hold at any size: constant rows (the top row and p - 1 are
    -1 mod p) give L c at position 0 and zeros elsewhere in both directions;
    a delta at position 0 gives all ones in both directions (its bit-reversed
    position is 0 as well); forward outputs of the delta-at-1 and uniform rows
    agree with the oracle's definition at sampled positions."""
    L = 1 << logL
    idx = {n: i for i, n in enumerate(ROWS)}
    for name, c in (("top", p - 1), ("p-1", p - 1), ("zero", 0), ("const", _const(p))):
        r = got[idx[name]]
        assert int(r[0]) == (L * c) % p and not np.any(r[1:]), f"{name} row"
    assert np.all(got[idx["delta0"]] == 1), "delta0 row"
    if not inverse:
        for name in ("delta1", "uniform"):
            for k, v in sampled_definition(p, logL, name).items():
                assert int(got[idx[name], k]) == v, f"{name} row, position {k}"


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("p,logL,split", [(p, l, s) for (p, l), v in CASES.items() for s in v],
                         ids=lambda x: str(x))
def test_edge_rows(p, logL, split, variant):
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    w = o.root_of_unity(p, L)
    dt = word_dtype(p)
    plan = ntt.ntt_plan(p, w, L)
    if split is not None:
        plan.set_split(split)
    plan.set_variant(variant)
    try:
        fwd_rows = fwd_out = None
        for inverse in (False, True):
            rows = edge_rows(p, L, top_of_interval(p, variant, inverse))
            got = run_rows(plan, rows, inverse, torch, dt)
            if not inverse:
                fwd_rows, fwd_out = rows, got
            if logL <= FULL_ORACLE_MAX_LOG:
                want = oracle_rows(p, logL, inverse)
                for i, name in enumerate(ROWS):
                    assert np.array_equal(got[i], want[i]), \
                        f"{'inverse' if inverse else 'forward'} row '{name}' (variant {variant}, split {split})"
            else:
                check_properties(p, logL, got, inverse)
        if logL > FULL_ORACLE_MAX_LOG:
            # at any size: inverse(forward(a)) = L a on every element of every row
            back = run_rows(plan, fwd_out, True, torch, dt)
            for i, name in enumerate(ROWS):
                assert np.array_equal(back[i], times_L(fwd_rows[i], p, logL)), f"{name} row round trip"
    finally:
        plan.destroy()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("p,logL", [(P_NTT30, 11), (P_NTT30, 20), (P_NTT62, 14)])
def test_edge_rows_dit_dif(p, logL, variant):
    """The bit-reversed-to-natural forward (DIT, Algorithm 4's butterfly and
    input interval [0, 4p)) and the natural-to-bit-reversed inverse (DIF,
    Algorithm 3's interval [0, 2p)) at the tops of their intervals."""
    torch = require_gpu()
    o = oracle.get()
    L = 1 << logL
    w = o.root_of_unity(p, L)
    wi = o.invmod(w, p)
    dt = word_dtype(p)
    plan = ntt.ntt_plan(p, w, L)
    plan.set_variant(variant)
    try:
        for dit in (True, False):
            top = p - 1 if variant == 1 else (4 * p - 1 if dit else 2 * p - 1)
            rows = edge_rows(p, L, top)
            d = to_dev(rows.astype(dt), torch)
            (ntt.ntt_forward_dit_batch if dit else ntt.ntt_inverse_dif_batch)(plan, d, len(ROWS))
            torch.cuda.synchronize()
            got = from_dev(d, dt).reshape(len(ROWS), L).astype(np.uint64)
            red = rows % np.uint64(p)
            want = o.intt_ref(p, wi, red) if dit else o.ntt_ref(p, wi, red)
            for i, name in enumerate(ROWS):
                assert np.array_equal(got[i], want[i]), f"{'DIT' if dit else 'DIF'} row '{name}' variant {variant}"
    finally:
        plan.destroy()


def test_edge_rows_uneven_batch():
    """One persistent launch (lazy butterflies) over transforms of several
    lengths and the three 30-bit primes whose words all sit at the top of the
    accepted interval, beside delta and zero rows."""
    torch = require_gpu()
    o = oracle.get()
    plans, items = {}, []
    for i, (logL, p, inverse) in enumerate([(8, P_UNEVEN[0], False), (9, P_UNEVEN[1], True), (12, P_UNEVEN[2], False),
                                            (13, P_UNEVEN[0], True), (16, P_UNEVEN[1], False),
                                            (16, P_UNEVEN[2], True), (11, P_UNEVEN[0], False)]):
        L = 1 << logL
        if (p, L) not in plans:
            plans[(p, L)] = ntt.ntt_plan(p, o.root_of_unity(p, L), L)
        kind = ROWS[i % len(ROWS)]
        top = 4 * p - 1 if inverse else 2 * p - 1
        a = edge_rows(p, L, top)[ROWS.index(kind)].astype(np.uint32)
        items.append((p, L, inverse, a, to_dev(a, torch), kind))
    ntt.ntt_execute_uneven([(plans[(p, L)], t, inv) for p, L, inv, _, t, _ in items])
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    for p, L, inv, a, t, kind in items:
        w = o.root_of_unity(p, L)
        red = a.astype(np.uint64) % np.uint64(p)
        want = o.intt_ref(p, w, red) if inv else o.ntt_ref(p, w, red)
        assert np.array_equal(from_dev(t, np.uint32).astype(np.uint64), want), f"L={L} p={p} inv={inv} row {kind}"
    for pl in plans.values():
        pl.destroy()
