"""The CPU oracle against its pins (definition, closed forms, Section 4
inverse, convolution theorem) and its number theory against sympy."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins
from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, P_UNEVEN, uniform_residues


@pytest.fixture(scope="module")
def o():
    return oracle.get()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(o, pin):
    pin(o)


def test_is_prime_matches_sympy(o):
    sympy = pytest.importorskip("sympy")
    for n in list(range(0, 3000)) + [561, 1105, 2047, 3215031751, 4759123141, 1122004669633,
                                     2152302898747, 3474749660383, 341550071728321,
                                     3825123056546413051, 318665857834031151167461 % (1 << 64)]:
        assert o.is_prime(n) == sympy.isprime(n), n
    for base in (1 << 30, 1 << 31, 1 << 61, (1 << 62) - 1000):
        for n in range(base - 300, base + 300):
            assert o.is_prime(n) == sympy.isprime(n), n


def test_workload_primes(o):
    sympy = pytest.importorskip("sympy")
    assert P_NTT30 == 119 * 2**23 + 1 and sympy.isprime(P_NTT30)
    assert o.smallest_qnr(P_NTT30) == 3  # "generator 3" of the 32-bit workloads
    # smallest prime > 2^61 with p = 1 mod 2^24: every earlier candidate is composite
    q = o.find_prime_above(1 << 61, 24)
    assert q == P_NTT62 and sympy.isprime(q) and (q - 1) % (1 << 24) == 0 and q < (1 << 62)
    c = ((1 << 61) // (1 << 24)) * (1 << 24) + 1
    while c <= (1 << 61):
        c += 1 << 24
    while c < q:
        assert not sympy.isprime(c)
        c += 1 << 24
    # three largest primes below 2^30 that are 1 mod 2^16
    found = []
    c = ((1 << 30) - 1) // (1 << 16) * (1 << 16) + 1
    while len(found) < 3:
        if c < (1 << 30) and sympy.isprime(c):
            found.append(c)
        c -= 1 << 16
    assert tuple(found) == P_UNEVEN
    for p in (P_NTT30, P_NTT62) + P_UNEVEN:
        g = o.smallest_qnr(p)
        assert not sympy.is_quad_residue(g, p)
        assert all(sympy.is_quad_residue(h, p) for h in range(2, g))


def test_root_of_unity_order(o):
    sympy = pytest.importorskip("sympy")
    for p, L in [(P_NTT30, 1 << 10), (P_NTT30, 1 << 23), (P_NTT62, 1 << 24), (P_NTT62, 1 << 20)] + \
                [(q, 1 << 16) for q in P_UNEVEN]:
        w = o.root_of_unity(p, L)
        assert sympy.n_order(w, p) == L
        assert o.powmod(w, L // 2, p) == p - 1
    assert o.root_of_unity(P_NTT30, 1 << 10) == 258648936  # 3^((p-1)/2^10)


def test_powmod_invmod_bitrev(o):
    p = P_NTT62
    for a in (1, 2, 3, p - 1, 123456789123456789):
        assert o.powmod(a, 12345, p) == pow(a, 12345, p)
        assert (o.invmod(a, p) * a) % p == 1
    for l in range(0, 12):
        for k in range(1 << l):
            assert o.bitrev(k, l) == oracle_pins.bitrev(k, l)


def test_inverse_large(o):
    """Section 4 inverse at a size the GPU configurations use."""
    p = P_NTT30
    L = 1 << 16
    w = o.root_of_unity(p, L)
    a = uniform_residues(77, L, p)
    back = o.intt_ref(p, w, o.ntt_ref(p, w, a))
    assert np.array_equal(back, (a.astype(object) * L % p).astype(np.uint64))


def _read_golden(name):
    import os
    d = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *vals = line.split()
            d[k] = [int(v) for v in vals]
    return d


def test_golden_hand_example(o):
    g = _read_golden("hand_p17_L4.txt")
    p, w = g["p"][0], g["omega"][0]
    assert [int(v) for v in o.ntt_ref(p, w, g["input"])] == g["output"]
    assert [int(v) for v in o.dft_naive(p, w, g["input"])] == g["output"]


def test_golden_forward_L1024_regenerates(o):
    g = _read_golden("forward_p998244353_L1024_seed1.txt")
    p, L, w, seed = g["p"][0], g["L"][0], g["omega"][0], g["seed"][0]
    a = uniform_residues(seed, L, p)
    assert [int(v) for v in a] == g["input"]
    assert [int(v) for v in o.dft_naive(p, w, a)] == g["output"]


def _schoolbook_limbs(a, b):
    """Long multiplication limb by limb with explicit carries (base 2^32): an
    algorithm independent of Python's big-integer product."""
    out = [0] * (len(a) + len(b))
    for i, ai in enumerate(a):
        carry = 0
        for j, bj in enumerate(b):
            t = out[i + j] + int(ai) * int(bj) + carry
            out[i + j] = t & 0xFFFFFFFF
            carry = t >> 32
        k = i + len(b)
        while carry:
            t = out[k] + carry
            out[k] = t & 0xFFFFFFFF
            carry = t >> 32
            k += 1
    return out


@pytest.mark.parametrize("na,nb,seed", [(1, 1, 0), (1, 9, 1), (7, 3, 2), (33, 65, 3), (128, 5, 4)])
def test_bigint_oracle_against_schoolbook(na, nb, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1 << 32, size=na, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 1 << 32, size=nb, dtype=np.uint64).astype(np.uint32)
    assert list(map(int, oracle.bigint_mul(a, b))) == _schoolbook_limbs(a, b)


@pytest.mark.parametrize("n", [1, 2, 17, 300])
def test_bigint_oracle_closed_forms(n):
    """(2^(32n) - 1)^2 = 2^(64n) - 2^(32n+1) + 1: limbs 1, 0.., then 0xFFFFFFFE,
    0xFFFFFFFF..; and x * 1 = x, x * 0 = 0."""
    ones = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    sq = oracle.bigint_mul(ones, ones)
    want = [1] + [0] * (n - 1) + [0xFFFFFFFE] + [0xFFFFFFFF] * (n - 1)
    assert list(map(int, sq)) == want
    x = np.arange(1, n + 1, dtype=np.uint32) * np.uint32(2654435761)
    assert list(map(int, oracle.bigint_mul(x, np.array([1], dtype=np.uint32)))) == list(map(int, x)) + [0]
    assert not oracle.bigint_mul(x, np.array([0], dtype=np.uint32)).any()


def test_golden_file_regenerates_from_the_oracle(tmp_path):
    """The stored forward golden file is exactly what its committed script
    writes from the oracle (no value in it came from anywhere else)."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = tmp_path / "forward.txt"
    mod.write_single_forward(str(out), P_NTT30, 1024, 1)
    with open(os.path.join(here, "forward_p998244353_L1024_seed1.txt")) as f:
        assert out.read_text() == f.read()
