"""Pins for the CPU oracle: checks against facts the paper and the mathematics
fix, never against the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError on
failure.  ``tests/test_oracle.py`` runs them on the real oracle, and
``tests/test_oracle_mutants.py`` runs them on builds with a planted mistake to
show that each kind of mistake is caught by at least one pin.

What pins what:

* Section 1 definition, brute force on tiny inputs: Horner evaluation of
  a_0 + a_1 x + ... at the points omega^j (the paper's equivalent reading of
  the NTT as polynomial evaluation), with Python integers.
* Closed forms: L = 2 gives (a0 + a1, a0 - a1); a delta at 0 gives all ones; a
  constant c gives L*c at position 0 and zeros elsewhere (bit reversal fixes
  0); a delta at i gives omega^(i * rev(k)) at position k; L = 4 by hand.
* Algorithm 1 against the definition at every size up to 2^10.
* Section 4 inverse: running Algorithm 1 backwards returns L * a.
* Convolution theorem versus the schoolbook product, and the schoolbook
  product versus numpy's own polynomial product on Python integers.
* Linearity of the transform.
"""
from __future__ import annotations

import numpy as np

from paper_1205_2926_gb300.inputs import uniform_residues

# ... plus two primes in Moeller's range beta/2 < p < beta/phi (end of Section 2) for 32- and 64-bit
# words, where the oracle's additions must not overflow 64 bits
SMALL_PRIMES = [17, 97, 257, 7681, 12289, 998244353, 1073479681, 2305843009448574977, 2649751553,
                11400714819167322113]


def v2(n: int) -> int:
    return (n & -n).bit_length() - 1


def bitrev(k: int, l: int) -> int:
    return int(format(k, f"0{l}b")[::-1], 2) if l > 0 else 0


def primitive_root_of_order(p: int, L: int) -> int:
    """A primitive L-th root found by trial: g^((p-1)/L) whose (L/2)-th power is -1."""
    for g in range(2, 10_000):
        w = pow(g, (p - 1) // L, p)
        if L == 1 or pow(w, L // 2, p) == p - 1:
            return w
    raise ValueError("no root found")


def horner_eval(coeffs, x: int, p: int) -> int:
    acc = 0
    for c in reversed([int(v) for v in coeffs]):
        acc = (acc * x + c) % p
    return acc


def pin_hand_example(o):
    # p = 17, L = 4, omega = 4 (4^2 = 16 = -1 mod 17), a = (1, 2, 3, 4):
    # b0 = 10, b1 = 1 + 8 + 48 + 256 = 313 = 7, b2 = 1 - 2 + 3 - 4 = -2 = 15,
    # b3 = 1 + 2*13 + 3*16 + 4*4 = 91 = 6 (13 = 4^3, 16 = 13^2, 4 = 13^3 mod 17).
    # Bit-reversed order for l = 2 is (b0, b2, b1, b3).
    want = [10, 15, 7, 6]
    assert list(o.dft_naive(17, 4, [1, 2, 3, 4])) == want
    assert list(o.ntt_ref(17, 4, [1, 2, 3, 4])) == want


def pin_definition_by_horner(o):
    for p in SMALL_PRIMES:
        for l in range(0, 6):
            L = 1 << l
            if (p - 1) % L:
                continue
            w = primitive_root_of_order(p, L)
            a = uniform_residues(1000 + l, L, p)
            want = [horner_eval(a, pow(w, bitrev(k, l), p), p) for k in range(L)]
            got = [int(v) for v in o.dft_naive(p, w, a)]
            assert got == want, (p, L)
            got = [int(v) for v in o.ntt_ref(p, w, a)]
            assert got == want, (p, L)


def pin_closed_forms(o):
    for p in SMALL_PRIMES:
        for l in range(1, 9):
            L = 1 << l
            if (p - 1) % L:
                continue
            w = primitive_root_of_order(p, L)
            for fn in (o.dft_naive, o.ntt_ref):
                if fn is o.dft_naive and l > 7:
                    continue
                # delta at 0 -> all ones
                d0 = np.zeros(L, dtype=np.uint64)
                d0[0] = 1
                assert np.all(fn(p, w, d0) == 1), (p, L, "delta0")
                # constant c -> L*c at position 0, zeros elsewhere
                c = (p - 1) // 3 + 1
                out = fn(p, w, np.full(L, c, dtype=np.uint64))
                assert int(out[0]) == (L * c) % p and np.all(out[1:] == 0), (p, L, "const")
                # delta at i -> omega^(i*rev(k))
                for i in (1, L // 2 + 1 if L > 2 else 1, L - 1):
                    di = np.zeros(L, dtype=np.uint64)
                    di[i] = 1
                    want = [pow(w, i * bitrev(k, l), p) for k in range(L)]
                    assert [int(v) for v in fn(p, w, di)] == want, (p, L, "delta", i)
            if l == 1:
                a0, a1 = p - 2, 5 % p
                assert [int(v) for v in o.ntt_ref(p, w, [a0, a1])] == [(a0 + a1) % p, (a0 - a1) % p]
                assert [int(v) for v in o.dft_naive(p, w, [a0, a1])] == [(a0 + a1) % p, (a0 - a1) % p]


def pin_alg1_vs_definition(o, max_l: int = 10):
    for p in SMALL_PRIMES:
        for l in range(1, max_l + 1):
            L = 1 << l
            if (p - 1) % L:
                continue
            w = primitive_root_of_order(p, L)
            a = uniform_residues(2000 + l, L, p)
            assert np.array_equal(o.ntt_ref(p, w, a), o.dft_naive(p, w, a)), (p, L)


def pin_inverse(o, max_l: int = 12):
    for p in SMALL_PRIMES:
        for l in range(1, max_l + 1):
            L = 1 << l
            if (p - 1) % L:
                continue
            w = primitive_root_of_order(p, L)
            a = uniform_residues(3000 + l, L, p)
            back = o.intt_ref(p, w, o.ntt_ref(p, w, a))
            want = np.array([(L * int(v)) % p for v in a], dtype=np.uint64)
            assert np.array_equal(back, want), (p, L, "intt_ref")
            if l <= 7:
                back = o.idft_naive(p, w, o.dft_naive(p, w, a))
                assert np.array_equal(back, want), (p, L, "idft_naive")
                y = uniform_residues(3500 + l, L, p)
                assert np.array_equal(o.intt_ref(p, w, y), o.idft_naive(p, w, y)), (p, L)


def pin_schoolbook_vs_numpy(o):
    for p in (17, 998244353, 2305843009448574977):
        for na, nb in [(1, 1), (1, 5), (2, 2), (3, 7), (16, 9), (33, 64)]:
            a = uniform_residues(4000 + na, na, p)
            b = uniform_residues(4100 + nb, nb, p)
            ref = np.convolve(np.array([int(v) for v in a], dtype=object),
                              np.array([int(v) for v in b], dtype=object))
            want = [int(v) % p for v in ref]
            assert [int(v) for v in o.polymul_schoolbook(p, a, b)] == want, (p, na, nb)


def pin_convolution_theorem(o):
    for p in (998244353, 2305843009448574977, 1072496641):
        for na, nb in [(1, 1), (2, 3), (5, 4), (64, 65), (300, 212), (1000, 1)]:
            a = uniform_residues(5000 + na, na, p)
            b = uniform_residues(5100 + nb, nb, p)
            assert np.array_equal(o.polymul_ntt(p, a, b), o.polymul_schoolbook(p, a, b)), (p, na, nb)


def pin_linearity(o):
    p = 998244353
    for l in (3, 8, 11):
        L = 1 << l
        w = primitive_root_of_order(p, L)
        a = uniform_residues(6000 + l, L, p)
        b = uniform_residues(6100 + l, L, p)
        s = np.array([(int(x) + int(y)) % p for x, y in zip(a, b)], dtype=np.uint64)
        fa, fb, fs = o.ntt_ref(p, w, a), o.ntt_ref(p, w, b), o.ntt_ref(p, w, s)
        assert [int(v) for v in fs] == [(int(x) + int(y)) % p for x, y in zip(fa, fb)]
        c = 123456789
        fc = o.ntt_ref(p, w, np.array([(c * int(x)) % p for x in a], dtype=np.uint64))
        assert [int(v) for v in fc] == [(c * int(x)) % p for x in fa]


ALL_PINS = [
    pin_hand_example,
    pin_definition_by_horner,
    pin_closed_forms,
    pin_alg1_vs_definition,
    pin_inverse,
    pin_schoolbook_vs_numpy,
    pin_convolution_theorem,
    pin_linearity,
]


def pin_dft_at(o):
    """One-position evaluation agrees with Horner evaluation at omega^rev(k)."""
    for p in (998244353, 2305843009448574977):
        for l in (1, 5, 9):
            L = 1 << l
            w = primitive_root_of_order(p, L)
            a = uniform_residues(7000 + l, L, p)
            for k in (0, 1, L // 2, L - 1):
                assert o.dft_at(p, w, a, k) == horner_eval(a, pow(w, bitrev(k, l), p), p)


ALL_PINS.append(pin_dft_at)


def pin_batch_wrappers(o):
    """The batched forms (``batch`` transforms ``stride`` words apart, stride >
    L) against Horner evaluation row by row, with the padding words between
    rows left untouched.  Forward: position k of row b is row b's polynomial at
    omega^rev(k) (Section 1 definition in Algorithm 1's order).  Inverse
    (Section 4, unnormalised): position i is sum_j omega^(-i j) y[rev(j)], the
    polynomial with coefficients y[rev(j)] evaluated at omega^-i."""
    import ctypes
    p64 = ctypes.POINTER(ctypes.c_uint64)
    sentinel = np.uint64(0xA5A5A5A5A5A5A5A5)
    for p in (17, 998244353, 2305843009448574977):
        for l, batch, pad in ((2, 3, 1), (4, 5, 3), (6, 3, 7)):
            L = 1 << l
            if (p - 1) % L:
                continue
            w = primitive_root_of_order(p, L)
            winv = pow(w, p - 2, p)
            stride = L + pad
            rows = [uniform_residues(8000 + 17 * l + b, L, p) for b in range(batch)]
            for inverse in (False, True):
                buf = np.full(batch * stride, sentinel, dtype=np.uint64)
                for b in range(batch):
                    buf[b * stride:b * stride + L] = rows[b]
                fn = o.lib.or_intt_ref_batch if inverse else o.lib.or_ntt_ref_batch
                fn(p, w, L, buf.ctypes.data_as(p64), batch, stride)
                for b in range(batch):
                    got = [int(v) for v in buf[b * stride:b * stride + L]]
                    if inverse:
                        coeffs = [int(rows[b][bitrev(j, l)]) for j in range(L)]
                        want = [horner_eval(coeffs, pow(winv, i, p), p) for i in range(L)]
                    else:
                        want = [horner_eval(rows[b], pow(w, bitrev(k, l), p), p) for k in range(L)]
                    assert got == want, (p, L, batch, stride, b, "inverse" if inverse else "forward")
                    assert np.all(buf[b * stride + L:(b + 1) * stride] == sentinel), (p, L, b, "padding")


ALL_PINS.append(pin_batch_wrappers)
