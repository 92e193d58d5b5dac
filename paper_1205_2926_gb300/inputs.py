"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds random-number generation and workload shapes only -- no
modular arithmetic of the transform.  It imports nothing from the library or
from the oracle, so both sides can draw identical inputs from it.

Generator: splitmix64 used as a counter-based generator, x_i = mix(seed +
(i + 1) * 0x9E3779B97F4A7C15), with Steele, Lea and Flood's published output
function.  Residues uniform in [0, p) come from rejection sampling on the top
bit_length(p) bits of each draw, so they are exactly uniform.

Workload recipes (the paper measures uniform residues at power-of-two lengths,
Section 5):

* ``P_NTT30 = 998244353`` = 119 * 2^23 + 1, beta = 2^32 path.
* ``P_NTT62 = 2305843009448574977``: the smallest prime > 2^61 that is 1 mod
  2^24 (the tests re-derive it by a deterministic Miller-Rabin search).
* ``P_UNEVEN``: the three largest primes below 2^30 that are 1 mod 2^16.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

P_NTT30 = 998244353
P_NTT62 = 2305843009448574977
P_UNEVEN = (1073479681, 1072496641, 1071513601)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Counter-based splitmix64 outputs for counters start .. start+n-1."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_residues(seed: int, n: int, p: int, dtype=np.uint64) -> np.ndarray:
    """n residues uniform in [0, p) by rejection sampling; deterministic in seed."""
    if n == 0:
        return np.zeros(0, dtype=dtype)
    bits = int(p - 1).bit_length()
    shift = np.uint64(64 - bits)
    out = np.empty(n, dtype=np.uint64)
    filled, ctr = 0, 0
    while filled < n:
        want = n - filled
        chunk = max(1024, int(want * 2.2) + 64)
        x = splitmix64(seed, ctr, chunk) >> shift
        ctr += chunk
        acc = x[x < np.uint64(p)]
        take = min(want, acc.size)
        out[filled:filled + take] = acc[:take]
        filled += take
    return out.astype(dtype, copy=False)


def word_dtype(p: int):
    """Storage type of the library for modulus p: uint32 for p < 2^30, else uint64."""
    return np.uint32 if p < (1 << 30) else np.uint64


def batch_inputs(seed: int, batch: int, L: int, p: int) -> np.ndarray:
    """(batch, L) array of uniform residues in the library's word type."""
    return uniform_residues(seed, batch * L, p, word_dtype(p)).reshape(batch, L)


def uniform_floats(seed: int, start: int, n: int) -> np.ndarray:
    """Doubles uniform in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, start, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uneven_batch_spec(seed: int = 4, n: int = 4096, lmin: int = 8, lmax: int = 16, primes=P_UNEVEN):
    """Uneven batch: n transforms, log2 L uniform in [lmin, lmax], p uniform over
    ``primes``, forward for even ids and inverse for odd ids.

    Returns a list of dicts {id, logL, p, inverse}."""
    u = splitmix64(seed, 0, 2 * n)
    spec = []
    for i in range(n):
        logL = lmin + int(u[2 * i] % np.uint64(lmax - lmin + 1))
        p = primes[int(u[2 * i + 1] % np.uint64(len(primes)))]
        spec.append({"id": i, "logL": logL, "p": p, "inverse": bool(i & 1)})
    return spec


def serving_trace(seed: int = 5, n: int = 1000, rate_per_s: float = 20000.0, dmin_log: float = 6.0,
                  dmax_log: float = 20.0):
    """Poisson arrival trace of polynomial products.

    Arrival gaps are exponential with mean 1/rate (inverse-CDF of seeded
    uniforms); each operand's degree d = floor(2^U(dmin_log, dmax_log)), so an
    operand has d + 1 coefficients.  Returns a list of dicts
    {id, t_arrive_s, na, nb}."""
    u = uniform_floats(seed, 0, 3 * n)
    t = 0.0
    trace = []
    for i in range(n):
        gap = -math.log(1.0 - u[3 * i]) / rate_per_s
        t += gap
        da = int(math.floor(2.0 ** (dmin_log + (dmax_log - dmin_log) * u[3 * i + 1])))
        db = int(math.floor(2.0 ** (dmin_log + (dmax_log - dmin_log) * u[3 * i + 2])))
        trace.append({"id": i, "t_arrive_s": t, "na": da + 1, "nb": db + 1})
    return trace
