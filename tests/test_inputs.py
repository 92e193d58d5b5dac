"""The seeded input generators match their stated definitions: splitmix64's
published output, exact uniform residues, and the workload recipes (uneven
batch and serving trace) with the documented shapes and distributions."""
import math

import numpy as np

from paper_1205_2926_gb300.inputs import (P_NTT30, P_NTT62, P_UNEVEN, batch_inputs, serving_trace, splitmix64,
                                          uneven_batch_spec, uniform_floats, uniform_residues)

M64 = (1 << 64) - 1


def _splitmix64_scalar(state: int) -> tuple[int, int]:
    """One step of the sequential generator (state += golden gamma, then mix)."""
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def test_splitmix64_published_value_and_counter_form():
    # first output of the generator seeded with 0 (Steele, Lea and Flood; Vigna's reference code)
    assert int(splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF
    # the counter form equals the sequential generator for any seed and offset
    for seed in (0, 1, 12345, M64):
        state, seq = seed, []
        for _ in range(200):
            state, z = _splitmix64_scalar(state)
            seq.append(z)
        assert [int(x) for x in splitmix64(seed, 0, 200)] == seq
        assert [int(x) for x in splitmix64(seed, 50, 20)] == seq[50:70]


def test_uniform_residues_exact_range_and_determinism():
    for p in (17, P_NTT30, P_NTT62) + P_UNEVEN:
        a = uniform_residues(3, 50_000, p)
        assert a.dtype == np.uint64 and a.size == 50_000
        assert int(a.max()) < p
        assert np.array_equal(a, uniform_residues(3, 50_000, p))
        assert not np.array_equal(a[:100], uniform_residues(4, 100, p))
        mean = float(a.astype(np.float64).mean())
        assert abs(mean - (p - 1) / 2) < 0.01 * p
    small = uniform_residues(9, 170_000, 17)
    counts = np.bincount(small.astype(np.int64), minlength=17)
    assert counts.size == 17 and abs(counts - 10_000).max() < 600  # every residue equally likely
    b = batch_inputs(1, 3, 1 << 10, P_NTT30)
    assert b.shape == (3, 1 << 10) and b.dtype == np.uint32
    assert batch_inputs(1, 2, 8, P_NTT62).dtype == np.uint64
    f = uniform_floats(2, 0, 10_000)
    assert f.min() >= 0.0 and f.max() < 1.0 and abs(f.mean() - 0.5) < 0.01


def test_uneven_batch_recipe():
    spec = uneven_batch_spec()
    assert len(spec) == 4096 and [d["id"] for d in spec] == list(range(4096))
    logs = np.array([d["logL"] for d in spec])
    assert logs.min() == 8 and logs.max() == 16
    counts = np.bincount(logs)[8:]
    assert counts.size == 9 and counts.min() > 355 and counts.max() < 555  # uniform over 8..16
    primes = [d["p"] for d in spec]
    assert set(primes) == set(P_UNEVEN) and min(primes.count(p) for p in P_UNEVEN) > 1200
    assert sum(d["inverse"] for d in spec) == 2048
    assert all(d["inverse"] == bool(d["id"] & 1) for d in spec)
    assert uneven_batch_spec() == spec  # seeded


def test_serving_trace_recipe():
    n, rate = 100_000, 20_000.0
    tr = serving_trace(seed=5, n=n, rate_per_s=rate)
    t = np.array([r["t_arrive_s"] for r in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() * rate - 1.0) < 0.02                      # Poisson: mean gap 1/rate
    assert abs(gaps.std() * rate - 1.0) < 0.03                       # exponential: std = mean
    d = np.array([r["na"] - 1 for r in tr] + [r["nb"] - 1 for r in tr])
    assert d.min() >= 64 and d.max() < (1 << 20)                     # degrees in [2^6, 2^20)
    assert abs(float(np.mean(d < (1 << 13))) - 0.5) < 0.01           # log-uniform: median 2^13
    assert abs(float(np.mean(np.log2(d))) - 13.0) < 0.05
    assert serving_trace(seed=5, n=100) == tr[:100]
