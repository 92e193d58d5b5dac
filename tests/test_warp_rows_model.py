"""A CPU model of the data movement of the warp-per-row pass (k_warp_row):
32 lanes holding R/32 words of each of G rows in registers, layout A
(word i in lane i mod 32, register i / 32), the stages of distance >= 32
inside a lane, one transpose to layout B (lane i / n holds n consecutive
words), the lane-exchange stages with their pairing of two register words
(word k of rows g and g + 1, or words k and k + 1 of one row) and two
shuffles, and the stages of distance < n inside a lane again; the inverse
runs the same steps backwards.  The model does the butterflies with fully
reduced arithmetic and must give the oracle's transform of every row
(Algorithm 1's output order) for every row length 2^5..2^10 and every group
size the kernel uses; a pairing or index mistake changes the result.  Also
the launch geometry: rows covered exactly once by the grid-stride loop over
groups, and the shared memory of a CTA within the per-CTA limit.  CPU only:
the GPU kernel itself is checked by tests/test_gpu_warp_rows.py."""
import numpy as np
import pytest

import oracle

P = 998244353
CTA_WARPS = 8           # kWarpRowsPerCta
GRID_CAP = 152 * 16     # most CTAs a warp-row launch uses
SMEM_LIMIT = 227 * 1024


def group_rows(word_bytes, log_r):
    """Rows per warp of the batched form: up to 32 (32-bit) or 16 (64-bit)
    words per thread, at most 8 rows."""
    n = (1 << log_r) // 32
    words = 32 if word_bytes == 4 else 16
    return 1 if n >= words else min(8, words // n)


def stage_tables(w, R):
    """tw[m + j] = (w^(R / 2m))^j for the stage of half-length m."""
    tw = [0] * R
    m = 1
    while m < R:
        wm = pow(w, R // (2 * m), P)
        for j in range(m):
            tw[m + j] = pow(wm, j, P)
        m *= 2
    return tw


def bfly(inverse, lo, hi, w):
    if not inverse:
        return (lo + hi) % P, (lo - hi) * w % P
    t = hi * w % P
    return (lo + t) % P, (lo - t) % P


def model(rows, inverse, log_r, tw, mutate=0):
    """x[lane][g][k] through the kernel's steps; returns the G rows.  mutate
    plants an index mistake in the lane exchange (negative controls): 1 the
    upper lane takes the twiddle of the lower lane's word, 2 the returned
    half lands in the other register."""
    G, R = rows.shape
    N = R // 32
    log_n = log_r - 5
    x = [[[0] * N for _ in range(G)] for _ in range(32)]

    def stages_a():
        for step in range(log_r - 5):
            lm = 5 + step if inverse else log_r - 1 - step
            h = 1 << (lm - 5)
            for lane in range(32):
                for k in range(N):
                    if k & h:
                        continue
                    w = tw[(1 << lm) + lane + 32 * (k & (h - 1))]
                    for g in range(G):
                        x[lane][g][k], x[lane][g][k + h] = bfly(inverse, x[lane][g][k], x[lane][g][k + h], w)

    def lane_pair(a, b, ta, tb, lb):
        """Registers a = (g, k) and b = (g', k') of every lane: the lower lane
        computes pair a, the upper lane pair b."""
        sent = [x[l][b[0]][b[1]] if not (l & lb) else x[l][a[0]][a[1]] for l in range(32)]
        got = [sent[l ^ lb] for l in range(32)]
        lo, hi = [0] * 32, [0] * 32
        for l in range(32):
            up = bool(l & lb)
            lo[l] = got[l] if up else x[l][a[0]][a[1]]
            hi[l] = x[l][b[0]][b[1]] if up else got[l]
            lo[l], hi[l] = bfly(inverse, lo[l], hi[l], tw[tb(l) if up and mutate != 1 else ta(l)])
        back_sent = [lo[l] if (l & lb) else hi[l] for l in range(32)]
        back = [back_sent[l ^ lb] for l in range(32)]
        for l in range(32):
            up = bool(l & lb)
            if mutate == 2:
                up = not up
            x[l][a[0]][a[1]] = back[l] if up else lo[l]
            x[l][b[0]][b[1]] = hi[l] if up else back[l]

    def stages_lanes():
        for step in range(5 - log_n):
            lm = log_n + step if inverse else 4 - step
            m = 1 << lm
            lb = m // N

            def idx(k):
                return lambda l: m + ((N * (l & ~lb) + k) & (m - 1))
            if G >= 2:
                for k in range(N):
                    for g in range(0, G - 1, 2):
                        lane_pair((g, k), (g + 1, k), idx(k), idx(k), lb)
            elif N >= 2:
                for k in range(0, N, 2):
                    lane_pair((0, k), (0, k + 1), idx(k), idx(k + 1), lb)
            else:
                v = [x[l][0][0] for l in range(32)]
                for l in range(32):
                    up = bool(l & lb)
                    u = v[l ^ lb]
                    lo, hi = (u, v[l]) if up else (v[l], u)
                    lo, hi = bfly(inverse, lo, hi, tw[idx(0)(l)])
                    x[l][0][0] = hi if up else lo

    def stages_b():
        for step in range(log_n):
            lm = step if inverse else log_n - 1 - step
            m = 1 << lm
            for lane in range(32):
                for k in range(N):
                    if k & m:
                        continue
                    w = tw[m + (k & (m - 1))]
                    for g in range(G):
                        x[lane][g][k], x[lane][g][k + m] = bfly(inverse, x[lane][g][k], x[lane][g][k + m], w)

    def transpose(a_to_b):
        for g in range(G):
            row = [0] * R
            for l in range(32):
                for k in range(N):
                    row[(l + 32 * k) if a_to_b else (N * l + k)] = x[l][g][k]
            for l in range(32):
                for k in range(N):
                    x[l][g][k] = row[(N * l + k) if a_to_b else (l + 32 * k)]

    out = np.zeros((G, R), dtype=np.uint64)
    if not inverse:
        for g in range(G):
            for l in range(32):
                for k in range(N):
                    x[l][g][k] = int(rows[g, l + 32 * k])
        stages_a()
        transpose(True)
        stages_lanes()
        stages_b()
        for g in range(G):
            for l in range(32):
                for k in range(N):
                    out[g, N * l + k] = x[l][g][k]
    else:
        for g in range(G):
            for l in range(32):
                for k in range(N):
                    x[l][g][k] = int(rows[g, N * l + k])
        stages_b()
        stages_lanes()
        transpose(False)
        stages_a()
        for g in range(G):
            for l in range(32):
                for k in range(N):
                    out[g, l + 32 * k] = x[l][g][k]
    return out


CASES = sorted({(lr, g) for lr in range(5, 11) for g in (1, group_rows(4, lr), group_rows(8, lr), 2)})


@pytest.mark.parametrize("log_r,G", CASES)
def test_model_of_warp_rows_equals_oracle(log_r, G):
    o = oracle.get()
    R = 1 << log_r
    w = o.root_of_unity(P, R)
    rng = np.random.default_rng(log_r * 10 + G)
    rows = rng.integers(0, P, size=(G, R), dtype=np.uint64)
    assert np.array_equal(model(rows, False, log_r, stage_tables(w, R)), o.ntt_ref(P, w, rows))
    assert np.array_equal(model(rows, True, log_r, stage_tables(o.invmod(w, P), R)), o.intt_ref(P, w, rows))


@pytest.mark.parametrize("log_r,G,mutate", [(6, 1, 1), (8, 1, 1), (6, 1, 2), (6, 4, 2), (8, 4, 2)])
def test_model_detects_lane_exchange_mistakes(log_r, G, mutate):
    """Negative controls: an index mistake planted in the lane exchange (the
    wrong twiddle for the upper lane's pair, or the returned half written to
    the other register) breaks agreement with the oracle."""
    o = oracle.get()
    R = 1 << log_r
    w = o.root_of_unity(P, R)
    rows = np.random.default_rng(5).integers(0, P, size=(G, R), dtype=np.uint64)
    assert not np.array_equal(model(rows, False, log_r, stage_tables(w, R), mutate=mutate), o.ntt_ref(P, w, rows))


@pytest.mark.parametrize("word_bytes", [4, 8])
def test_warp_row_launch_geometry(word_bytes):
    """Every row is visited exactly once by the grid-stride loop over groups
    of G rows (ragged ends included), and a CTA's shared memory (G rows of
    R + R/32 words per warp) stays within the per-CTA limit."""
    for log_r in range(5, 11):
        R = 1 << log_r
        g_max = group_rows(word_bytes, log_r)
        for G in sorted({1, g_max}):
            assert CTA_WARPS * G * (R + R // 32) * word_bytes <= SMEM_LIMIT
            for nrows in (1, 7, 8 * G + 3, G * CTA_WARPS * 152 * 2 + 5, 300_001):
                groups = -(-nrows // G)
                grid = max(1, min(-(-groups // CTA_WARPS), GRID_CAP))
                seen = np.zeros(nrows, dtype=np.int64)
                for cta_warp in range(grid * CTA_WARPS):
                    row0 = cta_warp * G
                    while row0 < nrows:
                        hi = min(row0 + G, nrows)
                        seen[row0:hi] += 1
                        row0 += grid * CTA_WARPS * G
                assert np.all(seen == 1), (word_bytes, log_r, G, nrows)
