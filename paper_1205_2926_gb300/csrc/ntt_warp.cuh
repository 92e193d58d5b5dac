// ntt_warp.cuh -- the row pass with one warp per row: register blocks of up
// to 32 words per thread, exchanged inside the warp.
//
// A row of R = 2^LOGR words (2^5 <= R <= 2^10) belongs to one warp; each of
// its 32 threads holds n = R/32 words in registers, in one of two layouts:
//   layout A: element i = lane + 32 k   (k < n)
//   layout B: element i = n lane + k
// Forward (Algorithm 1's stages, distances R/2 .. 1): load in layout A; the
// stages of distance m >= 32 pair registers of one thread; a transpose
// through the warp's own stretch of shared memory (one __syncwarp, no block
// barrier) gives layout B; the stages n <= m < 32 pair lanes l and l ^ (m/n),
// exchanged by __shfl_xor_sync; the stages m < n pair registers again.  The
// inverse (Algorithm 1 backwards, distances 1 .. R/2) runs the same steps in
// reverse order, B to A.  The stage twiddle of the pair (i, i + m) is
// tw[m + (i mod m)], the table of the other pass kernels.
//
// A warp may own G rows at once (G > 1 for batched passes with many rows):
// each twiddle load then serves G butterflies, and G rows' loads are in
// flight together.  In a lane-exchange stage two register words form a pair
// of butterflies (word k of rows g and g + 1, or words k and k + 1 of one
// row): the lower lane computes the first butterfly and the upper lane the
// second, each after one shuffle brings it the partner's word, and a second
// shuffle returns the half that the other lane holds -- half a butterfly per
// word and lane, against a whole one when both lanes compute the same pair
// (what a single word per thread and row, R = 2^5 with G = 1, still does).
// Shared memory is padded by one word per 32 (element i at i + i/32), which
// makes both transposes free of bank conflicts.
#pragma once

#include "ntt_kernels.cuh"

namespace ntt {

template <typename W, int LOGR>
__device__ __forceinline__ W *warp_row_ptr(const PassArgs<W> &a, uint64_t row) {
    if (a.rowptrs) return a.rowptrs[row];
    const int shift = a.logL - LOGR;
    return a.data + (row >> shift) * a.stride + ((row & ((1ull << shift) - 1ull)) << LOGR);
}

__device__ __forceinline__ uint32_t warp_pad(uint32_t i) { return i + (i >> 5); }

constexpr int kWarpRowsPerCta = 8;  // warps (256 threads) per CTA

// Rows per warp of the batched form: up to 32 (32-bit) or 16 (64-bit) words
// per thread, at most 8 rows.
template <typename W, int LOGR>
struct WarpGroup {
    static constexpr int N = (1 << LOGR) / 32;
    static constexpr int WORDS = sizeof(W) == 4 ? 32 : 16;
    static constexpr int G = N >= WORDS ? 1 : (WORDS / N > 8 ? 8 : WORDS / N);
};

template <typename W, int DIR, int VAR, int LOGR, int G>
__device__ __forceinline__ void warp_stages_a(W (&x)[G][(1 << LOGR) / 32], const PassArgs<W> &a, int lane) {
    // distances m = 2^lm >= 32: register distance h = m / 32
    constexpr int N = (1 << LOGR) / 32;
    const W p = a.p, p2 = (W)(2 * a.p);
#pragma unroll
    for (int step = 0; step < LOGR - 5; ++step) {
        const int lm = DIR == DIR_FWD ? LOGR - 1 - step : 5 + step;
        const int h = 1 << (lm - 5);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (k & h) continue;
            W w, wq;
            ld_pair(a.tw, (1 << lm) + lane + 32 * (k & (h - 1)), w, wq);
#pragma unroll
            for (int g = 0; g < G; ++g) bfly<W, DIR, VAR>(x[g][k], x[g][k + h], w, wq, p, p2, a.J);
        }
    }
}

// One pair of butterflies across lanes l and l ^ lb: the lower lane computes
// the butterfly of word xa (its own xa is the pair's first element, the
// partner's xa the second), the upper lane that of word xb (the partner's xb
// first, its own second); ta / tb are their twiddle indices.
template <typename W, int DIR, int VAR>
__device__ __forceinline__ void lane_pair(W &xa, W &xb, int ta, int tb, bool upper, int lb, const PassArgs<W> &a) {
    const W p = a.p, p2 = (W)(2 * a.p);
    const W r = __shfl_xor_sync(0xffffffffu, upper ? xa : xb, lb);
    W lo = upper ? r : xa, hi = upper ? xb : r;
    W w, wq;
    ld_pair(a.tw, upper ? tb : ta, w, wq);
    bfly<W, DIR, VAR>(lo, hi, w, wq, p, p2, a.J);
    const W back = __shfl_xor_sync(0xffffffffu, upper ? lo : hi, lb);
    xa = upper ? back : lo;
    xb = upper ? hi : back;
}

template <typename W, int DIR, int VAR, int LOGR, int G>
__device__ __forceinline__ void warp_stages_lanes(W (&x)[G][(1 << LOGR) / 32], const PassArgs<W> &a, int lane) {
    // distances n <= m < 32: lane distance m / n
    constexpr int N = (1 << LOGR) / 32;
    constexpr int LOGN = LOGR - 5;
    const W p = a.p, p2 = (W)(2 * a.p);
#pragma unroll
    for (int step = 0; step < 5 - LOGN; ++step) {
        const int lm = DIR == DIR_FWD ? 4 - step : LOGN + step;
        const int m = 1 << lm, lb = m / N;
        const bool upper = (lane & lb) != 0;
        const int llo = lane & ~lb;
        if constexpr (G >= 2) {
            // word k of rows g and g + 1: one twiddle for both lanes
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int t = m + ((N * llo + k) & (m - 1));
#pragma unroll
                for (int g = 0; g + 1 < G; g += 2) lane_pair<W, DIR, VAR>(x[g][k], x[g + 1][k], t, t, upper, lb, a);
            }
        } else if constexpr (N >= 2) {
            // words k and k + 1 of the one row
#pragma unroll
            for (int k = 0; k < N; k += 2)
                lane_pair<W, DIR, VAR>(x[0][k], x[0][k + 1], m + ((N * llo + k) & (m - 1)),
                                       m + ((N * llo + k + 1) & (m - 1)), upper, lb, a);
        } else {
            // a single word: both lanes compute the pair, each keeps its half
            const W v = x[0][0];
            const W u = __shfl_xor_sync(0xffffffffu, v, lb);
            W lo = upper ? u : v, hi = upper ? v : u;
            W w, wq;
            ld_pair(a.tw, m + (llo & (m - 1)), w, wq);
            bfly<W, DIR, VAR>(lo, hi, w, wq, p, p2, a.J);
            x[0][0] = upper ? hi : lo;
        }
    }
}

template <typename W, int DIR, int VAR, int LOGR, int G>
__device__ __forceinline__ void warp_stages_b(W (&x)[G][(1 << LOGR) / 32], const PassArgs<W> &a) {
    // distances m < n: register distance m; the twiddle index k mod m is the
    // same in every lane
    constexpr int N = (1 << LOGR) / 32;
    constexpr int LOGN = LOGR - 5;
    const W p = a.p, p2 = (W)(2 * a.p);
#pragma unroll
    for (int step = 0; step < LOGN; ++step) {
        const int lm = DIR == DIR_FWD ? LOGN - 1 - step : step;
        const int m = 1 << lm;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (k & m) continue;
            W w, wq;
            ld_pair(a.tw, m + (k & (m - 1)), w, wq);
#pragma unroll
            for (int g = 0; g < G; ++g) bfly<W, DIR, VAR>(x[g][k], x[g][k + m], w, wq, p, p2, a.J);
        }
    }
}

// G rows per warp, kWarpRowsPerCta warps per CTA, a grid-stride loop over
// groups of G consecutive rows (rows past nrows are neither read nor
// written).  Dynamic shared memory: kWarpRowsPerCta * G * (R + R/32) words.
template <typename W, int DIR, int VAR, int LOGR, int G>
__global__ void __launch_bounds__(kWarpRowsPerCta * 32) k_warp_row(const PassArgs<W> a) {
    constexpr int R = 1 << LOGR;
    constexpr int N = R / 32;
    constexpr int V = Lanes<W>::V;  // words per 16-byte vector
    extern __shared__ uint4 wsm_raw[];
    W *wsm = reinterpret_cast<W *>(wsm_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    W *sw = wsm + warp * G * (R + R / 32);
    const W p = a.p, p2 = (W)(2 * a.p);
    for (uint64_t row0 = ((uint64_t)blockIdx.x * kWarpRowsPerCta + warp) * G; row0 < a.nrows;
         row0 += (uint64_t)gridDim.x * kWarpRowsPerCta * G) {
        W x[G][N];
        if (DIR == DIR_FWD) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (row0 + g < a.nrows) {
                    const W *src = warp_row_ptr<W, LOGR>(a, row0 + g);
#pragma unroll
                    for (int k = 0; k < N; ++k) x[g][k] = __ldcg(src + lane + 32 * k);
                } else {
#pragma unroll
                    for (int k = 0; k < N; ++k) x[g][k] = 0;
                }
            }
            warp_stages_a<W, DIR, VAR, LOGR, G>(x, a, lane);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < N; ++k) sw[g * (R + R / 32) + warp_pad(lane + 32 * k)] = x[g][k];
            __syncwarp();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < N; ++k) x[g][k] = sw[g * (R + R / 32) + warp_pad(N * lane + k)];
            __syncwarp();  // every read done before the warp's next group writes
            warp_stages_lanes<W, DIR, VAR, LOGR, G>(x, a, lane);
            warp_stages_b<W, DIR, VAR, LOGR, G>(x, a);
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (row0 + g < a.nrows) {
                    const W *src = warp_row_ptr<W, LOGR>(a, row0 + g);
                    if (N % V == 0) {
#pragma unroll
                        for (int q = 0; q < N / V; ++q) {
                            W c[V];
                            unpack(__ldcg(reinterpret_cast<const uint4 *>(src + N * lane) + q), c);
#pragma unroll
                            for (int v = 0; v < V; ++v) x[g][q * V + v] = c[v];
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < N; ++k) x[g][k] = __ldcg(src + N * lane + k);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < N; ++k) x[g][k] = 0;
                }
            }
            warp_stages_b<W, DIR, VAR, LOGR, G>(x, a);
            warp_stages_lanes<W, DIR, VAR, LOGR, G>(x, a, lane);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < N; ++k) sw[g * (R + R / 32) + warp_pad(N * lane + k)] = x[g][k];
            __syncwarp();
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < N; ++k) x[g][k] = sw[g * (R + R / 32) + warp_pad(lane + 32 * k)];
            __syncwarp();
            warp_stages_a<W, DIR, VAR, LOGR, G>(x, a, lane);
        }
        if ((a.flags & F_NORMALIZE) && !Reduced<VAR>::ON) {
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int k = 0; k < N; ++k)
                    x[g][k] = DIR == DIR_FWD ? reduce2(x[g][k], p) : reduce4(x[g][k], p, p2);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (row0 + g >= a.nrows) continue;
            W *dst = warp_row_ptr<W, LOGR>(a, row0 + g);
            if (DIR == DIR_FWD) {
                // layout B: each thread's n words are consecutive
                if (N % V == 0) {
#pragma unroll
                    for (int q = 0; q < N / V; ++q) {
                        W c[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) c[v] = x[g][q * V + v];
                        *(reinterpret_cast<uint4 *>(dst + N * lane) + q) = pack<W>(c);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < N; ++k) dst[N * lane + k] = x[g][k];
                }
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) dst[lane + 32 * k] = x[g][k];  // layout A: coalesced words
            }
        }
    }
}

}  // namespace ntt
