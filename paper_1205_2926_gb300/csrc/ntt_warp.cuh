// ntt_warp.cuh -- the row pass with one warp per row: register blocks of up
// to 32 elements per thread, exchanged inside the warp.
//
// A row of R = 2^LOGR words (2^5 <= R <= 2^10) is one warp's; each of its 32
// threads holds n = R/32 words in registers, in one of two layouts:
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
// In the lane-exchange stages both lanes of a pair compute the whole
// butterfly from the two words and keep their own half, so those stages cost
// a butterfly per word instead of per pair; the other stages cost what they
// do in the radix-8 kernels.  Shared memory is padded by one word per 32
// (element i at i + i/32), which makes both transposes conflict-free.
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

constexpr int kWarpRowsPerCta = 8;  // 256 threads

template <typename W, int DIR, int VAR, int LOGR>
__device__ __forceinline__ void warp_stages_a(W (&x)[(1 << LOGR) / 32], const PassArgs<W> &a, int lane) {
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
            bfly<W, DIR, VAR>(x[k], x[k + h], w, wq, p, p2, a.J);
        }
    }
}

template <typename W, int DIR, int VAR, int LOGR>
__device__ __forceinline__ void warp_stages_lanes(W (&x)[(1 << LOGR) / 32], const PassArgs<W> &a, int lane) {
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
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const W v = x[k];
            const W u = __shfl_xor_sync(0xffffffffu, v, lb);
            W lo = upper ? u : v, hi = upper ? v : u;
            W w, wq;
            ld_pair(a.tw, m + ((N * llo + k) & (m - 1)), w, wq);
            bfly<W, DIR, VAR>(lo, hi, w, wq, p, p2, a.J);
            x[k] = upper ? hi : lo;
        }
    }
}

template <typename W, int DIR, int VAR, int LOGR>
__device__ __forceinline__ void warp_stages_b(W (&x)[(1 << LOGR) / 32], const PassArgs<W> &a) {
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
            bfly<W, DIR, VAR>(x[k], x[k + m], w, wq, p, p2, a.J);
        }
    }
}

template <typename W, int DIR, int VAR, int LOGR>
__global__ void __launch_bounds__(kWarpRowsPerCta * 32) k_warp_row(const PassArgs<W> a) {
    constexpr int R = 1 << LOGR;
    constexpr int N = R / 32;
    constexpr int V = Lanes<W>::V;  // words per 16-byte vector
    extern __shared__ uint4 wsm_raw[];
    W *wsm = reinterpret_cast<W *>(wsm_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    W *sw = wsm + warp * (R + R / 32);
    const W p = a.p, p2 = (W)(2 * a.p);
    for (uint64_t row = (uint64_t)blockIdx.x * kWarpRowsPerCta + warp; row < a.nrows;
         row += (uint64_t)gridDim.x * kWarpRowsPerCta) {
        W *g = warp_row_ptr<W, LOGR>(a, row);
        W x[N];
        if (DIR == DIR_FWD) {
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] = __ldcg(g + lane + 32 * k);
            warp_stages_a<W, DIR, VAR, LOGR>(x, a, lane);
#pragma unroll
            for (int k = 0; k < N; ++k) sw[warp_pad(lane + 32 * k)] = x[k];
            __syncwarp();
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] = sw[warp_pad(N * lane + k)];
            __syncwarp();  // every read done before the warp's next row writes
            warp_stages_lanes<W, DIR, VAR, LOGR>(x, a, lane);
            warp_stages_b<W, DIR, VAR, LOGR>(x, a);
        } else {
            if (N % V == 0) {
#pragma unroll
                for (int q = 0; q < N / V; ++q) {
                    W c[V];
                    unpack(__ldcg(reinterpret_cast<const uint4 *>(g + N * lane) + q), c);
#pragma unroll
                    for (int v = 0; v < V; ++v) x[q * V + v] = c[v];
                }
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) x[k] = __ldcg(g + N * lane + k);
            }
            warp_stages_b<W, DIR, VAR, LOGR>(x, a);
            warp_stages_lanes<W, DIR, VAR, LOGR>(x, a, lane);
#pragma unroll
            for (int k = 0; k < N; ++k) sw[warp_pad(N * lane + k)] = x[k];
            __syncwarp();
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] = sw[warp_pad(lane + 32 * k)];
            __syncwarp();
            warp_stages_a<W, DIR, VAR, LOGR>(x, a, lane);
        }
        if ((a.flags & F_NORMALIZE) && !Reduced<VAR>::ON) {
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] = DIR == DIR_FWD ? reduce2(x[k], p) : reduce4(x[k], p, p2);
        }
        if (DIR == DIR_FWD) {
            // layout B: each thread's n words are consecutive
            if (N % V == 0) {
#pragma unroll
                for (int q = 0; q < N / V; ++q) {
                    W c[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) c[v] = x[q * V + v];
                    *(reinterpret_cast<uint4 *>(g + N * lane) + q) = pack<W>(c);
                }
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) g[N * lane + k] = x[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < N; ++k) g[lane + 32 * k] = x[k];  // layout A: coalesced words
        }
    }
}

}  // namespace ntt
