// ntt_kernels.cuh -- sm_103a kernels of the batched NTT.
//
// Schedule.  Algorithm 1 (Section 1) is a radix-2 decimation-in-frequency
// transform: stage i pairs x[t+k] with x[t+k+m], m = 2^(l-i), twiddle
// zeta^k = omega^(k L / 2m).  A transform of length L = 2^l is cut into
// passes of l_0 + l_1 + ... = l stages (the four-step split, applied
// recursively).  With B_q the block length at pass q, R_q = 2^(l_q) and
// S_q = B_q / R_q, pass q runs, for every block and every column c < S_q, an
// R_q-point DIF transform over the elements blk*B_q + s*S_q + c (s < R_q),
// leaving them in bit-reversed order, and then multiplies element (s, c) by
// the middle twiddle omega^((L/B_q) c rev(s)); the last pass (S = 1) works on
// contiguous rows.  The result is Algorithm 1's bit-reversed DFT exactly.
// The inverse runs the passes backwards: row pass first, then each column
// pass multiplies by the inverse middle twiddle and runs the DIT stages of
// Algorithm 1 backwards (Section 4).
//
// Stage twiddles.  In an R-point sub-transform the stage of distance m uses
// omega_R^(k R / 2m) = omega^(k L / 2m): the same value as in the full-length
// Algorithm 1, independent of R.  One table tw[m - 1 + k] = (W, W') for
// k < m, m = 1, 2, 4, ... serves every pass (Shoup quotients W' =
// floor(W beta / p), Algorithms 2-4).
//
// On-chip work.  A CTA stages its tile in shared memory as 16-byte vectors
// of V words (V = 4 for 32-bit, 2 for 64-bit words); the V words of a vector
// belong to V independent sub-transforms that share every twiddle.  Each
// thread works on E = 8 vectors at a time in registers (a radix-8 block: up
// to three butterfly stages per round), then writes them back; rounds are
// separated by __syncthreads().  Global loads and stores are 16-byte and
// coalesced.
//
// Butterflies: Algorithm 3 / Algorithm 4 (lazy, redundant [0,2p) / [0,4p))
// or Algorithm 2 / its fully reduced inverse (the NTL-style baseline).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace ntt {

enum { DIR_FWD = 0, DIR_INV = 1 };
enum { VAR_LAZY = 0, VAR_NTL = 1 };
enum { F_NORMALIZE = 1, F_MIDDLE = 2, F_MB = 4 };

constexpr int kThreads = 256;  // threads per CTA of the pass kernels
constexpr int kE = 8;          // vectors per thread per round (radix-8 blocks)
constexpr int kLogE = 3;

template <typename W>
struct Lanes {
    static constexpr int V = 16 / sizeof(W);  // words per 16-byte vector
    static constexpr int LOGV = V == 4 ? 2 : 1;
};

// Arguments of one pass over a batch of transforms.
template <typename W>
struct PassArgs {
    W *data;          // transform 0
    uint64_t stride;  // words between consecutive transforms
    uint32_t batch;
    int32_t logL;
    int32_t logR;     // sub-transform length of this pass
    int32_t logS;     // column stride (0 for the contiguous row pass)
    int32_t per_cta;  // column pass: tiles per CTA; row pass: vector groups per CTA
    int32_t logTV;    // column pass: 16-byte vectors per tile row (tile width T = TV * V words)
    int32_t logTA;    // column pass: width of the middle-twiddle table MA (TA >= T)
    uint32_t flags;   // F_NORMALIZE | F_MIDDLE | F_MB
    const W *tw;      // stage twiddle pairs, forward or inverse roots
    const W *ma;      // middle twiddle pairs MA[s][c mod TA]
    const W *mb;      // middle twiddle pairs MB[c / TA][s]
    W p;
    uint64_t nrows;   // row pass: number of rows (batch * L / R)
    W *const *rowptrs;  // row pass over single-row transforms: address of each row (else null)
};

template <typename W>
__device__ __forceinline__ void load_pair(const W *__restrict__ t, uint32_t idx, W &w, W &wq);

template <>
__device__ __forceinline__ void load_pair<uint32_t>(const uint32_t *__restrict__ t, uint32_t idx, uint32_t &w,
                                                    uint32_t &wq) {
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(t) + idx);
    w = v.x;
    wq = v.y;
}

template <>
__device__ __forceinline__ void load_pair<uint64_t>(const uint64_t *__restrict__ t, uint32_t idx, uint64_t &w,
                                                    uint64_t &wq) {
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(t) + idx);
    w = v.x;
    wq = v.y;
}

template <typename W>
__device__ __forceinline__ void unpack(const uint4 &c, W (&x)[Lanes<W>::V]) {
    const W *px = reinterpret_cast<const W *>(&c);
#pragma unroll
    for (int v = 0; v < Lanes<W>::V; ++v) x[v] = px[v];
}

template <typename W>
__device__ __forceinline__ uint4 pack(const W (&x)[Lanes<W>::V]) {
    uint4 c;
    W *px = reinterpret_cast<W *>(&c);
#pragma unroll
    for (int v = 0; v < Lanes<W>::V; ++v) px[v] = x[v];
    return c;
}

// Round geometry: the thread's E vectors are s_j = hi | (j << b0) | lo with
// (hi, lo) taken from the unit index g; the round executes `nst` of the
// three stage bits b0+2, b0+1, b0 (the top ones when nst < 3).
struct Round {
    int b0, nst;
};

__device__ __forceinline__ Round round_geometry(int dir, int r, int nrounds, int logR) {
    int e0 = logR - kLogE * (nrounds - 1);  // 1..3 stages in the partial round
    Round g;
    if (dir == DIR_FWD) {
        g.b0 = r == 0 ? logR - kLogE : logR - e0 - kLogE * r;
        g.nst = r == 0 ? e0 : kLogE;
    } else {
        g.b0 = r == nrounds - 1 ? logR - kLogE : kLogE * r;
        g.nst = r == nrounds - 1 ? e0 : kLogE;
    }
    return g;
}

__device__ __forceinline__ uint32_t elem_index(uint32_t g, int b0, int j) {
    uint32_t lo = g & ((1u << b0) - 1u);
    return ((g >> b0) << (b0 + kLogE)) | ((uint32_t)j << b0) | lo;
}

// Butterfly stages of one round on E vectors held in registers.
template <typename W, int DIR, int VAR>
__device__ __forceinline__ void round_stages(W (&x)[kE][Lanes<W>::V], int b0, int nst, uint32_t lo,
                                             const W *__restrict__ tw, W p, W p2) {
    constexpr int V = Lanes<W>::V;
    if (DIR == DIR_FWD) {
#pragma unroll
        for (int lb = kLogE - 1; lb >= 0; --lb) {
            if (lb >= kLogE - nst) {
#pragma unroll
                for (int jl = 0; jl < (1 << lb); ++jl) {
                    uint32_t idx = (1u << (b0 + lb)) - 1u + (((uint32_t)jl << b0) | lo);
                    W w, wq;
                    load_pair(tw, idx, w, wq);
#pragma unroll
                    for (int jh = 0; jh < kE; jh += (2 << lb)) {
                        const int j = jh + jl, j2 = j + (1 << lb);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            if (VAR == VAR_LAZY)
                                bfly_fwd_lazy(x[j][v], x[j2][v], w, wq, p, p2);
                            else
                                bfly_fwd_ntl(x[j][v], x[j2][v], w, wq, p);
                        }
                    }
                }
            }
        }
    } else {
#pragma unroll
        for (int lb = 0; lb < kLogE; ++lb) {
            if (lb >= kLogE - nst) {
#pragma unroll
                for (int jl = 0; jl < (1 << lb); ++jl) {
                    uint32_t idx = (1u << (b0 + lb)) - 1u + (((uint32_t)jl << b0) | lo);
                    W w, wq;
                    load_pair(tw, idx, w, wq);
#pragma unroll
                    for (int jh = 0; jh < kE; jh += (2 << lb)) {
                        const int j = jh + jl, j2 = j + (1 << lb);
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            if (VAR == VAR_LAZY)
                                bfly_inv_lazy(x[j][v], x[j2][v], w, wq, p, p2);
                            else
                                bfly_inv_ntl(x[j][v], x[j2][v], w, wq, p);
                        }
                    }
                }
            }
        }
    }
}

template <typename W, int VAR>
__device__ __forceinline__ W mul_twiddle(W x, W w, W wq, W p) {
    W y = shoup_mul(x, w, wq, p);  // any x < beta -> [0, 2p)
    return VAR == VAR_NTL ? csub(y, p) : y;
}

// Middle twiddle of a column pass, omega^((L/B) c rev(s)), on the E vectors
// of rows s = 8 g + j (the round with b0 = 0), columns
// c = ct*T + tv*V + v.  It is factored as MB[c >> logTA][s] * MA[s][c mod TA]
// (two Shoup products) so that both tables stay near 2 R sqrt(S) entries.
template <typename W, int VAR>
__device__ __forceinline__ void middle_twiddle(W (&x)[kE][Lanes<W>::V], uint32_t g, uint32_t tv, uint32_t ct,
                                               const PassArgs<W> &a) {
    constexpr int V = Lanes<W>::V;
    const uint32_t R = 1u << a.logR;
    const uint32_t c0 = (ct << (a.logTV + Lanes<W>::LOGV)) + tv * V;  // first column of this vector
    const uint32_t TAm = (1u << a.logTA) - 1u;
    const uint32_t chi = c0 >> a.logTA;
#pragma unroll
    for (int j = 0; j < kE; ++j) {
        const uint32_t s = (g << kLogE) | j;
        if (a.flags & F_MB) {
            W w, wq;
            load_pair(a.mb, chi * R + s, w, wq);
#pragma unroll
            for (int v = 0; v < V; ++v) x[j][v] = mul_twiddle<W, VAR>(x[j][v], w, wq, a.p);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            W w, wq;
            load_pair(a.ma, (s << a.logTA) + ((c0 + v) & TAm), w, wq);
            x[j][v] = mul_twiddle<W, VAR>(x[j][v], w, wq, a.p);
        }
    }
}

template <typename W, int DIR, int VAR>
__device__ __forceinline__ void normalize(W (&x)[kE][Lanes<W>::V], W p, W p2) {
#pragma unroll
    for (int j = 0; j < kE; ++j)
#pragma unroll
        for (int v = 0; v < Lanes<W>::V; ++v) {
            if (VAR == VAR_LAZY) x[j][v] = DIR == DIR_FWD ? reduce2(x[j][v], p) : reduce4(x[j][v], p, p2);
        }
}

__device__ __forceinline__ uint4 ldg16(const void *p) { return *reinterpret_cast<const uint4 *>(p); }
// Load that bypasses L1: data written earlier in the same launch by other
// CTAs (the persistent uneven-batch kernel) must not be served from a stale
// L1 line.
__device__ __forceinline__ uint4 ldcg16(const void *p) { return __ldcg(reinterpret_cast<const uint4 *>(p)); }
__device__ __forceinline__ void stg16(void *p, const uint4 &v) { *reinterpret_cast<uint4 *>(p) = v; }

// ---------------------------------------------------------------------------
// Shared-memory layout of a tile: R rows (elements s of the sub-transforms)
// x TV 16-byte vectors per row.  Vector (s, tv) sits at chunk
//     (s*TV + tv) ^ (((s >> 3) * TV) & 7),
// an XOR swizzle inside aligned groups of 8 chunks.  For TV in {1,2,4,8} and
// every round geometry, the 8 threads of a quarter-warp then touch 8
// distinct bank groups, so the 16-byte shared loads and stores of the
// rounds are conflict-free (checked exhaustively for R = 2^3 .. 2^12).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t chunk_at(uint32_t s, uint32_t tv, int logTV) {
    return ((s << logTV) + tv) ^ (((s >> 3) << logTV) & 7u);
}

// Column pass (ROW = false): a tile is R rows x TV vectors (T = TV*V
// consecutive columns) of one block; global row s of the tile is TV*16
// contiguous bytes.  Row pass (ROW = true, TV = 1): a "vector group" is V
// consecutive rows of length R, vector s holding element s of each.
template <typename W>
__device__ __forceinline__ W *row_ptr(const PassArgs<W> &a, uint64_t row) {
    if (a.rowptrs) return a.rowptrs[row];
    const int shift = a.logL - a.logR;  // rows per transform = 2^shift
    const uint64_t b = row >> shift, within = row & ((1ull << shift) - 1ull);
    return a.data + b * a.stride + (within << a.logR);
}

template <typename W, bool STORE, bool COH>
__device__ __forceinline__ void row_copy(const PassArgs<W> &a, uint4 *sm, uint64_t row0, int groups) {
    constexpr int V = Lanes<W>::V, LOGV = Lanes<W>::LOGV;
    const int logR = a.logR;
    const uint32_t R = 1u << logR;
    const int logn16 = logR - LOGV;             // 16-byte chunks per row
    const uint32_t total = (uint32_t)groups << logR;  // groups * V rows * R/V chunks
    for (uint32_t i = threadIdx.x; i < total; i += kThreads) {
        uint32_t c, v, grp;
        if (logn16 >= 3) {  // 8 consecutive threads cover 128 contiguous bytes of one row
            c = (i & 7) | (((i >> (3 + LOGV)) & ((1u << (logn16 - 3)) - 1)) << 3);
            v = (i >> 3) & (V - 1);
        } else {
            c = i & ((1u << logn16) - 1);
            v = (i >> logn16) & (V - 1);
        }
        grp = i >> logR;
        const uint64_t row = row0 + grp * V + v;
        if (row >= a.nrows) continue;
        W *g = row_ptr(a, row) + c * V;
        W *base = reinterpret_cast<W *>(sm + grp * R);
        if (!STORE) {
            uint4 q = COH ? ldcg16(g) : ldg16(g);
            const W *pq = reinterpret_cast<const W *>(&q);
#pragma unroll
            for (int k = 0; k < V; ++k) base[chunk_at(c * V + k, 0, 0) * V + v] = pq[k];
        } else {
            uint4 q;
            W *pq = reinterpret_cast<W *>(&q);
#pragma unroll
            for (int k = 0; k < V; ++k) pq[k] = base[chunk_at(c * V + k, 0, 0) * V + v];
            stg16(g, q);
        }
    }
}

// Tile t of a column pass -> (transform b, block blk, column tile ct); all
// counts are powers of two: 2^ltb tiles per block, 2^lbt blocks per transform.
template <typename W>
struct ColTile {
    int ltb, lbt;
    __device__ __forceinline__ W *origin(const PassArgs<W> &a, uint32_t t, uint32_t &ct) const {
        ct = t & ((1u << ltb) - 1u);
        const uint32_t blk = (t >> ltb) & ((1u << lbt) - 1u), b = t >> (ltb + lbt);
        return a.data + (uint64_t)b * a.stride + ((uint64_t)blk << (a.logR + a.logS)) +
               ((uint64_t)ct << (a.logTV + Lanes<W>::LOGV));
    }
};

template <typename W, bool STORE, bool COH>
__device__ __forceinline__ void col_copy(const PassArgs<W> &a, uint4 *sm, const ColTile<W> &ct_info, uint32_t tile0,
                                         int ntile) {
    constexpr int V = Lanes<W>::V;
    const int logR = a.logR, logTV = a.logTV;
    const uint32_t R = 1u << logR, TV = 1u << logTV;
    const uint64_t S = 1ull << a.logS;
    const uint32_t total = (uint32_t)ntile << (logR + logTV);
    for (uint32_t i = threadIdx.x; i < total; i += kThreads) {
        const uint32_t cc = i & (TV - 1), s = (i >> logTV) & (R - 1), ti = i >> (logTV + logR);
        uint32_t ct;
        W *g = ct_info.origin(a, tile0 + ti, ct) + s * S + cc * V;
        uint4 *slot = sm + (ti << (logR + logTV)) + chunk_at(s, cc, logTV);
        if (!STORE)
            *slot = COH ? ldcg16(g) : ldg16(g);
        else
            stg16(g, *slot);
    }
}

// The work of one CTA in one pass.  Column pass: CTA `cta` takes tiles
// cta*per_cta ...; row pass: vector groups cta*per_cta ... (per_cta * V
// rows).  Unit u of a round -> (tile or group ti, vector tv, element group g).
// COH selects L1-bypassing loads (needed when other CTAs of the same launch
// produced the input).
template <typename W, int DIR, int VAR, bool ROW, bool COH>
__device__ __forceinline__ void pass_cta(const PassArgs<W> &a, uint32_t cta, uint4 *sm) {
    constexpr int V = Lanes<W>::V;
    const int logR = a.logR;
    const int logTV = ROW ? 0 : a.logTV;
    const uint32_t R = 1u << logR;
    const W p = a.p, p2 = (W)(2 * a.p);
    const int nrounds = (logR + kLogE - 1) / kLogE;

    ColTile<W> cti;
    cti.ltb = 0;
    uint32_t tile0 = 0;
    int ntile = a.per_cta;
    uint64_t row0 = 0;
    if (ROW) {
        row0 = (uint64_t)cta * a.per_cta * V;
        row_copy<W, false, COH>(a, sm, row0, a.per_cta);
    } else {
        cti.ltb = a.logS - a.logTV - Lanes<W>::LOGV;
        cti.lbt = a.logL - logR - a.logS;
        const uint32_t tiles_total = a.batch << (cti.ltb + cti.lbt);
        tile0 = cta * a.per_cta;
        ntile = min((uint32_t)a.per_cta, tiles_total - tile0);
        col_copy<W, false, COH>(a, sm, cti, tile0, ntile);
    }
    __syncthreads();

    const uint32_t units = (uint32_t)ntile << (logR - kLogE + logTV);
    for (int r = 0; r < nrounds; ++r) {
        const Round rg = round_geometry(DIR, r, nrounds, logR);
        for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
            const uint32_t tv = u & ((1u << logTV) - 1u);
            const uint32_t g = (u >> logTV) & ((R >> kLogE) - 1u);
            const uint32_t ti = u >> (logTV + logR - kLogE);
            uint4 *tsm = sm + (ti << (logR + logTV));
            W x[kE][V];
#pragma unroll
            for (int j = 0; j < kE; ++j) unpack(tsm[chunk_at(elem_index(g, rg.b0, j), tv, logTV)], x[j]);
            if (!ROW && (a.flags & F_MIDDLE) && ((DIR == DIR_INV && r == 0) || (DIR == DIR_FWD && r == nrounds - 1))) {
                if (DIR == DIR_FWD)
                    round_stages<W, DIR, VAR>(x, rg.b0, rg.nst, g & ((1u << rg.b0) - 1u), a.tw, p, p2);
                const uint32_t ct = (tile0 + ti) & ((1u << cti.ltb) - 1u);
                middle_twiddle<W, VAR>(x, g, tv, ct, a);
                if (DIR == DIR_INV)
                    round_stages<W, DIR, VAR>(x, rg.b0, rg.nst, g & ((1u << rg.b0) - 1u), a.tw, p, p2);
            } else {
                round_stages<W, DIR, VAR>(x, rg.b0, rg.nst, g & ((1u << rg.b0) - 1u), a.tw, p, p2);
            }
            if (r == nrounds - 1 && (a.flags & F_NORMALIZE)) normalize<W, DIR, VAR>(x, p, p2);
#pragma unroll
            for (int j = 0; j < kE; ++j) tsm[chunk_at(elem_index(g, rg.b0, j), tv, logTV)] = pack<W>(x[j]);
        }
        __syncthreads();
    }

    if (ROW)
        row_copy<W, true, COH>(a, sm, row0, a.per_cta);
    else
        col_copy<W, true, COH>(a, sm, cti, tile0, ntile);
}

// One pass over a batch, one CTA per `per_cta` tiles (or groups).
template <typename W, int DIR, int VAR, bool ROW>
__global__ void __launch_bounds__(kThreads) k_pass(const PassArgs<W> a) {
    extern __shared__ uint4 sm[];
    pass_cta<W, DIR, VAR, ROW, false>(a, blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// Lengths 2 and 4: one thread per transform, Algorithm 1 directly.
// ---------------------------------------------------------------------------
template <typename W, int DIR, int VAR>
__global__ void k_tiny(const PassArgs<W> a) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.batch) return;
    const W p = a.p, p2 = (W)(2 * a.p);
    const int L = 1 << a.logL;
    W *d = a.data + b * a.stride;
    W x[4];
    for (int i = 0; i < L; ++i) x[i] = d[i];
    if (DIR == DIR_FWD) {
        for (int m = L / 2; m >= 1; m >>= 1)
            for (int t = 0; t < L; t += 2 * m)
                for (int k = 0; k < m; ++k) {
                    W w, wq;
                    load_pair(a.tw, m - 1 + k, w, wq);
                    if (VAR == VAR_LAZY)
                        bfly_fwd_lazy(x[t + k], x[t + k + m], w, wq, p, p2);
                    else
                        bfly_fwd_ntl(x[t + k], x[t + k + m], w, wq, p);
                }
    } else {
        for (int m = 1; m < L; m <<= 1)
            for (int t = 0; t < L; t += 2 * m)
                for (int k = 0; k < m; ++k) {
                    W w, wq;
                    load_pair(a.tw, m - 1 + k, w, wq);
                    if (VAR == VAR_LAZY)
                        bfly_inv_lazy(x[t + k], x[t + k + m], w, wq, p, p2);
                    else
                        bfly_inv_ntl(x[t + k], x[t + k + m], w, wq, p);
                }
    }
    for (int i = 0; i < L; ++i) {
        W v = x[i];
        if (VAR == VAR_LAZY) v = DIR == DIR_FWD ? reduce2(v, p) : reduce4(v, p, p2);
        d[i] = v;
    }
}

}  // namespace ntt
