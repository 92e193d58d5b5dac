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
// Algorithm 1, independent of R.  One table tw[m + k] = (W, W') for k < m,
// m = 1, 2, 4, ... (entry 0 unused) serves every pass; W' = floor(W beta/p)
// is the precomputed Shoup quotient of Algorithms 2-4.  The offset m (rather
// than m - 1) keeps runs of consecutive k 16-byte aligned for vector loads.
//
// On-chip work.  A CTA stages a tile in shared memory as 16-byte vectors of
// V words (V = 4 for 32-bit, 2 for 64-bit words); the V lanes of a vector
// are the same element of V independent sub-transforms, so they share every
// twiddle:
//   column pass: lanes are V adjacent columns (one 16-byte global chunk);
//   row pass: lanes are V consecutive rows.
// Each thread holds E = 8 vectors in registers and runs up to three
// butterfly stages per round (radix-8 blocks); rounds exchange vectors
// through shared memory.  The vector of row s sits at chunk
// TV*(s + (s >> 3)) + tv (one padding chunk per eight), or TV*s + tv in
// column tiles of TV = 8 vectors: in every round the eight threads of a
// quarter-warp hit eight distinct bank groups, and the eight chunks of one
// thread sit at compile-time offsets from one base.  Only the threads that
// share a sub-tile synchronise between rounds (a warp, a named barrier or
// the CTA).
//
// Data movement.  CTAs are persistent: each walks its tiles with stride
// gridDim.x.  The first round of a pass loads its vectors straight from
// global memory into registers (coalesced, through L2 only), except in
// 64-bit column passes, which fetch the next tile into a second buffer
// while computing the current one: by tensor copies (cp.async.bulk.tensor,
// completion on an mbarrier) when tile rows are 128 bytes, else by cp.async.
// The last round of every pass writes straight from registers to HBM:
// 16-byte vectors in a column pass, eight consecutive words of each row in
// the forward row pass, and in the inverse row pass word stores in which
// neighbouring threads write neighbouring words of a row.
//
// Butterflies: Algorithm 3 / Algorithm 4 (lazy, redundant [0,2p) / [0,4p))
// or Algorithm 2 / its fully reduced inverse (the NTL-style baseline).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace ntt {

enum { DIR_FWD = 0, DIR_INV = 1 };
// Butterfly variants: Algorithms 3-4 (lazy, Shoup's product), Algorithm 2 and
// its fully reduced inverse (NTL-style), Algorithm 5 with its inverse
// counterpart (lazy ranges, Montgomery's product; the twiddle pairs then hold
// (W, beta W mod p)), and Moeller's form of Algorithm 2 (fully reduced, any
// p < beta/phi; end of Section 2).
enum { VAR_LAZY = 0, VAR_NTL = 1, VAR_MONT = 2, VAR_MOLLER = 3 };

// Variants whose values stay fully reduced in [0, p) between stages.
template <int VAR>
struct Reduced {
    static constexpr bool ON = VAR == VAR_NTL || VAR == VAR_MOLLER;
};
enum { F_NORMALIZE = 1, F_MIDDLE = 2, F_MB = 4, F_TMA = 8 };

constexpr int kThreads = 256;  // threads per CTA of the pass kernels

template <typename W>
struct Lanes {
    static constexpr int V = 16 / sizeof(W);  // words per 16-byte vector
    static constexpr int LOGV = V == 4 ? 2 : 1;
};

// Arguments of one pass over a batch of transforms.
template <typename W>
struct PassArgs {
    W *data;              // transform 0
    uint64_t stride;      // words between consecutive transforms
    uint32_t batch;
    int32_t logL;
    int32_t logS;         // column stride of a column pass (0 for the row pass)
    int32_t logTV;        // column pass: 16-byte vectors per tile row
    int32_t logTA;        // column pass: width of the middle-twiddle table MA
    int32_t per_cta;      // column pass: tiles per CTA iteration; row pass: rows per iteration
    uint32_t ntiles;      // CTA iterations in this pass
    uint32_t buf_chunks;  // 16-byte chunks of one shared-memory buffer
    uint32_t flags;       // F_NORMALIZE | F_MIDDLE | F_MB
    const W *tw;          // stage twiddle pairs tw[m + k], forward or inverse roots
    const W *ma;          // middle twiddle pairs MA[s][c mod TA]
    const W *mb;          // middle twiddle pairs MB[c / TA][s]
    W p;
    W J;                  // p^-1 mod beta (Montgomery variant)
    uint64_t nrows;       // row pass: number of rows (batch * L / R, or transforms)
    W *const *rowptrs;    // row pass over single-row transforms: address of each row (else null)
    int *status;          // device status word: NTT_ERR_TIMEOUT when a tile copy never lands
    long long wait_budget;  // clock cycles a CTA waits for one tile copy
    uint32_t tx_extra;      // bytes each tile copy expects beyond its own (0; a test sets more)
};

// ------------------------------------------------------------- small helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint4 *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename W>
__device__ __forceinline__ void ld_pair(const W *__restrict__ t, int idx, W &w, W &wq);

template <>
__device__ __forceinline__ void ld_pair<uint32_t>(const uint32_t *__restrict__ t, int idx, uint32_t &w,
                                                  uint32_t &wq) {
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(t) + idx);
    w = v.x;
    wq = v.y;
}

template <>
__device__ __forceinline__ void ld_pair<uint64_t>(const uint64_t *__restrict__ t, int idx, uint64_t &w,
                                                  uint64_t &wq) {
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(t) + idx);
    w = v.x;
    wq = v.y;
}

// V consecutive pairs starting at pair index idx (a multiple of V, so that
// the two 16-byte loads are aligned).
template <typename W>
__device__ __forceinline__ void ld_pairs(const W *__restrict__ t, int idx, W (&w)[Lanes<W>::V],
                                         W (&wq)[Lanes<W>::V]);

template <>
__device__ __forceinline__ void ld_pairs<uint32_t>(const uint32_t *__restrict__ t, int idx, uint32_t (&w)[4],
                                                   uint32_t (&wq)[4]) {
    const uint4 *q = reinterpret_cast<const uint4 *>(t + 2 * idx);
    const uint4 a = __ldg(q), b = __ldg(q + 1);
    w[0] = a.x, wq[0] = a.y, w[1] = a.z, wq[1] = a.w;
    w[2] = b.x, wq[2] = b.y, w[3] = b.z, wq[3] = b.w;
}

template <>
__device__ __forceinline__ void ld_pairs<uint64_t>(const uint64_t *__restrict__ t, int idx, uint64_t (&w)[2],
                                                   uint64_t (&wq)[2]) {
    const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(t) + idx;
    const ulonglong2 a = __ldg(q), b = __ldg(q + 1);
    w[0] = a.x, wq[0] = a.y, w[1] = b.x, wq[1] = b.y;
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

template <typename W, int DIR, int VAR>
__device__ __forceinline__ void bfly(W &x, W &y, W w, W wq, W p, W p2, W J) {
    if (DIR == DIR_FWD) {
        if (VAR == VAR_LAZY)
            bfly_fwd_lazy(x, y, w, wq, p, p2);
        else if (VAR == VAR_MONT)
            bfly_fwd_mont(x, y, wq, J, p, p2);
        else if (VAR == VAR_MOLLER)
            bfly_fwd_moller(x, y, w, wq, p);
        else
            bfly_fwd_ntl(x, y, w, wq, p);
    } else {
        if (VAR == VAR_LAZY)
            bfly_inv_lazy(x, y, w, wq, p, p2);
        else if (VAR == VAR_MONT)
            bfly_inv_mont(x, y, wq, J, p, p2);
        else if (VAR == VAR_MOLLER)
            bfly_inv_moller(x, y, w, wq, p);
        else
            bfly_inv_ntl(x, y, w, wq, p);
    }
}

// Butterfly with W = 1 (no product; see modarith.cuh).
template <typename W, int DIR, int VAR>
__device__ __forceinline__ void bfly_w1(W &x, W &y, W p, W p2) {
    if (VAR == VAR_MOLLER) {
        bfly_moller_w1(x, y, p);
    } else if (DIR == DIR_FWD) {
        if (VAR != VAR_NTL)
            bfly_fwd_lazy_w1(x, y, p2);
        else
            bfly_fwd_ntl_w1(x, y, p);
    } else {
        if (VAR != VAR_NTL)
            bfly_inv_lazy_w1(x, y, p2);
        else
            bfly_inv_ntl_w1(x, y, p);
    }
}

template <typename W, int VAR>
__device__ __forceinline__ W mul_twiddle(W x, W w, W wq, W p, W J) {
    if (VAR == VAR_MONT) return mont_mul(x, wq, J, p);  // x < 4p -> [0, 2p)
    W y = shoup_mul(x, w, wq, p);                       // any x < beta -> [0, 2p); x < p -> [0, phi p)
    return Reduced<VAR>::ON ? csub(y, p) : y;
}

// ------------------------------------------------------- compile-time rounds
//
// LOGS vector-index bits are handled by rounds of up to LE = 3 stages.  In
// round r the thread's E vectors are s_j = hi | (j << b0) | lo, with (hi, lo)
// taken from the unit's group index g; the round executes `nst` of its local
// stage bits (the top ones when the partial round has fewer than LE).
template <int LOGS>
struct Sched {
    static constexpr int LE = LOGS < 3 ? LOGS : 3;
    static constexpr int E = 1 << LE;
    static constexpr int NR = (LOGS + LE - 1) / LE;
    static constexpr int E0 = LOGS - LE * (NR - 1);
    __host__ __device__ static constexpr int b0(int dir, int r) {
        return dir == DIR_FWD ? (r == 0 ? LOGS - LE : LOGS - E0 - LE * r) : (r == NR - 1 ? LOGS - LE : LE * r);
    }
    __host__ __device__ static constexpr int nst(int dir, int r) {
        return dir == DIR_FWD ? (r == 0 ? E0 : LE) : (r == NR - 1 ? E0 : LE);
    }
};

// Butterfly stages of one round on E vectors held in registers; the V lanes
// of a vector share every twiddle.  twp points at tw + (low index bits of
// the unit).  In the round with b0 = 0 the pairs with jl = 0 have k = 0 for
// every unit, hence W = 1: they skip the product.
// SKIP1 leaves out the stage of distance 1 (lb = 0 in the round with
// b0 = 0), which the caller fuses with the middle twiddle.
template <typename W, int DIR, int VAR, int LE, int B0, int NST, bool SKIP1 = false>
__device__ __forceinline__ void round_regs(W (&x)[1 << LE][Lanes<W>::V], const W *__restrict__ twp, W p, W p2,
                                           W J) {
    constexpr int V = Lanes<W>::V;
    constexpr int E = 1 << LE;
#pragma unroll
    for (int step = 0; step < NST; ++step) {
        const int lb = DIR == DIR_FWD ? LE - 1 - step : LE - NST + step;
        if (SKIP1 && B0 == 0 && lb == 0) continue;
#pragma unroll
        for (int jl = 0; jl < (1 << lb); ++jl) {
            const int off = (1 << (B0 + lb)) + (jl << B0);
            if (B0 == 0 && jl == 0) {
#pragma unroll
                for (int jh = 0; jh < E; jh += (2 << lb)) {
#pragma unroll
                    for (int v = 0; v < V; ++v) bfly_w1<W, DIR, VAR>(x[jh][v], x[jh + (1 << lb)][v], p, p2);
                }
            } else {
                W w, wq;
                ld_pair(twp, off, w, wq);
#pragma unroll
                for (int jh = 0; jh < E; jh += (2 << lb)) {
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        bfly<W, DIR, VAR>(x[jh + jl][v], x[jh + jl + (1 << lb)][v], w, wq, p, p2, J);
                }
            }
        }
    }
}

template <typename W, int DIR, int VAR, int E>
__device__ __forceinline__ void normalize(W (&x)[E][Lanes<W>::V], W p, W p2) {
    if constexpr (!Reduced<VAR>::ON) {
#pragma unroll
        for (int j = 0; j < E; ++j)
#pragma unroll
            for (int v = 0; v < Lanes<W>::V; ++v)
                x[j][v] = DIR == DIR_FWD ? reduce2(x[j][v], p) : reduce4(x[j][v], p, p2);
    }
}

// Middle twiddle of a column pass, omega^((L/B) c rev(s)), on the E vectors
// of rows s = s0 + j (the round with b0 = 0), columns c = c0 + v.  Factored
// as MB[c >> logTA][s] * MA[s][c mod TA]: two Shoup products from two small
// tables (about 2 R sqrt(S) entries in all) instead of one table of B.
template <typename W, int VAR, int E>
__device__ __forceinline__ void middle_twiddle(W (&x)[E][Lanes<W>::V], uint32_t s0, uint32_t c0, uint32_t R,
                                               const PassArgs<W> &a) {
    constexpr int V = Lanes<W>::V;
    const uint32_t TAm = (1u << a.logTA) - 1u;
    const W *mbp = a.mb + 2 * ((uint64_t)(c0 >> a.logTA) * R + s0);
    const W *map = a.ma + 2 * (((uint64_t)s0 << a.logTA) + (c0 & TAm));
#pragma unroll
    for (int j = 0; j < E; ++j) {
        if (a.flags & F_MB) {
            W w, wq;
            ld_pair(mbp, j, w, wq);
#pragma unroll
            for (int v = 0; v < V; ++v) x[j][v] = mul_twiddle<W, VAR>(x[j][v], w, wq, a.p, a.J);
        }
        W w[V], wq[V];
        ld_pairs<W>(map, j << a.logTA, w, wq);
#pragma unroll
        for (int v = 0; v < V; ++v) x[j][v] = mul_twiddle<W, VAR>(x[j][v], w[v], wq[v], a.p, a.J);
    }
}

// Distance-1 stage (W = 1) fused with the middle twiddle of a forward column
// pass: X' = M_s (X + Y), Y' = M_{s+1} (X - Y + 2p).  Shoup's product accepts
// any input below beta and Montgomery's any below 4p, so the two reductions
// of the W = 1 butterfly go away (lazy variants; the NTL variant keeps its
// reductions).
template <typename W, int VAR, int E>
__device__ __forceinline__ void last_stage_and_twiddle(W (&x)[E][Lanes<W>::V], uint32_t s0, uint32_t c0, uint32_t R,
                                                       const PassArgs<W> &a) {
    constexpr int V = Lanes<W>::V;
    const W p2 = (W)(2 * a.p);
#pragma unroll
    for (int j = 0; j < E; j += 2) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (!Reduced<VAR>::ON) {
                const W s = (W)(x[j][v] + x[j + 1][v]);
                const W t = (W)(x[j][v] - x[j + 1][v] + p2);
                x[j][v] = s;
                x[j + 1][v] = t;
            } else {
                bfly_w1<W, DIR_FWD, VAR>(x[j][v], x[j + 1][v], a.p, p2);
            }
        }
    }
    middle_twiddle<W, VAR, E>(x, s0, c0, R, a);
}

// Inverse counterpart: the middle twiddle leaves every value in [0, 2p)
// (lazy), so the following W = 1 butterfly needs no reduction:
// X' = X + Y, Y' = X - Y + 2p.
template <typename W, int VAR, int E>
__device__ __forceinline__ void twiddle_and_first_stage(W (&x)[E][Lanes<W>::V], uint32_t s0, uint32_t c0, uint32_t R,
                                                        const PassArgs<W> &a) {
    constexpr int V = Lanes<W>::V;
    const W p2 = (W)(2 * a.p);
    middle_twiddle<W, VAR, E>(x, s0, c0, R, a);
#pragma unroll
    for (int j = 0; j < E; j += 2) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (!Reduced<VAR>::ON) {
                const W s = (W)(x[j][v] + x[j + 1][v]);
                const W t = (W)(x[j][v] - x[j + 1][v] + p2);
                x[j][v] = s;
                x[j + 1][v] = t;
            } else {
                bfly_w1<W, DIR_INV, VAR>(x[j][v], x[j + 1][v], a.p, p2);
            }
        }
    }
}

// ------------------------------------------------------------ tile geometry

// Column pass: CTA iteration `tile` covers sub-tiles tile*per_cta + ti, each
// R rows x TV vectors of one block; 2^ltb sub-tiles per block, 2^lbt blocks
// per transform.  Row pass: iteration `tile` covers vector groups
// tile*per_cta + ti; group ti holds V consecutive rows, one per lane.
template <typename W, int LOGR, bool ROW, int TVC = -1>
struct Geo {
    static constexpr int LOGS = LOGR;                                // element-index bits
    static constexpr uint32_t NS = 1u << LOGS;                       // vectors per sub-transform
    // Column tiles of 8 vectors per row (128 bytes) need no padding: the
    // eight threads of a quarter-warp read one whole row.  Every other
    // layout pads one chunk per eight rows.
    static constexpr bool PAD = ROW || TVC != 3;
    static constexpr uint32_t NSP = PAD ? NS + (NS >> 3) : NS;       // rows of one sub-tile, with padding
    __host__ __device__ static constexpr uint32_t pidx(uint32_t s) { return PAD ? s + (s >> 3) : s; }
    using S = Sched<LOGS>;

    int logTV_, ltb, lbt;
    uint32_t sub_total;  // column pass: sub-tiles in the pass

    // log2 of the tile width in vectors: a compile-time constant for row
    // passes and for the common column-pass width, else the runtime value
    __device__ __forceinline__ int logTV() const { return ROW ? 0 : (TVC >= 0 ? TVC : logTV_); }

    __device__ __forceinline__ explicit Geo(const PassArgs<W> &a) {
        logTV_ = ROW ? 0 : a.logTV;
        ltb = ROW ? 0 : a.logS - a.logTV - Lanes<W>::LOGV;
        lbt = ROW ? 0 : a.logL - LOGR - a.logS;
        sub_total = ROW ? 0 : (a.batch << (ltb + lbt));
    }
    // column pass: origin of sub-tile t, and its column-tile index ct
    __device__ __forceinline__ W *col_origin(const PassArgs<W> &a, uint32_t t, uint32_t &ct) const {
        ct = t & ((1u << ltb) - 1u);
        const uint32_t blk = (t >> ltb) & ((1u << lbt) - 1u), b = t >> (ltb + lbt);
        return a.data + (uint64_t)b * a.stride + ((uint64_t)blk << (LOGR + a.logS)) +
               ((uint64_t)ct << (logTV() + Lanes<W>::LOGV));
    }
    __device__ __forceinline__ W *row_ptr(const PassArgs<W> &a, uint64_t row) const {
        if (a.rowptrs) return a.rowptrs[row];
        const int shift = a.logL - LOGR;
        const uint64_t b = row >> shift, within = row & ((1ull << shift) - 1ull);
        return a.data + b * a.stride + (within << LOGR);
    }
};

// Which passes prefetch their next tile into a second shared buffer (by
// tensor copies when tile rows are 128 bytes and the host enabled them, else
// by cp.async) and which let their first round load straight from global
// memory into registers: the direct load is faster for every 32-bit pass and
// for 64-bit row passes (measured); 64-bit column passes keep the prefetch.
template <typename W, bool ROW>
struct Prefetch {
    static constexpr bool ON = !ROW && sizeof(W) == 8;
};

// Global -> shared copy of one CTA iteration of a prefetching column pass,
// issued as cp.async copies (completed through commit/wait groups):
// consecutive threads take consecutive 16-byte chunks of a tile row
// (coalesced), addresses advance by constant strides from a per-thread base.
// Other passes have nothing to copy ahead: their first round loads straight
// from global memory (tile_round).
template <typename W, int LOGR, bool ROW, int TVC>
__device__ __forceinline__ void tile_copy(const PassArgs<W> &a, const Geo<W, LOGR, ROW, TVC> &geo, uint32_t tile,
                                          uint4 *buf) {
    using G = Geo<W, LOGR, ROW, TVC>;
    constexpr int V = Lanes<W>::V;
    if (!Prefetch<W, ROW>::ON) {
        // nothing to copy ahead: the first round reads global memory
    } else {
        const int logTV = geo.logTV();
        const uint32_t cc = threadIdx.x & ((1u << logTV) - 1u);
        const uint32_t rows_step = (uint32_t)kThreads >> logTV;  // >= 32, a multiple of 8
        const uint64_t S = 1ull << a.logS;
        for (uint32_t srow = threadIdx.x >> logTV; srow < ((uint32_t)a.per_cta << LOGR);) {
            const uint32_t ti = srow >> LOGR;
            const uint32_t t = tile * a.per_cta + ti;
            if (t >= geo.sub_total) break;
            uint32_t ct;
            uint32_t s = srow & ((1u << LOGR) - 1u);
            const W *g = geo.col_origin(a, t, ct) + s * S + cc * V;
            uint4 *sp = buf + ((ti * G::NSP + G::pidx(s)) << logTV) + cc;
            const uint64_t gstep = rows_step * S;
            const uint32_t sstep = G::pidx(rows_step) << logTV;
            for (; s < (1u << LOGR); s += rows_step, srow += rows_step) {
                cp_async16(sp, g);
                g += gstep;
                sp += sstep;
            }
        }
    }
}

// Butterflies of one unit (E vectors in registers) in round RI, then the
// write-back: to shared memory, or, in the last round of a direct-store
// pass, straight to global memory.
template <typename W, int DIR, int VAR, int LOGR, bool ROW, int TVC, int RI>
__device__ __forceinline__ void unit_round(const PassArgs<W> &a, const Geo<W, LOGR, ROW, TVC> &geo, uint32_t tile,
                                           uint4 *rp, uint32_t ti, uint32_t tv, uint32_t s0, uint32_t lo,
                                           W (&x)[Geo<W, LOGR, ROW, TVC>::S::E][Lanes<W>::V]) {
    using G = Geo<W, LOGR, ROW, TVC>;
    using S = typename G::S;
    constexpr int V = Lanes<W>::V;
    constexpr int LE = S::LE, E = S::E;
    constexpr int B0 = S::b0(DIR, RI), NST = S::nst(DIR, RI);
    constexpr bool FIRST = RI == 0, LAST = RI == S::NR - 1;
    const W p = a.p, p2 = (W)(2 * a.p);
    const int logTV = geo.logTV();
    const bool mid = !ROW && (a.flags & F_MIDDLE) && ((DIR == DIR_INV && FIRST) || (DIR == DIR_FWD && LAST));
    uint32_t c0 = 0;
    if (mid) {
        uint32_t ct;
        geo.col_origin(a, tile * a.per_cta + ti, ct);
        c0 = ((ct << logTV) + tv) * V;
    }
    // rounds holding the distance-1 stage (b0 = 0) of a column pass fuse
    // it with the middle twiddle; every other round runs as is
    constexpr bool FUSE = !ROW && B0 == 0 && LE == 3 && ((DIR == DIR_INV && FIRST) || (DIR == DIR_FWD && LAST));
    if (FUSE && mid) {
        if (DIR == DIR_INV) twiddle_and_first_stage<W, VAR, E>(x, s0, c0, 1u << LOGR, a);
        round_regs<W, DIR, VAR, LE, B0, NST, true>(x, a.tw + 2 * lo, p, p2, a.J);
        if (DIR == DIR_FWD) last_stage_and_twiddle<W, VAR, E>(x, s0, c0, 1u << LOGR, a);
    } else {
        if (DIR == DIR_INV && FIRST && mid) middle_twiddle<W, VAR, E>(x, s0, c0, 1u << LOGR, a);
        round_regs<W, DIR, VAR, LE, B0, NST>(x, a.tw + 2 * lo, p, p2, a.J);
        if (DIR == DIR_FWD && LAST && mid) middle_twiddle<W, VAR, E>(x, s0, c0, 1u << LOGR, a);
    }
    if (LAST && (a.flags & F_NORMALIZE)) normalize<W, DIR, VAR, E>(x, p, p2);
    if (LAST) {
        // the last round writes straight to global memory
        if (ROW) {
            const uint64_t row0 = ((uint64_t)tile * a.per_cta + ti) * V;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (row0 + v < a.nrows) {
                    W *gp = geo.row_ptr(a, row0 + v) + s0;
                    if (B0 == 0) {
                        // elements s0 .. s0+7 of the lane's row: 8 consecutive words
#pragma unroll
                        for (int q = 0; q < E; q += V) {
                            uint4 c;
                            W *pc = reinterpret_cast<W *>(&c);
#pragma unroll
                            for (int k = 0; k < V; ++k) pc[k] = x[q + k][v];
                            *reinterpret_cast<uint4 *>(gp + q) = c;
                        }
                    } else {
                        // element s0 + (j << b0): neighbouring threads hold
                        // neighbouring elements, so each word store of a warp
                        // covers consecutive words of the row
#pragma unroll
                        for (int j = 0; j < E; ++j) gp[j << B0] = x[j][v];
                    }
                }
            }
        } else {
            const uint32_t t = tile * a.per_cta + ti;
            if (t < geo.sub_total) {
                uint32_t ct;
                const uint64_t S = 1ull << a.logS;
                W *gp = geo.col_origin(a, t, ct) + s0 * S + tv * V;
#pragma unroll
                for (int j = 0; j < E; ++j)
                    *reinterpret_cast<uint4 *>(gp + (uint64_t)(j << B0) * S) = pack<W>(x[j]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const uint32_t cj = G::pidx((uint32_t)j << B0);
            rp[cj << logTV] = pack<W>(x[j]);
        }
    }
}

// One round over the tile in shared memory (compile-time round index RI).
// A unit is E vectors of one sub-transform: s_j = hi | (j << b0) | lo.
template <typename W, int DIR, int VAR, int LOGR, bool ROW, int TVC, int RI>
__device__ __forceinline__ void tile_round(const PassArgs<W> &a, const Geo<W, LOGR, ROW, TVC> &geo, uint32_t tile,
                                           uint4 *buf) {
    using G = Geo<W, LOGR, ROW, TVC>;
    using S = typename G::S;
    constexpr int V = Lanes<W>::V;
    constexpr int LE = S::LE, E = S::E;
    constexpr int B0 = S::b0(DIR, RI);
    const int logTV = geo.logTV();
    const uint32_t units = (uint32_t)a.per_cta << (G::LOGS - LE + logTV);
    if constexpr (ROW && RI == 0) {
        // First round of a row pass: element s_j of each of the unit's V rows
        // comes straight from global memory into lane j of the registers.
        // Neighbouring threads take neighbouring elements (16-byte chunks when
        // b0 = 0), so every warp load is coalesced; loads go through L2 only.
        for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
            const uint32_t g = u & ((G::NS >> LE) - 1u);
            const uint32_t ti = u >> (G::LOGS - LE);
            const uint32_t lo = g & ((1u << B0) - 1u);
            const uint32_t s0 = ((g >> B0) << (B0 + LE)) | lo;
            uint4 *rp = buf + ti * G::NSP + G::pidx(s0);
            const uint64_t row0 = ((uint64_t)tile * a.per_cta + ti) * V;
            W x[E][V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (row0 + v < a.nrows) {
                    const W *gp = geo.row_ptr(a, row0 + v) + s0;
                    if (B0 == 0) {
#pragma unroll
                        for (int q = 0; q < E / V; ++q) {
                            W c[V];
                            unpack(__ldcg(reinterpret_cast<const uint4 *>(gp) + q), c);
#pragma unroll
                            for (int k = 0; k < V; ++k) x[q * V + k][v] = c[k];
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < E; ++j) x[j][v] = __ldcg(gp + (j << B0));
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < E; ++j) x[j][v] = 0;
                }
            }
            unit_round<W, DIR, VAR, LOGR, ROW, TVC, RI>(a, geo, tile, rp, ti, 0, s0, lo, x);
        }
        return;
    }
    if constexpr (!ROW && RI == 0 && !Prefetch<W, ROW>::ON) {
        // First round of a column pass without prefetch: the unit's E vectors
        // (rows s_j of its V adjacent columns, one 16-byte chunk each) come
        // straight from global memory; the TV threads of a tile row read one
        // contiguous 16*TV-byte run.  Loads go through L2 only.
        for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
            const uint32_t tv = u & ((1u << logTV) - 1u);
            const uint32_t g = (u >> logTV) & ((G::NS >> LE) - 1u);
            const uint32_t ti = u >> (logTV + G::LOGS - LE);
            const uint32_t lo = g & ((1u << B0) - 1u);
            const uint32_t s0 = ((g >> B0) << (B0 + LE)) | lo;
            uint4 *rp = buf + ((ti * G::NSP + G::pidx(s0)) << logTV) + tv;
            const uint32_t t = tile * a.per_cta + ti;
            W x[E][V];
            if (t < geo.sub_total) {
                uint32_t ct;
                const uint64_t S = 1ull << a.logS;
                const W *gp = geo.col_origin(a, t, ct) + s0 * S + tv * V;
#pragma unroll
                for (int j = 0; j < E; ++j)
                    unpack(__ldcg(reinterpret_cast<const uint4 *>(gp + (uint64_t)(j << B0) * S)), x[j]);
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j)
#pragma unroll
                    for (int v = 0; v < V; ++v) x[j][v] = 0;
            }
            unit_round<W, DIR, VAR, LOGR, ROW, TVC, RI>(a, geo, tile, rp, ti, tv, s0, lo, x);
        }
        return;
    }
    for (uint32_t u = threadIdx.x; u < units; u += kThreads) {
        const uint32_t tv = u & ((1u << logTV) - 1u);
        const uint32_t g = (u >> logTV) & ((G::NS >> LE) - 1u);
        const uint32_t ti = u >> (logTV + G::LOGS - LE);
        const uint32_t lo = g & ((1u << B0) - 1u);
        const uint32_t s0 = ((g >> B0) << (B0 + LE)) | lo;
        uint4 *rp = buf + ((ti * G::NSP + G::pidx(s0)) << logTV) + tv;
        W x[E][V];
#pragma unroll
        for (int j = 0; j < E; ++j) {
            const uint32_t cj = G::pidx((uint32_t)j << B0);
            unpack(rp[cj << logTV], x[j]);
        }
        unit_round<W, DIR, VAR, LOGR, ROW, TVC, RI>(a, geo, tile, rp, ti, tv, s0, lo, x);
    }
}

// Barrier among the threads that share one sub-tile's shared memory: the
// threads of sub-tile ti are the contiguous block [ti T, (ti + 1) T), T =
// R TV / 8 (one unit each).  Whole CTA when T >= 256, the warp when T <= 32,
// else a named barrier (ids 1 .. 8) over the T threads.
template <typename W, int LOGR, bool ROW, int TVC>
__device__ __forceinline__ void group_sync(const Geo<W, LOGR, ROW, TVC> &geo) {
    const int logT = LOGR - 3 + geo.logTV();
    if (logT >= 8) {
        __syncthreads();
    } else if (logT <= 5) {
        __syncwarp();
    } else {
        const uint32_t id = 1u + (threadIdx.x >> logT), n = 1u << logT;
        asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
    }
}

template <typename W, int DIR, int VAR, int LOGR, bool ROW, int TVC, int RI = 0>
__device__ __forceinline__ void tile_rounds(const PassArgs<W> &a, const Geo<W, LOGR, ROW, TVC> &geo, uint32_t tile,
                                            uint4 *buf) {
    tile_round<W, DIR, VAR, LOGR, ROW, TVC, RI>(a, geo, tile, buf);
    if constexpr (RI + 1 < Geo<W, LOGR, ROW, TVC>::S::NR) {
        group_sync(geo);
        tile_rounds<W, DIR, VAR, LOGR, ROW, TVC, RI + 1>(a, geo, tile, buf);
    }
}

// Widest column tile for a sub-transform length: R * TV <= 2^LOGMAX vectors
// per shared buffer, at most 8 vectors (128 bytes) per row.  Column passes of
// R >= 2^10 that load their first round straight from global memory (one
// buffer) take tiles of up to 4096 vectors (64 KiB), so that each tile row is
// at least 64 bytes wide (measured: 20-30 % faster than 32- or 16-byte rows);
// shorter ones stay at 2048 vectors, which keeps 4 CTAs per SM.  Prefetching
// passes hold two buffers of up to 2048 vectors, and so does the uneven-batch
// kernel.
template <int LOGR, int LOGMAX = 11>
struct ColWidth {
    static constexpr int LOGTV = (LOGMAX - LOGR) < 3 ? (LOGMAX - LOGR) : 3;
};

template <typename W, int LOGR>
struct ColTileLog {
    static constexpr int MAX = (!Prefetch<W, false>::ON && LOGR >= 10) ? 12 : 11;
};

// The two halves of one CTA iteration, for the persistent uneven-batch kernel
// (which pipelines them across its work items itself): issue the tile's
// global -> shared copies, and run the tile's rounds once they have landed.
// Column tiles have the widest default width only (the uneven-batch planner
// guarantees it), so that one tile body is instantiated per (R, direction).
template <typename W, int LOGR, bool ROW>
__device__ __forceinline__ void tile_load(const PassArgs<W> &a, uint32_t tile, uint4 *buf) {
    constexpr int TVC = ROW ? 0 : ColWidth<LOGR>::LOGTV;
    const Geo<W, LOGR, ROW, TVC> geo(a);
    tile_copy<W, LOGR, ROW>(a, geo, tile, buf);
}

template <typename W, int DIR, int VAR, int LOGR, bool ROW>
__device__ __forceinline__ void tile_compute(const PassArgs<W> &a, uint32_t tile, uint4 *buf) {
    constexpr int TVC = ROW ? 0 : ColWidth<LOGR>::LOGTV;
    const Geo<W, LOGR, ROW, TVC> geo(a);
    tile_rounds<W, DIR, VAR, LOGR, ROW, TVC>(a, geo, tile, buf);
}

// ---------------------------------------------------------------- TMA tiles
//
// Column passes whose tile rows are 128 bytes (8 vectors) can fetch a whole
// sub-tile with tensor copies (cp.async.bulk.tensor) described by a 3-D map
// {column S, row L/S, transform}: one copy of up to 256 rows x 128 bytes.
// One thread issues them; completion is counted in bytes on an mbarrier per
// buffer, so the next tile streams in while the CTA computes the current one.
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier, for at most `budget` clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget) {
    if (mbar_try(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

template <typename W, int LOGR, bool ROW, int TVC>
__device__ __forceinline__ void tma_tile(const PassArgs<W> &a, const Geo<W, LOGR, ROW, TVC> &geo,
                                         const CUtensorMap *map, uint32_t tile, uint4 *buf, uint64_t *bar) {
    using G = Geo<W, LOGR, ROW, TVC>;
    constexpr uint32_t R = 1u << LOGR;
    constexpr uint32_t BOX = R < 256 ? R : 256;
    const int logTV = geo.logTV();
    uint32_t n = 0;
    for (uint32_t ti = 0; ti < (uint32_t)a.per_cta && tile * a.per_cta + ti < geo.sub_total; ++ti) ++n;
    mbar_expect(bar, n * (R << logTV) * 16u + a.tx_extra);
    for (uint32_t ti = 0; ti < n; ++ti) {
        const uint32_t t = tile * a.per_cta + ti;
        const uint32_t ct = t & ((1u << geo.ltb) - 1u);
        const uint32_t blk = (t >> geo.ltb) & ((1u << geo.lbt) - 1u), b = t >> (geo.ltb + geo.lbt);
        const int x = (int)(ct << (logTV + Lanes<W>::LOGV));
#pragma unroll
        for (uint32_t r0 = 0; r0 < R; r0 += BOX) {
            const int y = (int)((blk << LOGR) + r0);
            uint4 *dst = buf + ((ti * G::NSP + r0) << logTV);
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];\n" ::"r"(smem_addr(dst)),
                "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"((int)b), "r"(smem_addr(bar))
                : "memory");
        }
    }
}

// One pass whose column tiles arrive by tensor copies, double buffered.  A
// copy that has not landed within a.wait_budget cycles (about a second by
// default) sets NTT_ERR_TIMEOUT in the status word; the CTA then waits (also
// bounded) for its other copy in flight and stops.
template <typename W, int DIR, int VAR, int LOGR, bool ROW, int TVC>
__device__ __forceinline__ void pass_loop_tma(const PassArgs<W> &a, const CUtensorMap *map, uint4 *sm) {
    const Geo<W, LOGR, ROW, TVC> geo(a);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 2 * a.buf_chunks);  // after the two buffers
    const long long kBudget = a.wait_budget;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0]);
        mbar_init(&bars[1]);
        fence_proxy_async();
    }
    __syncthreads();
    uint32_t tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < a.ntiles) tma_tile<W, LOGR, ROW, TVC>(a, geo, map, tile, sm, &bars[0]);
    for (uint32_t it = 0; tile < a.ntiles; tile += gridDim.x, ++it) {
        uint4 *cur = (it & 1) ? sm + a.buf_chunks : sm;
        uint4 *nxt = (it & 1) ? sm : sm + a.buf_chunks;
        const uint32_t next = tile + gridDim.x;
        const bool more = next < a.ntiles;
        if (threadIdx.x == 0 && more) tma_tile<W, LOGR, ROW, TVC>(a, geo, map, next, nxt, &bars[(it + 1) & 1]);
        const bool ok = mbar_wait(&bars[it & 1], (it >> 1) & 1, kBudget);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicExch(a.status, NTT_ERR_TIMEOUT);
                if (more) mbar_wait(&bars[(it + 1) & 1], ((it + 1) >> 1) & 1, kBudget);
            }
            return;
        }
        tile_rounds<W, DIR, VAR, LOGR, ROW, TVC>(a, geo, tile, cur);
        fence_proxy_async();  // this tile's shared-memory writes before a later copy overwrites them
        __syncthreads();
    }
}

// One pass over a batch: persistent CTAs; prefetching passes double-buffer
// their tiles with cp.async, the others use one buffer and load directly.
template <typename W, int DIR, int VAR, int LOGR, bool ROW, int TVC>
__device__ __forceinline__ void pass_loop(const PassArgs<W> &a, uint4 *sm) {
    const Geo<W, LOGR, ROW, TVC> geo(a);
    uint32_t tile = blockIdx.x;
    if (tile < a.ntiles) tile_copy<W, LOGR, ROW>(a, geo, tile, sm);
    cp_async_commit();
    for (uint32_t it = 0; tile < a.ntiles; tile += gridDim.x, ++it) {
        // passes without prefetch use one buffer
        constexpr bool PF = Prefetch<W, ROW>::ON;
        uint4 *cur = (PF && (it & 1)) ? sm + a.buf_chunks : sm;
        uint4 *nxt = (PF && (it & 1)) ? sm : sm + a.buf_chunks;
        const uint32_t next = tile + gridDim.x;
        if (PF) {
            if (next < a.ntiles) tile_copy<W, LOGR, ROW>(a, geo, next, nxt);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
        }
        tile_rounds<W, DIR, VAR, LOGR, ROW, TVC>(a, geo, tile, cur);
        if (PF)
            __syncthreads();
        else
            group_sync(geo);  // this tile's last reads before the next tile's first writes
    }
    cp_async_wait<0>();
}

// Resident CTAs per SM the register budget is cut for: 4 (64 registers) for
// 32-bit passes up to R = 2^9, 3 (80 registers) for the longer 32-bit passes,
// 2 for 64-bit words -- the faster choice per pass length (measured).
template <typename W, int LOGR>
struct Occupancy {
    static constexpr int CTAS = sizeof(W) == 4 ? (LOGR <= 9 ? 4 : 3) : 2;
};

template <typename W, int DIR, int VAR, int LOGR, bool ROW>
__global__ void __launch_bounds__(kThreads, (Occupancy<W, LOGR>::CTAS))
    k_pass(const PassArgs<W> a, const __grid_constant__ CUtensorMap map) {
    extern __shared__ uint4 sm[];
    constexpr int TVF = ColWidth<LOGR, ColTileLog<W, LOGR>::MAX>::LOGTV;
    if constexpr (!ROW && TVF == 3 && sizeof(W) == 8) {  // tensor copies: 64-bit column passes
        if (a.flags & F_TMA) {
            pass_loop_tma<W, DIR, VAR, LOGR, ROW, 3>(a, &map, sm);
            return;
        }
    }
    if (ROW || a.logTV == TVF)
        pass_loop<W, DIR, VAR, LOGR, ROW, ROW ? 0 : TVF>(a, sm);
    else
        pass_loop<W, DIR, VAR, LOGR, ROW, -1>(a, sm);
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
                    ld_pair(a.tw, m + k, w, wq);
                    bfly<W, DIR, VAR>(x[t + k], x[t + k + m], w, wq, p, p2, a.J);
                }
    } else {
        for (int m = 1; m < L; m <<= 1)
            for (int t = 0; t < L; t += 2 * m)
                for (int k = 0; k < m; ++k) {
                    W w, wq;
                    ld_pair(a.tw, m + k, w, wq);
                    bfly<W, DIR, VAR>(x[t + k], x[t + k + m], w, wq, p, p2, a.J);
                }
    }
    for (int i = 0; i < L; ++i) {
        W v = x[i];
        if (!Reduced<VAR>::ON) v = DIR == DIR_FWD ? reduce2(v, p) : reduce4(v, p, p2);
        d[i] = v;
    }
}

}  // namespace ntt
