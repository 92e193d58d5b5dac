// modarith.cuh -- word-level modular arithmetic and the butterflies of
// Harvey, "Faster arithmetic for number-theoretic transforms" (arXiv:1205.2926).
//
// Everything here is templated on the machine word W (beta = 2^bits(W)) and
// compiles both for sm_103a and, without CUDA, for the host: the exhaustive
// small-word checks of Theorems 1-4 instantiate it with uint8_t/uint16_t.
//
// Conditional adjustments are written branch-free as an unsigned minimum:
// for 0 <= x < 2c (and 2c <= beta), min(x, x - c) computed mod beta equals
// x - c when x >= c and x otherwise (x - c wraps to >= beta - c > x).  This is
// the GPU counterpart of the conditional moves discussed after Algorithm 2.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define NTT_HD __host__ __device__ __forceinline__
#else
#define NTT_HD inline
#endif

namespace ntt {

template <typename W>
struct Word;

template <>
struct Word<uint8_t> {
    static NTT_HD uint8_t mulhi(uint8_t a, uint8_t b) { return (uint8_t)(((uint32_t)a * b) >> 8); }
    static NTT_HD uint8_t mullo(uint8_t a, uint8_t b) { return (uint8_t)((uint32_t)a * b); }
};

template <>
struct Word<uint16_t> {
    static NTT_HD uint16_t mulhi(uint16_t a, uint16_t b) { return (uint16_t)(((uint32_t)a * b) >> 16); }
    static NTT_HD uint16_t mullo(uint16_t a, uint16_t b) { return (uint16_t)((uint32_t)a * b); }
};

template <>
struct Word<uint32_t> {
    static NTT_HD uint32_t mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
        return __umulhi(a, b);
#else
        return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
    }
    static NTT_HD uint32_t mullo(uint32_t a, uint32_t b) { return a * b; }
};

template <>
struct Word<uint64_t> {
    static NTT_HD uint64_t mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
        return __umul64hi(a, b);
#else
        return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
    }
    static NTT_HD uint64_t mullo(uint64_t a, uint64_t b) { return a * b; }
};

template <typename W>
NTT_HD W umin(W a, W b) {
    return a < b ? a : b;
}

// x - c if x >= c else x, for 0 <= x < 2c, 2c <= beta.
template <typename W>
NTT_HD W csub(W x, W c) {
    return umin(x, (W)(x - c));
}

// Shoup's product (Algorithm 2, multiplication lines; Theorem 1's proof):
// with W' = floor(W beta / p) and ANY 0 <= t < beta, Q = floor(W' t / beta)
// gives 0 <= W t - Q p < 2p, so the low word of W t - Q p is exact.
template <typename W>
NTT_HD W shoup_mul(W t, W w, W wq, W p) {
    W q = Word<W>::mulhi(wq, t);
    return (W)(Word<W>::mullo(w, t) - Word<W>::mullo(q, p));
}

// Algorithm 2 (NTL butterfly, fully reduced): X, Y in [0, p), p < beta/2.
// The subtraction uses the borrow form noted at the end of Section 2
// (T = X - Y wraps when X < Y; adding p back is then the smaller value),
// which gives the same T as the signed test T < 0.
template <typename W>
NTT_HD void bfly_fwd_ntl(W &x, W &y, W w, W wq, W p) {
    W s = csub((W)(x + y), p);
    W t = (W)(x - y);
    t = umin(t, (W)(t + p));
    W r = csub(shoup_mul(t, w, wq, p), p);
    x = s;
    y = r;
}

// x - c if x >= c else x, written as a compare and select (same result as
// csub for 0 <= x < 2c).  The compiler schedules the product-free W = 1
// butterfly better with this form; the general butterflies use csub.
template <typename W>
NTT_HD W csub_sel(W x, W c) {
    return x >= c ? (W)(x - c) : x;
}

// Algorithm 3 (modified Shoup butterfly): X, Y in [0, 2p), p < beta/4;
// X' = X + Y reduced once by 2p, T = X - Y + 2p in [0, 4p) without any test,
// Y' = W T - Q p in [0, 2p) without the final correction.
template <typename W>
NTT_HD void bfly_fwd_lazy(W &x, W &y, W w, W wq, W p, W p2) {
    W s = csub((W)(x + y), p2);
    W t = (W)(x - y + p2);
    y = shoup_mul(t, w, wq, p);
    x = s;
}

// Butterflies with W = 1 (the stage of distance 1, and the k = 0 pairs of
// other stages; Section 5 notes L - 1 of them per transform).  Same outputs
// and ranges as the general butterflies with W = 1, without the product:
// forward lazy: Y' = T reduced once from [0, 4p) to [0, 2p);
// inverse lazy: T = Y reduced once from [0, 4p) to [0, 2p).
template <typename W>
NTT_HD void bfly_fwd_lazy_w1(W &x, W &y, W p2) {
    W s = csub_sel((W)(x + y), p2);
    W t = (W)(x - y + p2);
    y = csub_sel(t, p2);
    x = s;
}

template <typename W>
NTT_HD void bfly_fwd_ntl_w1(W &x, W &y, W p) {
    W s = csub((W)(x + y), p);
    W t = (W)(x - y);
    y = umin(t, (W)(t + p));
    x = s;
}

template <typename W>
NTT_HD void bfly_inv_lazy_w1(W &x, W &y, W p2) {
    W a = csub(x, p2);
    W t = csub(y, p2);
    x = (W)(a + t);
    y = (W)(a - t + p2);
}

template <typename W>
NTT_HD void bfly_inv_ntl_w1(W &x, W &y, W p) {
    W s = csub((W)(x + y), p);
    W d = (W)(x - y);
    y = umin(d, (W)(d + p));
    x = s;
}

// Algorithm 4 (modified inverse butterfly, (X, Y) -> (X + WY, X - WY)):
// X, Y in [0, 4p); X reduced once by 2p; T = W Y mod p in [0, 2p) (Shoup
// accepts any Y < beta); X' = X + T, Y' = X - T + 2p, both in [0, 4p).
template <typename W>
NTT_HD void bfly_inv_lazy(W &x, W &y, W w, W wq, W p, W p2) {
    W a = csub(x, p2);
    W t = shoup_mul(y, w, wq, p);
    x = (W)(a + t);
    y = (W)(a - t + p2);
}

// Fully reduced inverse butterfly used by the NTL-style comparison path:
// X, Y in [0, p) -> (X + WY, X - WY) in [0, p).
template <typename W>
NTT_HD void bfly_inv_ntl(W &x, W &y, W w, W wq, W p) {
    W t = csub(shoup_mul(y, w, wq, p), p);
    W s = csub((W)(x + t), p);
    W d = (W)(x - t);
    d = umin(d, (W)(d + p));
    x = s;
    y = d;
}

// Multiplication part of Algorithm 5 (Montgomery): with W' = beta W mod p in
// [0, p), J = p^-1 mod beta and 0 <= t < beta, returns a representative of
// W t mod p in [0, 2p):  R1 beta + R0 = W' t, Q = R0 J mod beta,
// H = floor(Q p / beta), result R1 - H + p.  With t < 2p and W' replaced by
// any value below 2p it still lands in [0, 2p) when p < beta/4 (R1 < p).
template <typename W>
NTT_HD W mont_mul(W t, W wm, W J, W p) {
    W r0 = Word<W>::mullo(wm, t);
    W r1 = Word<W>::mulhi(wm, t);
    W q = Word<W>::mullo(r0, J);
    W h = Word<W>::mulhi(q, p);
    return (W)(r1 - h + p);
}

// Algorithm 5 (modified Montgomery butterfly): X, Y in [0, 2p).
template <typename W>
NTT_HD void bfly_fwd_mont(W &x, W &y, W wm, W J, W p, W p2) {
    W s = csub((W)(x + y), p2);
    W t = (W)(x - y + p2);
    y = mont_mul(t, wm, J, p);
    x = s;
}

// Inverse counterpart of Algorithm 5 (the paper gives the forward butterfly
// only; this is Algorithm 4 with Montgomery's product in place of Shoup's):
// X, Y in [0, 4p); X reduced once by 2p; T = W Y mod p in [0, 2p) by
// mont_mul (valid for Y < 4p when p < beta/4: R1 < p); X' = X + T,
// Y' = X - T + 2p, both in [0, 4p).
template <typename W>
NTT_HD void bfly_inv_mont(W &x, W &y, W wm, W J, W p, W p2) {
    W a = csub(x, p2);
    W t = mont_mul(y, wm, J, p);
    x = (W)(a + t);
    y = (W)(a - t + p2);
}

// Moeller's refinement of Algorithm 2 (end of Section 2): the fully reduced
// butterfly for any p < beta/phi, phi = (1 + sqrt 5)/2, where X + Y may
// exceed beta.  The subtraction takes its correction from the borrow
// (X < Y); the addition is rewritten X - (p - Y), corrected by the borrow
// X < p - Y.  The candidate remainder W T - Q p of Shoup's product is below
// (1 + p/beta) p < phi p < beta, so its low word is exact and one
// subtraction of p reduces it.  Compare-and-select forms: the unsigned
// minimum of csub would need 2p <= beta here.
template <typename W>
NTT_HD W addmod_borrow(W x, W y, W p) {
    const W t = (W)(p - y);
    const W s = (W)(x - t);
    return x < t ? (W)(s + p) : s;
}

template <typename W>
NTT_HD W submod_borrow(W x, W y, W p) {
    const W s = (W)(x - y);
    return x < y ? (W)(s + p) : s;
}

// x - c if x >= c else x, for 0 <= x < min(2c, beta) (any c < beta).
template <typename W>
NTT_HD W csub_any(W x, W c) {
    return x >= c ? (W)(x - c) : x;
}

template <typename W>
NTT_HD void bfly_fwd_moller(W &x, W &y, W w, W wq, W p) {
    const W s = addmod_borrow(x, y, p);
    const W t = submod_borrow(x, y, p);
    y = csub_any(shoup_mul(t, w, wq, p), p);
    x = s;
}

// Inverse counterpart (X + WY, X - WY), fully reduced, p < beta/phi.
template <typename W>
NTT_HD void bfly_inv_moller(W &x, W &y, W w, W wq, W p) {
    const W t = csub_any(shoup_mul(y, w, wq, p), p);
    const W s = addmod_borrow(x, t, p);
    y = submod_borrow(x, t, p);
    x = s;
}

template <typename W>
NTT_HD void bfly_moller_w1(W &x, W &y, W p) {
    const W s = addmod_borrow(x, y, p);
    y = submod_borrow(x, y, p);
    x = s;
}

// Final normalisation (end of Section 3): [0, 2p) -> [0, p), [0, 4p) -> [0, p).
template <typename W>
NTT_HD W reduce2(W x, W p) {
    return csub(x, p);
}
template <typename W>
NTT_HD W reduce4(W x, W p, W p2) {
    return csub(csub(x, p2), p);
}

}  // namespace ntt
