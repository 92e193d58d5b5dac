/*
 * ntt_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * number-theoretic transform over F_p (Harvey, "Faster arithmetic for
 * number-theoretic transforms", arXiv:1205.2926).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library: every routine here is written from the mathematics.
 *
 * Arithmetic: every value is a fully reduced residue in [0, p) held in a
 * uint64_t; every product goes through unsigned __int128 and is reduced with
 * the C `%` operator.  There is no lazy reduction, no Shoup quotient and no
 * Montgomery form anywhere in this file -- the oracle is independent of the
 * method it checks.
 *
 * Functions (each cites the passage it follows):
 *   or_dft_naive     -- Section 1 definition b_j = sum_i w^{ij} a_i, placed in
 *                       bit-reversed order as Algorithm 1's output is.
 *   or_dft_at        -- one output position of the definition, O(L).
 *   or_idft_naive    -- the definition of the inverse map used by running
 *                       Algorithm 1 backwards (Section 4): unnormalised.
 *   or_ntt_ref       -- Algorithm 1 (Section 1) with fully reduced arithmetic.
 *   or_intt_ref      -- Algorithm 1 run backwards (Section 4), inverse roots.
 *   or_polymul_*     -- the application named in Section 1 (polynomial
 *                       multiplication): schoolbook definition and the
 *                       convolution theorem through or_ntt_ref.
 *   or_is_prime etc. -- number theory needed to name the workloads' primes and
 *                       roots (Section 1: p word-sized, p = 1 mod L).
 *
 * Planted-mistake builds: compiling with -DORACLE_MUTANT=k (k >= 1) plants one
 * deliberate error (see the MUTANT() sites below).  The test suite builds each
 * mutant and checks that at least one pin fails, which shows the pins can see
 * that kind of mistake.  The default build (no macro) plants nothing.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- basics */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a * (u128)b) % p);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a + (u128)b) % p);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t p) {
    /* a - b mod p with a, b in [0, p) */
    return (uint64_t)(((u128)a + (u128)p - (u128)b) % p);
}

uint64_t or_powmod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

/* Inverse by Fermat (p prime). */
uint64_t or_invmod(uint64_t a, uint64_t p) { return or_powmod(a, p - 2, p); }

/* rev_l(k): reverse the low l bits of k (Algorithm 1's output order). */
uint64_t or_bitrev(uint64_t k, int l) {
    uint64_t r = 0;
    for (int i = 0; i < l; i++) {
        r = (r << 1) | ((k >> i) & 1);
    }
    return r;
}

static int ilog2_exact(uint64_t L) {
    int l = 0;
    while (((uint64_t)1 << l) < L) l++;
    return l;
}

/* ------------------------------------------------------- number theory */

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every
 * n < 3.3e24, which covers all 64-bit n. */
int or_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Smallest quadratic non-residue of an odd prime p (Euler's criterion). */
uint64_t or_smallest_qnr(uint64_t p) {
    for (uint64_t g = 2; g < p; g++) {
        if (or_powmod(g, (p - 1) / 2, p) == p - 1) return g;
    }
    return 0;
}

/* Smallest prime q > lo with q = 1 mod 2^k (searched in steps of 2^k). */
uint64_t or_find_prime_above(uint64_t lo, int k) {
    uint64_t step = (uint64_t)1 << k;
    uint64_t q = (lo / step) * step + 1;
    while (q <= lo) q += step;
    for (; q > lo; q += step) {
        if (or_is_prime(q)) return q;
    }
    return 0;
}

/* omega = g^((p-1)/L) with g the smallest QNR: a primitive L-th root of
 * unity when L is a power of two dividing p-1 (g has order divisible by the
 * full 2-part of p-1). */
uint64_t or_root_of_unity(uint64_t p, uint64_t L) {
    uint64_t g = or_smallest_qnr(p);
    if (g == 0 || (p - 1) % L != 0) return 0;
    return or_powmod(g, (p - 1) / L, p);
}

/* ------------------------------------------------------ the definition */

/* Section 1: b_j = sum_{i<L} w^{ij} a_i.  Algorithm 1 emits the DFT in
 * bit-reversed order, so out[k] = b_{rev_l(k)}.  O(L^2). */
void or_dft_naive(uint64_t p, uint64_t w, uint64_t L, const uint64_t *a, uint64_t *out) {
    int l = ilog2_exact(L);
    for (uint64_t k = 0; k < L; k++) {
        uint64_t j = MUTANT(1) ? k : or_bitrev(k, l);
        uint64_t wj = or_powmod(w, j, p);
        uint64_t acc = 0, x = 1;
        for (uint64_t i = 0; i < L; i++) {
            acc = addmod(acc, mulmod(x, a[i], p), p);
            x = mulmod(x, wj, p);
        }
        out[k] = acc;
    }
}

/* Inverse map obtained by running Algorithm 1 backwards (Section 4): takes
 * y in bit-reversed order and returns out[i] = sum_j w^{-ij} y[rev(j)],
 * which equals L * a_i when y is the forward transform of a.  O(L^2). */
void or_idft_naive(uint64_t p, uint64_t w, uint64_t L, const uint64_t *y, uint64_t *out) {
    int l = ilog2_exact(L);
    uint64_t winv = or_invmod(w, p);
    for (uint64_t i = 0; i < L; i++) {
        uint64_t wi = or_powmod(winv, i, p);
        uint64_t acc = 0, x = 1;
        for (uint64_t j = 0; j < L; j++) {
            acc = addmod(acc, mulmod(x, y[or_bitrev(j, l)], p), p);
            x = mulmod(x, wi, p);
        }
        out[i] = acc;
    }
}

/* ------------------------------------------------------ Algorithm 1 */

/* Algorithm 1 (Section 1), in place: for i = 1..l, zeta = w^(2^(i-1)),
 * m = 2^(l-i); for each block t = 2jm and k < m the pair
 * (x[t+k], x[t+k+m]) becomes (x[t+k] + x[t+k+m], zeta^k (x[t+k] - x[t+k+m])).
 * Every operation is fully reduced mod p.  Output in bit-reversed order. */
void or_ntt_ref(uint64_t p, uint64_t w, uint64_t L, uint64_t *x) {
    int l = ilog2_exact(L);
    for (int i = 1; i <= l; i++) {
        uint64_t zeta = or_powmod(w, (uint64_t)1 << (i - 1), p);
        uint64_t m = (uint64_t)1 << (l - i);
        for (uint64_t j = 0; j < ((uint64_t)1 << (i - 1)); j++) {
            uint64_t t = 2 * j * m;
            uint64_t zk = MUTANT(3) ? zeta : 1; /* zeta^k, k = 0 */
            for (uint64_t k = 0; k < m; k++) {
                uint64_t X = x[t + k], Y = x[t + k + m];
                x[t + k] = addmod(X, Y, p);
                x[t + k + m] = MUTANT(2) ? mulmod(zk, submod(Y, X, p), p)
                                         : mulmod(zk, submod(X, Y, p), p);
                zk = mulmod(zk, zeta, p);
            }
        }
    }
}

/* Algorithm 1 run backwards (Section 4): stages i = l..1 with the inverse
 * twiddle zeta^{-k}; the pair (X, Y) becomes (X + zeta^{-k} Y,
 * X - zeta^{-k} Y), the inverse of the forward butterfly up to a factor 2.
 * Bit-reversed input, natural-order output, unnormalised (scaled by L). */
void or_intt_ref(uint64_t p, uint64_t w, uint64_t L, uint64_t *x) {
    int l = ilog2_exact(L);
    uint64_t winv = MUTANT(4) ? w : or_invmod(w, p);
    for (int i = l; i >= 1; i--) {
        uint64_t zeta = or_powmod(winv, (uint64_t)1 << (i - 1), p);
        uint64_t m = (uint64_t)1 << (l - i);
        for (uint64_t j = 0; j < ((uint64_t)1 << (i - 1)); j++) {
            uint64_t t = 2 * j * m;
            uint64_t zk = 1;
            for (uint64_t k = 0; k < m; k++) {
                uint64_t X = x[t + k];
                uint64_t WY = mulmod(zk, x[t + k + m], p);
                x[t + k] = addmod(X, WY, p);
                x[t + k + m] = submod(X, WY, p);
                zk = mulmod(zk, zeta, p);
            }
        }
    }
}

/* Batched forms: `batch` transforms at a distance of `stride` words. */
void or_ntt_ref_batch(uint64_t p, uint64_t w, uint64_t L, uint64_t *x, uint64_t batch, uint64_t stride) {
    for (uint64_t b = 0; b < batch; b++) or_ntt_ref(p, w, L, x + b * (MUTANT(6) ? L : stride));
}

void or_intt_ref_batch(uint64_t p, uint64_t w, uint64_t L, uint64_t *x, uint64_t batch, uint64_t stride) {
    for (uint64_t b = 0; b < batch; b++) or_intt_ref(p, w, L, x + b * (MUTANT(6) ? L : stride));
}

/* ------------------------------------------- polynomial multiplication */

/* Section 1 application: c_k = sum_{i+j=k} a_i b_j mod p, schoolbook. */
void or_polymul_schoolbook(uint64_t p, const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb,
                           uint64_t *c) {
    if (na == 0 || nb == 0) return;
    for (uint64_t k = 0; k < na + nb - 1; k++) c[k] = 0;
    for (uint64_t i = 0; i < na; i++) {
        for (uint64_t j = 0; j < nb; j++) {
            uint64_t k = MUTANT(5) ? i + j + (i == 1 && j == 1) : i + j;
            if (k >= na + nb - 1) k = na + nb - 2;
            c[k] = addmod(c[k], mulmod(a[i], b[j], p), p);
        }
    }
}

/* Convolution theorem through Algorithm 1: zero-pad both operands to
 * L = nextpow2(na + nb - 1), forward-transform them with a primitive L-th
 * root, multiply pointwise, run the transform backwards and divide by L.
 * Returns 0 on success, -1 when p has no L-th root or memory runs out. */
int or_polymul_ntt(uint64_t p, const uint64_t *a, uint64_t na, const uint64_t *b, uint64_t nb, uint64_t *c) {
    if (na == 0 || nb == 0) return 0;
    uint64_t n = na + nb - 1, L = 1;
    while (L < n) L <<= 1;
    if (L < 2) L = 2;
    uint64_t w = or_root_of_unity(p, L);
    if (w == 0) return -1;
    uint64_t *A = (uint64_t *)calloc(L, sizeof(uint64_t));
    uint64_t *B = (uint64_t *)calloc(L, sizeof(uint64_t));
    if (!A || !B) { free(A); free(B); return -1; }
    memcpy(A, a, na * sizeof(uint64_t));
    memcpy(B, b, nb * sizeof(uint64_t));
    or_ntt_ref(p, w, L, A);
    or_ntt_ref(p, w, L, B);
    for (uint64_t i = 0; i < L; i++) A[i] = mulmod(A[i], B[i], p);
    or_intt_ref(p, w, L, A);
    uint64_t Linv = or_invmod(L % p, p);
    for (uint64_t i = 0; i < n; i++) c[i] = mulmod(A[i], Linv, p);
    free(A);
    free(B);
    return 0;
}

/* One output position of the forward transform, straight from the Section 1
 * definition: out[k] = b_{rev_l(k)} = sum_i w^(i rev_l(k)) a_i.  O(L); used to
 * check sampled positions of transforms too large for a full comparison. */
uint64_t or_dft_at(uint64_t p, uint64_t w, uint64_t L, const uint64_t *a, uint64_t k) {
    int l = ilog2_exact(L);
    uint64_t wj = or_powmod(w, or_bitrev(k, l), p);
    uint64_t acc = 0, x = 1;
    for (uint64_t i = 0; i < L; i++) {
        acc = addmod(acc, mulmod(x, a[i], p), p);
        x = mulmod(x, wj, p);
    }
    return acc;
}
