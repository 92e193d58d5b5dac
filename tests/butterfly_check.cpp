// Host-side check of the library's butterflies (csrc/modarith.cuh) against
// Theorems 1-4 of Harvey, arXiv:1205.2926: for every input in the stated
// range, each output lies in the stated interval and is congruent to the
// exact value mod p.  Exhaustive at beta = 2^8 (every prime in range, every
// W, every X and Y), sampled with extreme values at beta = 2^16, 2^32 and
// 2^64.  Test infrastructure: built and run by tests/test_butterflies.py.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <initializer_list>

#include "modarith.cuh"

using namespace ntt;
typedef unsigned __int128 u128;

static long long fails = 0;
static bool quiet = false;  // the negative control expects failures

static bool isprime_u64(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t d = 2; d * d <= n && d < 100000; d++)
        if (n % d == 0) return n == d;
    return true;  // only used with n < 2^33 or with known primes below
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

template <typename W>
struct Consts {
    W p, p2, w, wq, wm, J;
};

template <typename W>
static Consts<W> make(uint64_t p, uint64_t w, int bits) {
    Consts<W> c;
    c.p = (W)p;
    c.p2 = (W)(2 * p);
    c.w = (W)w;
    c.wq = (W)(((u128)w << bits) / p);                        // floor(W beta / p)
    c.wm = (W)(((u128)w << bits) % p);                        // beta W mod p
    uint64_t inv = 1;                                         // p^-1 mod 2^64 by Newton
    for (int i = 0; i < 7; i++) inv *= 2 - p * inv;
    c.J = (W)inv;
    return c;
}

template <typename W>
static void check_one(const Consts<W> &c, uint64_t X, uint64_t Y, uint64_t p, int which) {
    uint64_t w = c.w;
    W x = (W)X, y = (W)Y;
    uint64_t ex, ey, lim;
    switch (which) {
        case 2:  // Algorithm 2: [0,p) -> [0,p)
            bfly_fwd_ntl(x, y, c.w, c.wq, c.p);
            ex = (X + Y) % p;
            ey = mulmod(w, (X + p - Y % p) % p, p);
            lim = p;
            break;
        case 3:  // Algorithm 3: [0,2p) -> [0,2p)
            bfly_fwd_lazy(x, y, c.w, c.wq, c.p, c.p2);
            ex = (X + Y) % p;
            ey = mulmod(w, (X % p + p - Y % p) % p, p);
            lim = 2 * p;
            break;
        case 4:  // Algorithm 4: [0,4p) -> [0,4p)
            bfly_inv_lazy(x, y, c.w, c.wq, c.p, c.p2);
            ex = (X % p + mulmod(w, Y % p, p)) % p;
            ey = (X % p + p - mulmod(w, Y % p, p)) % p;
            lim = 4 * p;
            break;
        case 5:  // Algorithm 5: [0,2p) -> [0,2p)
            bfly_fwd_mont(x, y, c.wm, c.J, c.p, c.p2);
            ex = (X + Y) % p;
            ey = mulmod(w, (X % p + p - Y % p) % p, p);
            lim = 2 * p;
            break;
        case 7:  // Montgomery inverse (Algorithm 4 with Algorithm 5's product): [0,4p) -> [0,4p)
            bfly_inv_mont(x, y, c.wm, c.J, c.p, c.p2);
            ex = (X % p + mulmod(w, Y % p, p)) % p;
            ey = (X % p + p - mulmod(w, Y % p, p)) % p;
            lim = 4 * p;
            break;
        case 6:  // fully reduced inverse: [0,p) -> [0,p)
            bfly_inv_ntl(x, y, c.w, c.wq, c.p);
            ex = (X + mulmod(w, Y, p)) % p;
            ey = (X + p - mulmod(w, Y, p)) % p;
            lim = p;
            break;
        case 13:  // W = 1 forms (only called with w == 1)
            bfly_fwd_lazy_w1(x, y, c.p2);
            ex = (X + Y) % p;
            ey = (X % p + p - Y % p) % p;
            lim = 2 * p;
            break;
        case 12:
            bfly_fwd_ntl_w1(x, y, c.p);
            ex = (X + Y) % p;
            ey = (X + p - Y) % p;
            lim = p;
            break;
        case 14:
            bfly_inv_lazy_w1(x, y, c.p2);
            ex = (X % p + Y % p) % p;
            ey = (X % p + p - Y % p) % p;
            lim = 4 * p;
            break;
        case 8:  // Moeller's Algorithm 2, p < beta/phi: [0,p) -> [0,p)
            bfly_fwd_moller(x, y, c.w, c.wq, c.p);
            ex = (uint64_t)(((u128)X + Y) % p);
            ey = mulmod(w, (uint64_t)(((u128)X + p - Y) % p), p);
            lim = p;
            break;
        case 9:  // its fully reduced inverse, p < beta/phi
            bfly_inv_moller(x, y, c.w, c.wq, c.p);
            ex = (uint64_t)(((u128)X + mulmod(w, Y, p)) % p);
            ey = (uint64_t)(((u128)X + p - mulmod(w, Y, p)) % p);
            lim = p;
            break;
        case 18:  // Moeller's W = 1 form
            bfly_moller_w1(x, y, c.p);
            ex = (uint64_t)(((u128)X + Y) % p);
            ey = (uint64_t)(((u128)X + p - Y) % p);
            lim = p;
            break;
        default:  // 16: fully reduced inverse with W = 1
            bfly_inv_ntl_w1(x, y, c.p);
            ex = (X + Y) % p;
            ey = (X + p - Y) % p;
            lim = p;
            break;
    }
    uint64_t gx = (uint64_t)x, gy = (uint64_t)y;
    if (gx >= lim || gy >= lim || gx % p != ex || gy % p != ey) {
        if (fails < 10 && !quiet)
            printf("FAIL alg%d p=%llu W=%llu X=%llu Y=%llu -> %llu %llu (want %llu %llu mod p, < %llu)\n", which,
                   (unsigned long long)p, (unsigned long long)w, (unsigned long long)X, (unsigned long long)Y,
                   (unsigned long long)gx, (unsigned long long)gy, (unsigned long long)ex, (unsigned long long)ey,
                   (unsigned long long)lim);
        fails++;
    }
}

static uint64_t in_limit(int which, uint64_t p) {
    return which == 3 || which == 5 || which == 13 ? 2 * p : which == 4 || which == 7 || which == 14 ? 4 * p : p;
}

// Exhaustive at beta = 2^8.
static long long exhaustive8() {
    long long n = 0;
    for (uint64_t p = 3; p < 256; p++) {
        if (!isprime_u64(p)) continue;
        for (int which : {2, 3, 4, 5, 6, 7, 8, 9, 12, 13, 14, 16, 18}) {
            bool lazy = which == 3 || which == 4 || which == 5 || which == 7 || which == 13 || which == 14;
            bool moller = which == 8 || which == 9 || which == 18;
            if (lazy && p >= 64) continue;                 // p < beta/4 (Algorithms 3-5)
            if (!lazy && !moller && p >= 128) continue;    // p < beta/2 (Algorithm 2)
            if (moller && 1.6180339887498949 * p >= 256.0) continue;  // p < beta/phi (end of Section 2)
            for (uint64_t w = 1; w < (which >= 12 ? 2 : p); w++) {
                Consts<uint8_t> c = make<uint8_t>(p, w, 8);
                uint64_t lim = in_limit(which, p);
                for (uint64_t X = 0; X < lim; X++)
                    for (uint64_t Y = 0; Y < lim; Y++, n++) check_one(c, X, Y, p, which);
            }
        }
    }
    return n;
}

static uint64_t rng_state = 88172645463325252ull;
static uint64_t rnd() {
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}

template <typename W>
static long long sampled(uint64_t p, int bits, int samples) {
    long long n = 0;
    const long double beta = bits == 64 ? 18446744073709551616.0L : (long double)(1ull << bits);
    for (int which : {2, 3, 4, 5, 6, 7, 8, 9, 12, 13, 14, 16, 18}) {
        const bool lazy = which == 3 || which == 4 || which == 5 || which == 7 || which == 13 || which == 14;
        const bool moller = which == 8 || which == 9 || which == 18;
        if (lazy && (long double)p * 4 >= beta) continue;
        if (!lazy && !moller && (long double)p * 2 >= beta) continue;
        if (moller && (long double)p * 1.6180339887498948482L >= beta) continue;
        uint64_t lim = in_limit(which, p);
        for (int s = 0; s < samples; s++) {
            uint64_t w = 1 + rnd() % (p - 1);
            if (s < 4) w = s < 2 ? 1 + s : p - 1 - (s - 2);
            if (which >= 12) w = 1;
            Consts<W> c = make<W>(p, w, bits);
            uint64_t edge[6] = {0, 1, p - 1, p % lim, lim - 1, lim - 2};
            for (int t = 0; t < 64; t++) {
                uint64_t X = t < 36 ? edge[t % 6] : rnd() % lim;
                uint64_t Y = t < 36 ? edge[t / 6] : rnd() % lim;
                if (X >= lim) X = lim - 1;
                if (Y >= lim) Y = lim - 1;
                check_one(c, X, Y, p, which);
                n++;
            }
        }
    }
    return n;
}

// Negative control: the unmodified Algorithm 2 leaves beta/2 <= p < beta/phi
// uncovered (X + Y overflows the word), which is what Moeller's form fixes.
static long long alg2_beyond_half8() {
    const long long before = fails;
    quiet = true;
    for (uint64_t p = 128; 1.6180339887498949 * p < 256.0; p++) {
        if (!isprime_u64(p)) continue;
        for (uint64_t w = 1; w < p; w++) {
            Consts<uint8_t> c = make<uint8_t>(p, w, 8);
            for (uint64_t X = 0; X < p; X++)
                for (uint64_t Y = 0; Y < p; Y++) check_one(c, X, Y, p, 2);
        }
    }
    const long long bad = fails - before;
    fails = before;  // expected failures, not counted
    quiet = false;
    return bad;
}

int main() {
    long long n = exhaustive8();
    printf("beta=2^8 exhaustive: %lld cases\n", n);
    const long long neg = alg2_beyond_half8();
    printf("unmodified Algorithm 2 at beta/2 <= p < beta/phi (beta=2^8): %lld wrong outputs (expected > 0)\n", neg);
    if (neg == 0) fails++;
    // beta = 2^16: primes just below beta/4 and beta/2 and a few small ones
    for (uint64_t p : {16381ull, 16369ull, 12289ull, 7681ull, 257ull}) n += sampled<uint16_t>(p, 16, 20000);
    // beta = 2^32: the library's 32-bit primes and the largest prime below 2^30
    for (uint64_t p : {998244353ull, 1073479681ull, 1072496641ull, 1071513601ull, 1073741789ull})
        n += sampled<uint32_t>(p, 32, 20000);
    // beta = 2^64: the 62-bit workload prime and primes close to 2^62
    for (uint64_t p : {2305843009448574977ull, 4611686018427387847ull, 4611686018326724609ull})
        n += sampled<uint64_t>(p, 64, 20000);
    // Moeller's range beta/2 <= p < beta/phi (and just below beta/2)
    for (uint64_t p : {40499ull, 40193ull, 32771ull, 32749ull}) n += sampled<uint16_t>(p, 16, 20000);
    for (uint64_t p : {2654435761ull, 2649751553ull, 2147483659ull, 2147483647ull}) n += sampled<uint32_t>(p, 32, 20000);
    for (uint64_t p : {11400714819323198393ull, 11400714819167322113ull, 9223372036854775837ull})
        n += sampled<uint64_t>(p, 64, 20000);
    printf("total cases %lld, failures %lld\n", n, fails);
    return fails == 0 ? 0 : 1;
}
