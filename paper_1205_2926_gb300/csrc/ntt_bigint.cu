// ntt_bigint.cu -- products of large integers through the transform: the
// application of Section 1 of Harvey, arXiv:1205.2926 ("multiplying large
// integers" via products of polynomials over F_p for word-sized primes p).
//
// The integers are little-endian arrays of 32-bit limbs, i.e. the values at
// x = 2^32 of polynomials with coefficients < 2^32.  Their product's
// coefficients are below min(na, nb) * (2^32 - 1)^2 < 2^86, so three products
// modulo p1 = 998244353, p2 = 167772161, p3 = 469762049 (p1 p2 p3 > 2^86,
// each 1 mod 2^23) determine them exactly (Chinese remaindering, Garner's
// mixed-radix form).  Each modular product is the library's polynomial
// product (forward transforms, pointwise product, inverse transform); the
// recombined coefficients V_k (< 2^87, three words) are then summed at their
// word offsets and the carries propagated with a parallel scan: the carry
// out of a run of limbs is a function of the carry in (0, 1 or 2), and such
// functions compose.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "modarith.cuh"
#include "ntt_internal.hpp"
#include "ntt_polymul.hpp"

namespace ntt {

constexpr uint32_t kP1 = 998244353u, kP2 = 167772161u, kP3 = 469762049u;
constexpr int kCrtLogMax = 23;      // product length up to 2^23 limbs
constexpr int kChunk = 16;          // limbs per thread in the carry scan
constexpr int kScanThreads = 256;

// buf[0:L] = a mod p zero-padded, buf[L:2L] = b mod p zero-padded.
__global__ void k_pad_reduce(uint32_t *__restrict__ buf, const uint32_t *__restrict__ a, uint64_t na,
                             const uint32_t *__restrict__ b, uint64_t nb, uint64_t L, uint32_t p) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (uint64_t)gridDim.x * blockDim.x) {
        buf[i] = i < na ? a[i] % p : 0u;
        buf[L + i] = i < nb ? b[i] % p : 0u;
    }
}

struct CrtConsts {
    uint32_t inv12;   // p1^-1 mod p2
    uint32_t inv13;   // p1^-1 mod p3
    uint32_t inv23;   // p2^-1 mod p3
};

// Coefficient k of the product from its residues (Garner):
// V = x1 + p1 x2 + p1 p2 x3 with x1 = r1, x2 = (r2 - x1) p1^-1 mod p2,
// x3 = ((r3 - x1) p1^-1 - x2) p2^-1 mod p3; V < p1 p2 p3 < 2^87.  Its three
// 32-bit words overwrite the three residues in place (each k is one
// thread's).
__global__ void k_crt(uint32_t *__restrict__ r1, uint32_t *__restrict__ r2, uint32_t *__restrict__ r3, uint64_t n,
                      CrtConsts c) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x1 = r1[k];
        const uint64_t x2 = (uint64_t)((r2[k] + kP2 - (uint32_t)(x1 % kP2)) % kP2) * c.inv12 % kP2;
        uint64_t t = (uint64_t)((r3[k] + kP3 - (uint32_t)(x1 % kP3)) % kP3) * c.inv13 % kP3;
        t = (t + kP3 - x2 % kP3) % kP3;
        const uint64_t x3 = t * c.inv23 % kP3;
        const unsigned __int128 v =
            (unsigned __int128)x1 + (unsigned __int128)kP1 * x2 + (unsigned __int128)kP1 * kP2 * x3;
        r1[k] = (uint32_t)v;
        r2[k] = (uint32_t)(v >> 32);
        r3[k] = (uint32_t)(v >> 64);
    }
}

// S_k = word 0 of V_k + word 1 of V_{k-1} + word 2 of V_{k-2} (< 2^33 + 2^23).
__device__ __forceinline__ uint64_t limb_sum(const uint32_t *w0, const uint32_t *w1, const uint32_t *w2, uint64_t k,
                                             uint64_t n) {
    uint64_t s = k < n ? w0[k] : 0;
    if (k >= 1 && k - 1 < n) s += w1[k - 1];
    if (k >= 2 && k - 2 < n) s += w2[k - 2];
    return s;
}

// A carry function maps carry-in 0, 1, 2 to carry-out 0, 1, 2 (2 bits each).
__device__ __forceinline__ uint32_t cf_apply(uint32_t f, uint32_t cin) { return (f >> (2 * cin)) & 3u; }
__device__ __forceinline__ uint32_t cf_then(uint32_t f, uint32_t g) {  // g after f
    return cf_apply(g, cf_apply(f, 0)) | (cf_apply(g, cf_apply(f, 1)) << 2) | (cf_apply(g, cf_apply(f, 2)) << 4);
}
constexpr uint32_t kCfIdentity = 0u | (1u << 2) | (2u << 4);

// The limb sums of [k0, k0 + kChunk) and their carry function (carries
// 0, 1, 2: S_k + 2 < 2^34, so the carry out is at most 2).
__device__ uint32_t chunk_function(const uint32_t *w0, const uint32_t *w1, const uint32_t *w2, uint64_t k0,
                                   uint64_t n, uint64_t nc, uint64_t (&s)[kChunk]) {
#pragma unroll
    for (int j = 0; j < kChunk; ++j) s[j] = k0 + j < nc ? limb_sum(w0, w1, w2, k0 + j, n) : 0;
    uint32_t f = 0;
#pragma unroll
    for (uint32_t cin = 0; cin < 3; ++cin) {
        uint64_t carry = cin;
#pragma unroll
        for (int j = 0; j < kChunk; ++j) carry = (s[j] + carry) >> 32;
        f |= (uint32_t)carry << (2 * cin);
    }
    return f;
}

// Exclusive scan of carry functions across the block (Hillis-Steele in
// shared memory); returns the composition of the functions before this
// thread's and stores the block's full composition in *total.
__device__ uint32_t block_scan(uint32_t f, uint32_t *sh, uint32_t *total) {
    sh[threadIdx.x] = f;
    __syncthreads();
    for (int d = 1; d < kScanThreads; d <<= 1) {
        const uint32_t mine = sh[threadIdx.x];
        const uint32_t prev = threadIdx.x >= (unsigned)d ? sh[threadIdx.x - d] : kCfIdentity;
        __syncthreads();
        sh[threadIdx.x] = cf_then(prev, mine);
        __syncthreads();
    }
    const uint32_t incl = sh[threadIdx.x];
    const uint32_t excl = threadIdx.x ? sh[threadIdx.x - 1] : kCfIdentity;
    *total = sh[kScanThreads - 1];
    __syncthreads();
    (void)incl;
    return excl;
}

// Pass 1: the carry function of each block's run of limbs.
__global__ void __launch_bounds__(kScanThreads) k_carry_blocks(const uint32_t *w0, const uint32_t *w1,
                                                                 const uint32_t *w2, uint64_t n, uint64_t nc,
                                                                 uint32_t *block_f) {
    __shared__ uint32_t sh[kScanThreads];
    const uint64_t k0 = ((uint64_t)blockIdx.x * kScanThreads + threadIdx.x) * kChunk;
    uint64_t s[kChunk];
    const uint32_t f = k0 < nc ? chunk_function(w0, w1, w2, k0, n, nc, s) : kCfIdentity;
    uint32_t total;
    block_scan(f, sh, &total);
    if (threadIdx.x == 0) block_f[blockIdx.x] = total;
}

// Pass 2: carry into each block (one thread; at most 2^23 / 4096 blocks).
__global__ void k_carry_prefix(const uint32_t *block_f, uint32_t nblocks, uint8_t *block_cin) {
    if (threadIdx.x || blockIdx.x) return;
    uint32_t carry = 0;
    for (uint32_t b = 0; b < nblocks; ++b) {
        block_cin[b] = (uint8_t)carry;
        carry = cf_apply(block_f[b], carry);
    }
}

// Pass 3: each thread finds its carry-in and writes its limbs.
__global__ void __launch_bounds__(kScanThreads) k_carry_apply(const uint32_t *w0, const uint32_t *w1,
                                                                const uint32_t *w2, uint64_t n, uint64_t nc,
                                                                const uint8_t *block_cin, uint32_t *out) {
    __shared__ uint32_t sh[kScanThreads];
    const uint64_t k0 = ((uint64_t)blockIdx.x * kScanThreads + threadIdx.x) * kChunk;
    uint64_t s[kChunk];
    const uint32_t f = k0 < nc ? chunk_function(w0, w1, w2, k0, n, nc, s) : kCfIdentity;
    uint32_t total;
    const uint32_t before = block_scan(f, sh, &total);
    uint64_t carry = cf_apply(before, block_cin[blockIdx.x]);
#pragma unroll
    for (int j = 0; j < kChunk; ++j) {
        const uint64_t t = s[j] + carry;
        if (k0 + j < nc) out[k0 + j] = (uint32_t)t;
        carry = t >> 32;
    }
}

static uint64_t inv_mod(uint64_t a, uint64_t m) { return nt::powmod(a % m, m - 2, m); }

static unsigned grid_for(uint64_t n) { return (unsigned)std::min<uint64_t>((n + 255) / 256, 152 * 16); }

}  // namespace ntt

using namespace ntt;

extern "C" int bigint_mul(const uint32_t *a, size_t na, const uint32_t *b, size_t nb, uint32_t *c, void *stream) {
    if (!a || !b || !c || na == 0 || nb == 0) return NTT_ERR_ARG;
    const uint64_t n = (uint64_t)na + nb - 1;  // product coefficients
    uint64_t L = 2;
    while (L < n) L <<= 1;
    if (L > (1ull << kCrtLogMax)) return NTT_ERR_RANGE;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t primes[3] = {kP1, kP2, kP3};
    ntt_plan_s *plans[3];
    for (int i = 0; i < 3; ++i) {
        int rc = polymul_plan(primes[i], L, &plans[i]);
        if (rc) return rc;
    }
    const uint64_t nc = (uint64_t)na + nb;  // product limbs
    const uint64_t nblocks = (nc + (uint64_t)kScanThreads * kChunk - 1) / ((uint64_t)kScanThreads * kChunk);
    uint32_t *buf = nullptr;
    const size_t bytes = 3 * 2 * L * sizeof(uint32_t) + nblocks * (sizeof(uint32_t) + 1) + 16;
    cudaError_t e = scratch_alloc((void **)&buf, bytes, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "bigint scratch");
    int rc = NTT_OK;
    for (int i = 0; i < 3 && rc == NTT_OK; ++i) {
        uint32_t *bi = buf + (size_t)i * 2 * L;
        k_pad_reduce<<<grid_for(L), 256, 0, st>>>(bi, a, na, b, nb, L, primes[i]);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_pad_reduce");
        if (rc == NTT_OK) rc = enqueue_transform(plans[i], 0, bi, 2, L, st);
        if (rc == NTT_OK) rc = enqueue_pointwise(plans[i], bi, bi + L, L, st);
        if (rc == NTT_OK) rc = enqueue_transform(plans[i], 1, bi, 1, L, st);
    }
    if (rc == NTT_OK) {
        CrtConsts cc;
        cc.inv12 = (uint32_t)inv_mod(kP1, kP2);
        cc.inv13 = (uint32_t)inv_mod(kP1, kP3);
        cc.inv23 = (uint32_t)inv_mod(kP2, kP3);
        uint32_t *r1 = buf, *r2 = buf + 2 * L, *r3 = buf + 4 * L;
        uint32_t *block_f = buf + 6 * L;
        uint8_t *block_cin = reinterpret_cast<uint8_t *>(block_f + nblocks);
        k_crt<<<grid_for(n), 256, 0, st>>>(r1, r2, r3, n, cc);
        k_carry_blocks<<<(unsigned)nblocks, kScanThreads, 0, st>>>(r1, r2, r3, n, nc, block_f);
        k_carry_prefix<<<1, 32, 0, st>>>(block_f, (uint32_t)nblocks, block_cin);
        k_carry_apply<<<(unsigned)nblocks, kScanThreads, 0, st>>>(r1, r2, r3, n, nc, block_cin, c);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "carry scan");
    }
    e = cudaFreeAsync(buf, st);
    if (rc == NTT_OK && e != cudaSuccess) rc = cuda_fail(e, "bigint free");
    return rc;
}
