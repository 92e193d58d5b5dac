// ntt_polymul.cu -- polynomial products mod p through the transform (the
// application named in Section 1 of Harvey, arXiv:1205.2926):
// c = a * b = L^-1 * inverse(forward(a) . forward(b)), L = nextpow2(na+nb-1).
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "modarith.cuh"
#include "ntt_internal.hpp"
#include "ntt_polymul.hpp"

namespace ntt {

// buf[0:L] = a zero-padded, buf[L:2L] = b zero-padded.
template <typename W>
__global__ void k_pad2(W *__restrict__ buf, const W *__restrict__ a, uint64_t na, const W *__restrict__ b,
                       uint64_t nb, uint64_t L) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (uint64_t)gridDim.x * blockDim.x) {
        buf[i] = i < na ? a[i] : (W)0;
        buf[L + i] = i < nb ? b[i] : (W)0;
    }
}

// A_i <- A_i B_i L^-1 mod p.  The general product uses the Montgomery
// reduction of Algorithm 5 (R1 beta + R0 = A B, Q = R0 J, H = hi(Q p),
// R1 - H + p = A B beta^-1 in [0, 2p) since A, B < 2p and p < beta/4), then
// a Shoup product by K = L^-1 beta mod p (precomputed K' = floor(K beta/p))
// removes beta^-1 and scales by L^-1; the result stays in [0, 2p), inside the
// inverse transform's input range [0, 4p).
template <typename W>
__global__ void k_pointwise(W *__restrict__ A, const W *__restrict__ B, uint64_t L, W p, W J, W K, W Kq) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += (uint64_t)gridDim.x * blockDim.x) {
        W y = mont_mul(A[i], B[i], J, p);
        // fully reduced: the inverse transform's input interval is [0, p)
        // for the fully reduced butterflies (Algorithm 2)
        A[i] = csub(shoup_mul(y, K, Kq, p), p);
    }
}

template <typename W>
__global__ void k_copy(W *__restrict__ dst, const W *__restrict__ src, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

static unsigned grid_for(uint64_t n) {
    uint64_t g = (n + 255) / 256;
    return (unsigned)std::min<uint64_t>(g, 152 * 16);
}

// Plans cached per (device, p, L, butterfly variant; -1 = the plan's
// default); kept for the life of the process.
static std::mutex g_cache_mu;
static std::map<std::tuple<int, uint64_t, uint64_t, int>, ntt_plan_s *> g_cache;

int polymul_plan(uint64_t p, uint64_t L, ntt_plan_s **out, int variant) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto key = std::make_tuple(dev, p, L, variant);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return NTT_OK;
    }
    uint64_t w = 0;
    int rc = ntt_root_of_unity(p, L, &w);
    if (rc) return rc;
    ntt_plan_t pl = nullptr;
    rc = ntt_plan(&pl, p, w, L);
    if (rc) return rc;
    if (variant >= 0) {
        rc = ntt_plan_set_variant(pl, variant);
        if (rc) {
            ntt_plan_destroy(pl);
            return rc;
        }
    }
    g_cache[key] = pl;
    *out = pl;
    return NTT_OK;
}

int polymul_validate(uint64_t p, size_t na, size_t nb, uint64_t *L_out) {
    if (na == 0 || nb == 0) return NTT_ERR_ARG;
    if (p < 3 || p >= (1ull << 62) || !nt::is_prime(p)) return NTT_ERR_MODULUS;
    const uint64_t n = (uint64_t)na + nb - 1;
    uint64_t L = 2;
    while (L < n) L <<= 1;
    if (L > (1ull << 26)) return NTT_ERR_RANGE;
    if ((p - 1) % L) return NTT_ERR_LENGTH;
    *L_out = L;
    return NTT_OK;
}

template <typename W>
static int enqueue_pointwise_t(ntt_plan_s *pl, W *A, const W *B, uint64_t L, cudaStream_t st) {
    const int bits = pl->wbytes * 8;
    uint64_t J = 1;
    for (int i = 0; i < 7; ++i) J *= 2 - pl->p * J;
    const uint64_t K = (uint64_t)(((unsigned __int128)pl->L_inv << bits) % pl->p);
    const uint64_t Kq = nt::shoup_quotient(K, pl->p, bits);
    k_pointwise<W><<<grid_for(L), 256, 0, st>>>(A, B, L, (W)pl->p, (W)J, (W)K, (W)Kq);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "k_pointwise");
}

int enqueue_pointwise(ntt_plan_s *pl, void *A, const void *B, uint64_t L, cudaStream_t st) {
    if (pl->wbytes == 4) return enqueue_pointwise_t<uint32_t>(pl, (uint32_t *)A, (const uint32_t *)B, L, st);
    return enqueue_pointwise_t<uint64_t>(pl, (uint64_t *)A, (const uint64_t *)B, L, st);
}

template <typename W>
static int enqueue_polymul_t(ntt_plan_s *pl, const W *a, size_t na, const W *b, size_t nb, W *c, W *buf,
                             cudaStream_t st) {
    const uint64_t L = pl->L, n = (uint64_t)na + nb - 1;
    const W p = (W)pl->p;
    const int bits = pl->wbytes * 8;
    k_pad2<W><<<grid_for(L), 256, 0, st>>>(buf, a, na, b, nb, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_pad2");
    int rc = enqueue_transform(pl, 0, buf, 2, L, st);
    if (rc) return rc;
    // J = p^-1 mod beta (Newton iteration), K = L^-1 beta mod p, K' = floor(K beta / p)
    uint64_t J = 1;
    for (int i = 0; i < 7; ++i) J *= 2 - pl->p * J;
    const uint64_t K = (uint64_t)(((unsigned __int128)pl->L_inv << bits) % pl->p);
    const uint64_t Kq = nt::shoup_quotient(K, pl->p, bits);
    k_pointwise<W><<<grid_for(L), 256, 0, st>>>(buf, buf + L, L, p, (W)J, (W)K, (W)Kq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_pointwise");
    rc = enqueue_transform(pl, 1, buf, 1, L, st);
    if (rc) return rc;
    k_copy<W><<<grid_for(n), 256, 0, st>>>(c, buf, n);
    e = cudaGetLastError();
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "k_copy");
}

int enqueue_polymul(ntt_plan_s *pl, const void *a, size_t na, const void *b, size_t nb, void *c, void *buf,
                    cudaStream_t st) {
    if (pl->wbytes == 4)
        return enqueue_polymul_t<uint32_t>(pl, (const uint32_t *)a, na, (const uint32_t *)b, nb, (uint32_t *)c,
                                           (uint32_t *)buf, st);
    return enqueue_polymul_t<uint64_t>(pl, (const uint64_t *)a, na, (const uint64_t *)b, nb, (uint64_t *)c,
                                       (uint64_t *)buf, st);
}

}  // namespace ntt

using namespace ntt;

extern "C" int polymul_mod_p(uint64_t p, const void *d_a, size_t na, const void *d_b, size_t nb, void *d_c,
                             void *stream) {
    if (!d_a || !d_b || !d_c) return NTT_ERR_ARG;
    uint64_t L = 0;
    int rc = polymul_validate(p, na, nb, &L);
    if (rc) return rc;
    const size_t wb = p < (1ull << 30) ? 4 : 8;
    if (((uintptr_t)d_a | (uintptr_t)d_b | (uintptr_t)d_c) & (wb - 1)) return NTT_ERR_ALIGN;
    ntt_plan_s *pl = nullptr;
    rc = polymul_plan(p, L, &pl);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void *buf = nullptr;
    cudaError_t e = scratch_alloc(&buf, 2 * L * wb, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "cudaMallocAsync");
    rc = enqueue_polymul(pl, d_a, na, d_b, nb, d_c, buf, st);
    e = cudaFreeAsync(buf, st);
    if (rc) return rc;
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "cudaFreeAsync");
}

// ---------------------------------------------------------------------------
// polymul_mod_p without any allocation.  Its scratch lives in a file-scope
// __device__ array; host code cannot use the array's name as a device
// address (on the host the name is only a stand-in), so the address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, and passed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[NTT_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];

static int noalloc_scratch(int dev, void **out) {
    if (dev < 0 || dev >= 64) return NTT_ERR_ARG;  // devices beyond the table: not supported
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                       "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return NTT_OK;
}

extern "C" int polymul_mod_p_noalloc(ntt_plan_t plan, const void *d_a, size_t na, const void *d_b, size_t nb,
                                     void *d_c, void *stream) {
    if (!plan || !d_a || !d_b || !d_c || na == 0 || nb == 0) return NTT_ERR_ARG;
    if (plan->variant != NTT_VARIANT_LAZY) return NTT_ERR_ARG;
    const uint64_t n = (uint64_t)na + nb - 1;
    if (n > plan->L) return NTT_ERR_LENGTH;
    const size_t wb = (size_t)plan->wbytes;
    if (2 * plan->L * wb > (uint64_t)NTT_NOALLOC_SCRATCH_BYTES) return NTT_ERR_RANGE;
    if (((uintptr_t)d_a | (uintptr_t)d_b | (uintptr_t)d_c) & (wb - 1)) return NTT_ERR_ALIGN;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->device) return NTT_ERR_ARG;
    void *buf = nullptr;
    int rc = noalloc_scratch(dev, &buf);
    if (rc) return rc;
    return enqueue_polymul(plan, d_a, na, d_b, nb, d_c, buf, (cudaStream_t)stream);
}
