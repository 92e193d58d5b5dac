// butterfly_rate.cu -- register-only throughput of the library's butterflies
// on the current GPU (the integer-pipe roof used by bench.py).
//
// Each thread keeps 8 vectors of 4 residues in registers and runs rounds of
// three radix-2 stages (12 butterflies per lane) with twiddles held in
// registers, so no memory traffic limits the rate.  Reported: butterflies
// per clock per SM at the GPU's maximum clock, per butterfly form, and the
// raw rates of mul.hi.u32 and mad.lo.u32 chains.  out[] (grid*block words)
// receives an xor of each thread's data so nothing is optimised away.
// Built and run by `python bench.py --workload probe` (not part of the library).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "modarith.cuh"  // the library's butterflies (compiled with -I paper_1205_2926_gb300/csrc)

using namespace ntt;

// Alternative instruction forms of Algorithm 3's butterfly (same results):
// the Shoup product written with explicit PTX multiplies, the final
// low-product difference as one multiply-add by -p, and the additions in
// different groupings.
__device__ __forceinline__ uint32_t shoup_ptx(uint32_t t, uint32_t w, uint32_t wq, uint32_t negp) {
    uint32_t q, r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(q) : "r"(wq), "r"(t));
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(w), "r"(t));
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(q), "r"(negp), "r"(r));
    return r;
}

template <int F>
__device__ __forceinline__ void bf(uint32_t &x, uint32_t &y, uint32_t w, uint32_t wq, uint32_t p, uint32_t p2) {
    if (F == 0) bfly_fwd_lazy(x, y, w, wq, p, p2);
    if (F == 1) bfly_fwd_ntl(x, y, w, wq, p);
    if (F == 2) bfly_inv_lazy(x, y, w, wq, p, p2);
    if (F == 3) bfly_inv_ntl(x, y, w, wq, p);
    if (F == 4) bfly_fwd_lazy_w1(x, y, p2);
    if (F == 5) {  // PTX Shoup product with mad by -p
        const uint32_t s = umin(x + y, x + y - p2);
        const uint32_t t = x - y + p2;
        y = shoup_ptx(t, w, wq, 0u - p);
        x = s;
    }
    if (F == 6) {  // t first, sum reduced by select
        const uint32_t t = x - y + p2;
        const uint32_t u = x + y;
        x = u >= p2 ? u - p2 : u;
        y = shoup_ptx(t, w, wq, 0u - p);
    }
    if (F == 7) {  // sum by a signed correction: u - 2p, plus 2p when negative
        const uint32_t t = x - y + p2;
        const int32_t d = (int32_t)(x + y - p2);
        x = (uint32_t)d + (p2 & (uint32_t)(d >> 31));
        y = shoup_ptx(t, w, wq, 0u - p);
    }
    if (F == 8) {  // Algorithm 2 with the PTX Shoup product
        const uint32_t s = umin(x + y, x + y - p);
        uint32_t t = x - y;
        t = umin(t, t + p);
        const uint32_t r = shoup_ptx(t, w, wq, 0u - p);
        x = s;
        y = umin(r, r - p);
    }
    if (F == 10) {  // Algorithm 3 written out in PTX, minimum form
        asm("{\n .reg .u32 u, s2, t, q, r;\n"
            " add.u32 u, %0, %1;\n sub.u32 s2, u, %4;\n"
            " sub.u32 t, %0, %1;\n add.u32 t, t, %4;\n"
            " mul.hi.u32 q, %3, t;\n mul.lo.u32 r, %2, t;\n mad.lo.u32 %1, q, %5, r;\n"
            " min.u32 %0, u, s2;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p));
    }
    if (F == 11) {  // PTX, compare-and-select form of the sum
        asm("{\n .reg .u32 u, s2, t, q, r;\n .reg .pred g;\n"
            " add.u32 u, %0, %1;\n sub.u32 t, %0, %1;\n add.u32 t, t, %4;\n"
            " mul.hi.u32 q, %3, t;\n mul.lo.u32 r, %2, t;\n mad.lo.u32 %1, q, %5, r;\n"
            " setp.ge.u32 g, u, %4;\n sub.u32 s2, u, %4;\n selp.u32 %0, s2, u, g;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p));
    }
    if (F == 12) {  // PTX, X - Y + 2p as X + (2p - Y), sum by minimum
        asm("{\n .reg .u32 u, s2, t, q, r;\n"
            " sub.u32 t, %4, %1;\n add.u32 t, t, %0;\n add.u32 u, %0, %1;\n sub.u32 s2, u, %4;\n"
            " mul.hi.u32 q, %3, t;\n mul.lo.u32 r, %2, t;\n mad.lo.u32 %1, q, %5, r;\n"
            " min.u32 %0, u, s2;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p));
    }
    if (F == 13) {  // PTX, Shoup difference as an explicit subtraction of q p
        asm("{\n .reg .u32 u, s2, t, q, r, qp;\n .reg .pred g;\n"
            " add.u32 u, %0, %1;\n sub.u32 t, %0, %1;\n add.u32 t, t, %4;\n"
            " mul.hi.u32 q, %3, t;\n mul.lo.u32 r, %2, t;\n mul.lo.u32 qp, q, %6;\n sub.u32 %1, r, qp;\n"
            " setp.ge.u32 g, u, %4;\n sub.u32 s2, u, %4;\n selp.u32 %0, s2, u, g;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p), "r"(p));
    }
    if (F == 14) {  // Algorithm 4 in PTX, minimum form
        asm("{\n .reg .u32 a, a2, q, r, tt;\n"
            " sub.u32 a2, %0, %4;\n min.u32 a, %0, a2;\n"
            " mul.hi.u32 q, %3, %1;\n mul.lo.u32 r, %2, %1;\n mad.lo.u32 tt, q, %5, r;\n"
            " add.u32 %0, a, tt;\n sub.u32 %1, a, tt;\n add.u32 %1, %1, %4;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p));
    }
    if (F == 15) {  // Algorithm 4 in PTX, compare-and-select form
        asm("{\n .reg .u32 a, a2, q, r, tt;\n .reg .pred g;\n"
            " setp.ge.u32 g, %0, %4;\n sub.u32 a2, %0, %4;\n selp.u32 a, a2, %0, g;\n"
            " mul.hi.u32 q, %3, %1;\n mul.lo.u32 r, %2, %1;\n mad.lo.u32 tt, q, %5, r;\n"
            " add.u32 %0, a, tt;\n sub.u32 %1, a, tt;\n add.u32 %1, %1, %4;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p));
    }
    if (F == 16) {  // Algorithm 2 in PTX, compare-and-select corrections
        asm("{\n .reg .u32 u, s2, t, t2, q, r, r2;\n .reg .pred g, h, k;\n"
            " add.u32 u, %0, %1;\n sub.u32 t, %0, %1;\n"
            " setp.lt.u32 h, %0, %1;\n add.u32 t2, t, %6;\n selp.u32 t, t2, t, h;\n"
            " mul.hi.u32 q, %3, t;\n mul.lo.u32 r, %2, t;\n mad.lo.u32 r, q, %5, r;\n"
            " setp.ge.u32 k, r, %6;\n sub.u32 r2, r, %6;\n selp.u32 %1, r2, r, k;\n"
            " setp.ge.u32 g, u, %6;\n sub.u32 s2, u, %6;\n selp.u32 %0, s2, u, g;\n}"
            : "+r"(x), "+r"(y)
            : "r"(w), "r"(wq), "r"(p2), "r"(0u - p), "r"(p));
    }
    if (F == 9) {  // inverse lazy (Algorithm 4) with the PTX Shoup product
        const uint32_t a = umin(x, x - p2);
        const uint32_t t = shoup_ptx(y, w, wq, 0u - p);
        x = a + t;
        y = a - t + p2;
    }
}

template <int F>
__global__ void k_rate(uint32_t *out, int iters, uint32_t p, uint32_t w0, uint32_t wq0) {
    uint32_t x[8][4];
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 4; ++v) x[j][v] = (threadIdx.x * 37u + j * 11u + v) % p;
    uint32_t w[7], wq[7];
    for (int i = 0; i < 7; ++i) {
        w[i] = w0 + i;
        wq[i] = wq0 + i;
    }
    const uint32_t p2 = 2 * p;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int lb = 2; lb >= 0; --lb)
#pragma unroll
            for (int jl = 0; jl < (1 << lb); ++jl)
#pragma unroll
                for (int jh = 0; jh < 8; jh += (2 << lb))
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        bf<F>(x[jh + jl][v], x[jh + jl + (1 << lb)][v], w[(1 << lb) - 1 + jl], wq[(1 << lb) - 1 + jl],
                              p, p2);
    }
    uint32_t s = 0;
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 4; ++v) s ^= x[j][v];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// OP 0: mul.hi.u32; 1: mad.lo.u32; 2: the 64-bit product of two 32-bit
// words (both halves used, one add to fold them).
template <int OP>
__global__ void k_mul(uint32_t *out, int iters, uint32_t seed) {
    uint32_t a[8], b = seed * 2654435761u + threadIdx.x;
    for (int i = 0; i < 8; ++i) a[i] = b + i * 977u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == 0) a[i] = __umulhi(a[i], b) ^ i;
            if (OP == 1) a[i] = a[i] * b + 0x9E3779B9u;
            if (OP == 2) {
                const uint64_t r = (uint64_t)a[i] * b;
                a[i] = (uint32_t)(r >> 32) + (uint32_t)r;
            }
        }
    }
    uint32_t s = 0;
    for (int i = 0; i < 8; ++i) s ^= a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 64-bit words: the lazy forward butterfly and the raw 64-bit multiplies
// (mul.hi.u64 and mul.lo.u64, each built by the compiler from 32-bit
// multiplies on this GPU).
__global__ void k_rate64(uint64_t *out, int iters, uint64_t p, uint64_t w0, uint64_t wq0) {
    uint64_t x[8][2];
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 2; ++v) x[j][v] = (threadIdx.x * 37ull + j * 11ull + v) % p;
    uint64_t w[7], wq[7];
    for (int i = 0; i < 7; ++i) {
        w[i] = w0 + i;
        wq[i] = wq0 + i;
    }
    const uint64_t p2 = 2 * p;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int lb = 2; lb >= 0; --lb)
#pragma unroll
            for (int jl = 0; jl < (1 << lb); ++jl)
#pragma unroll
                for (int jh = 0; jh < 8; jh += (2 << lb))
#pragma unroll
                    for (int v = 0; v < 2; ++v)
                        bfly_fwd_lazy(x[jh + jl][v], x[jh + jl + (1 << lb)][v], w[(1 << lb) - 1 + jl],
                                      wq[(1 << lb) - 1 + jl], p, p2);
    }
    uint64_t s = 0;
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 2; ++v) s ^= x[j][v];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// High word of a 64 x 64-bit product without the low partial products: a1 b1 +
// hi(a1 b0) + hi(a0 b1), at most 2 below the exact high word.
__device__ __forceinline__ uint64_t mulhi64_trunc(uint64_t a, uint64_t b) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    return (uint64_t)a1 * b1 + __umulhi(a1, b0) + __umulhi(a0, b1);
}

// Algorithm 3 at 64 bits with the truncated quotient: Q' in [Q - 2, Q], so
// W T - Q' p lies in [0, 4p) (p < beta/4) and one subtraction of 2p returns it
// to [0, 2p).
__global__ void k_rate64_trunc(uint64_t *out, int iters, uint64_t p, uint64_t w0, uint64_t wq0) {
    uint64_t x[8][2];
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 2; ++v) x[j][v] = (threadIdx.x * 37ull + j * 11ull + v) % p;
    uint64_t w[7], wq[7];
    for (int i = 0; i < 7; ++i) {
        w[i] = w0 + i;
        wq[i] = wq0 + i;
    }
    const uint64_t p2 = 2 * p;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int lb = 2; lb >= 0; --lb)
#pragma unroll
            for (int jl = 0; jl < (1 << lb); ++jl)
#pragma unroll
                for (int jh = 0; jh < 8; jh += (2 << lb))
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        uint64_t &xx = x[jh + jl][v], &yy = x[jh + jl + (1 << lb)][v];
                        const uint64_t s = umin(xx + yy, xx + yy - p2);
                        const uint64_t t = xx - yy + p2;
                        const uint64_t q = mulhi64_trunc(wq[(1 << lb) - 1 + jl], t);
                        const uint64_t r = w[(1 << lb) - 1 + jl] * t - q * p;
                        yy = umin(r, r - p2);
                        xx = s;
                    }
    }
    uint64_t s = 0;
    for (int j = 0; j < 8; ++j)
        for (int v = 0; v < 2; ++v) s ^= x[j][v];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
__global__ void k_mul64(uint64_t *out, int iters, uint64_t seed) {
    uint64_t a[8], b = seed * 0x9E3779B97F4A7C15ull + threadIdx.x;
    for (int i = 0; i < 8; ++i) a[i] = b + i * 977ull;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
            a[i] = OP == 0 ? __umul64hi(a[i], b) ^ i : OP == 2 ? mulhi64_trunc(a[i], b) ^ i : a[i] * b + 0x9E3779B97F4A7C15ull;
    }
    uint64_t s = 0;
    for (int i = 0; i < 8; ++i) s ^= a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename K, typename... A>
static double timed(K k, int grid, int block, A... args) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k<<<grid, block>>>(args...);
    cudaEventRecord(e0);
    k<<<grid, block>>>(args...);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

int main() {
    int dev = 0, sms = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    const int grid = sms * 4, block = 256, iters = 256;
    uint32_t *out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * block * sizeof(uint32_t)) != cudaSuccess) return 1;
    const uint32_t p = 998244353u, w0 = 12345u, wq0 = (uint32_t)(((uint64_t)w0 << 32) / p);
    const double clk = clk_khz * 1e3, bf = 48.0 * iters * (double)grid * block;
    const char *names[17] = {"lazy_fwd", "ntl_fwd", "lazy_inv", "ntl_inv", "lazy_fwd_w1", "lazy_fwd_ptx",
                             "lazy_fwd_ptx_sel", "lazy_fwd_ptx_sign", "ntl_fwd_ptx", "lazy_inv_ptx",
                             "lazy_fwd_asm_min", "lazy_fwd_asm_sel", "lazy_fwd_asm_min2", "lazy_fwd_asm_subqp",
                             "lazy_inv_asm_min", "lazy_inv_asm_sel", "ntl_fwd_asm_sel"};
    double ms[17];
    ms[0] = timed(k_rate<0>, grid, block, out, iters, p, w0, wq0);
    ms[1] = timed(k_rate<1>, grid, block, out, iters, p, w0, wq0);
    ms[2] = timed(k_rate<2>, grid, block, out, iters, p, w0, wq0);
    ms[3] = timed(k_rate<3>, grid, block, out, iters, p, w0, wq0);
    ms[4] = timed(k_rate<4>, grid, block, out, iters, p, w0, wq0);
    ms[5] = timed(k_rate<5>, grid, block, out, iters, p, w0, wq0);
    ms[6] = timed(k_rate<6>, grid, block, out, iters, p, w0, wq0);
    ms[7] = timed(k_rate<7>, grid, block, out, iters, p, w0, wq0);
    ms[8] = timed(k_rate<8>, grid, block, out, iters, p, w0, wq0);
    ms[9] = timed(k_rate<9>, grid, block, out, iters, p, w0, wq0);
    ms[10] = timed(k_rate<10>, grid, block, out, iters, p, w0, wq0);
    ms[11] = timed(k_rate<11>, grid, block, out, iters, p, w0, wq0);
    ms[12] = timed(k_rate<12>, grid, block, out, iters, p, w0, wq0);
    ms[13] = timed(k_rate<13>, grid, block, out, iters, p, w0, wq0);
    ms[14] = timed(k_rate<14>, grid, block, out, iters, p, w0, wq0);
    ms[15] = timed(k_rate<15>, grid, block, out, iters, p, w0, wq0);
    ms[16] = timed(k_rate<16>, grid, block, out, iters, p, w0, wq0);
    printf("{\"sms\": %d, \"max_clock_mhz\": %.0f", sms, clk / 1e6);
    for (int i = 0; i < 17; ++i)
        printf(", \"%s_bfly_per_clk_sm\": %.3f", names[i], bf / (ms[i] * 1e-3) / clk / sms);
    const double mops = 8.0 * 4096 * (double)grid * block;
    const double t_hi = timed(k_mul<0>, grid, block, out, 4096, 1u), t_lo = timed(k_mul<1>, grid, block, out, 4096, 1u);
    const double t_wide = timed(k_mul<2>, grid, block, out, 4096, 1u);
    printf(", \"mulhi_per_clk_sm\": %.2f, \"madlo_per_clk_sm\": %.2f, \"mulwide_plus_add_per_clk_sm\": %.2f",
           mops / (t_hi * 1e-3) / clk / sms, mops / (t_lo * 1e-3) / clk / sms, mops / (t_wide * 1e-3) / clk / sms);
    uint64_t *out64 = nullptr;
    if (cudaMalloc(&out64, (size_t)grid * block * sizeof(uint64_t)) == cudaSuccess) {
        const uint64_t p64 = 2305843009448574977ull, w64 = 1234567ull;
        const uint64_t wq64 = (uint64_t)(((unsigned __int128)w64 << 64) / p64);
        const double bf64 = 24.0 * iters * (double)grid * block;
        const double t64 = timed(k_rate64, grid, block, out64, iters, p64, w64, wq64);
        const double mops64 = 8.0 * 1024 * (double)grid * block;
        const double h64 = timed(k_mul64<0>, grid, block, out64, 1024, (uint64_t)1);
        const double l64 = timed(k_mul64<1>, grid, block, out64, 1024, (uint64_t)1);
        const double ht64 = timed(k_mul64<2>, grid, block, out64, 1024, (uint64_t)1);
        const double tt64 = timed(k_rate64_trunc, grid, block, out64, iters, p64, w64, wq64);
        printf(", \"lazy_fwd_u64_bfly_per_clk_sm\": %.3f, \"mulhi_u64_per_clk_sm\": %.2f, \"mullo_u64_per_clk_sm\": %.2f",
               bf64 / (t64 * 1e-3) / clk / sms, mops64 / (h64 * 1e-3) / clk / sms, mops64 / (l64 * 1e-3) / clk / sms);
        printf(", \"mulhi_u64_trunc_per_clk_sm\": %.2f, \"lazy_fwd_u64_trunc_bfly_per_clk_sm\": %.3f",
               mops64 / (ht64 * 1e-3) / clk / sms, bf64 / (tt64 * 1e-3) / clk / sms);
        cudaFree(out64);
    }
    printf(", \"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
    cudaFree(out);
    return 0;
}
