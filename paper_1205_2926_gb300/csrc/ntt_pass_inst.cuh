// ntt_pass_inst.cuh -- instantiation and launch of the pass kernels for one
// word type; included by ntt_pass_u32.cu and ntt_pass_u64.cu so that the two
// word types compile in parallel.
#pragma once

#include <algorithm>
#include <mutex>

#include "ntt_internal.hpp"
#include "ntt_kernels.cuh"
#include "ntt_warp.cuh"

namespace ntt {

template <typename W>
static PassArgs<W> to_args(const LaunchSpec &s) {
    PassArgs<W> a;
    a.data = static_cast<W *>(s.data);
    a.stride = s.stride;
    a.batch = s.batch;
    a.logL = s.logL;
    a.logS = s.logS;
    a.logTV = s.logTV;
    a.logTA = s.logTA;
    a.per_cta = s.per_cta;
    a.ntiles = s.ntiles;
    a.buf_chunks = s.buf_chunks;
    a.flags = s.flags;
    a.tw = static_cast<const W *>(s.tw);
    a.ma = static_cast<const W *>(s.ma);
    a.mb = static_cast<const W *>(s.mb);
    a.p = (W)s.p;
    a.J = (W)s.J;
    a.nrows = s.nrows;
    a.rowptrs = nullptr;
    a.status = s.status;
    a.wait_budget = s.wait_budget;
    a.tx_extra = s.tx_extra;
    return a;
}

// Per kernel: shared-memory opt-in once per device, and the number of CTAs
// that fit on one SM for the launch's shared-memory size (cached).  The
// caches are per kernel instantiation (template arguments), not per
// function type, which every k_pass of one word type shares.  smem == 0:
// the opt-in only (no launch has an empty shared-memory buffer).
template <typename W, int DIR, int VAR, int LOGR, bool ROW>
static cudaError_t kernel_slots(size_t smem, int *per_sm, int *sms) {
    auto kern = k_pass<W, DIR, VAR, LOGR, ROW>;
    constexpr int kSizes = 8;  // shared-memory sizes remembered per device (round robin)
    static std::mutex mu;
    static int configured[64] = {0};
    static int cache_sms[64], cache_occ[64][kSizes], cache_next[64];
    static size_t cache_smem[64][kSizes];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        cudaDeviceGetAttribute(&cache_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        for (int i = 0; i < kSizes; ++i) cache_smem[dev][i] = (size_t)-1;
        configured[dev] = 1;
    }
    if (smem == 0) return cudaSuccess;
    *sms = cache_sms[dev];
    for (int i = 0; i < kSizes; ++i)
        if (cache_smem[dev][i] == smem) {
            *per_sm = cache_occ[dev][i];
            return cudaSuccess;
        }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int slot = cache_next[dev]++ % kSizes;
    cache_smem[dev][slot] = smem;
    cache_occ[dev][slot] = std::max(occ, 1);
    *per_sm = cache_occ[dev][slot];
    return cudaSuccess;
}

// Persistent grid: no more CTAs than fit on the device at once.
template <typename W, int DIR, int VAR, int LOGR, bool ROW>
static cudaError_t launch_k(const LaunchSpec &s, cudaStream_t st) {
    auto kern = k_pass<W, DIR, VAR, LOGR, ROW>;
    int per_sm = 1, sms = 1;
    cudaError_t e = kernel_slots<W, DIR, VAR, LOGR, ROW>(s.smem, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    const uint64_t slots = (uint64_t)per_sm * sms;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(s.ntiles, slots));
    kern<<<grid, kThreads, s.smem, st>>>(to_args<W>(s), s.map);
    return cudaGetLastError();
}

template <typename W, int DIR, int VAR, bool ROW, int LO, int HI>
static cudaError_t launch_logr(const LaunchSpec &s, int logR, cudaStream_t st) {
    if (logR == LO) return launch_k<W, DIR, VAR, LO, ROW>(s, st);
    if constexpr (LO < HI) return launch_logr<W, DIR, VAR, ROW, LO + 1, HI>(s, logR, st);
    return cudaErrorInvalidValue;
}

// Row pass with one warp per row (kind 3, 2^5 <= R <= 2^10): eight warps per
// CTA, each owning G consecutive rows at a time, a grid-stride loop over the
// groups, shared memory for the warps' transposes.
template <typename W, int DIR, int VAR, int LOGR, int G>
static cudaError_t launch_warp_rows(const LaunchSpec &s, cudaStream_t st) {
    auto kern = k_warp_row<W, DIR, VAR, LOGR, G>;
    const size_t smem = (size_t)kWarpRowsPerCta * G * ((1u << LOGR) + (1u << LOGR) / 32) * sizeof(W);
    static int configured[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    const uint64_t groups = (s.nrows + G - 1) / G;
    const uint64_t ctas = (groups + kWarpRowsPerCta - 1) / kWarpRowsPerCta;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ctas, 152ull * 16));
    kern<<<grid, kWarpRowsPerCta * 32, smem, st>>>(to_args<W>(s));
    return cudaGetLastError();
}

// Several rows per warp once there are enough rows for two CTAs of such
// groups per SM; one row per warp for short launches, whose time is the
// length of one warp's chain.
template <typename W, int DIR, int VAR, int LO, int HI>
static cudaError_t launch_warp_logr(const LaunchSpec &s, cudaStream_t st) {
    if (s.logR == LO) {
        constexpr int G = WarpGroup<W, LO>::G;
        if constexpr (G > 1) {
            if (s.nrows >= (uint64_t)G * kWarpRowsPerCta * 152 * 2) return launch_warp_rows<W, DIR, VAR, LO, G>(s, st);
        }
        return launch_warp_rows<W, DIR, VAR, LO, 1>(s, st);
    }
    if constexpr (LO < HI) return launch_warp_logr<W, DIR, VAR, LO + 1, HI>(s, st);
    return cudaErrorInvalidValue;
}

// Load (and configure) every pass kernel of one (word, direction, variant)
// without launching it: under CUDA's lazy module loading a kernel is
// otherwise loaded at its first launch.
template <typename W, int DIR, int VAR, bool ROW, int LO, int HI>
static cudaError_t preload_logr() {
    int per_sm = 1, sms = 1;
    cudaError_t e = kernel_slots<W, DIR, VAR, LO, ROW>(0, &per_sm, &sms);
    if (e != cudaSuccess) return e;
    if constexpr (LO < HI) return preload_logr<W, DIR, VAR, ROW, LO + 1, HI>();
    return cudaSuccess;
}

template <typename W, int DIR, int VAR>
static cudaError_t launch_kind(const LaunchSpec &s, int kind, cudaStream_t st) {
    if (kind == KIND_PRELOAD) {
        cudaError_t e = preload_logr<W, DIR, VAR, false, 3, kMaxColLog>();
        if (e == cudaSuccess) e = preload_logr<W, DIR, VAR, true, 3, kMaxRowLog>();
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_tiny<W, DIR, VAR>);
        return e;
    }
    if (kind == 3) return launch_warp_logr<W, DIR, VAR, 5, 10>(s, st);
    if (kind == 0) return launch_logr<W, DIR, VAR, false, 3, kMaxColLog>(s, s.logR, st);
    if (kind == 1) return launch_logr<W, DIR, VAR, true, 3, kMaxRowLog>(s, s.logR, st);
    k_tiny<W, DIR, VAR><<<s.grid, 128, 0, st>>>(to_args<W>(s));
    return cudaGetLastError();
}

// One (word type, direction, variant) per translation unit
// (ntt_pass_<word>_<dir>_<variant>.cu), so that the instantiations compile in
// parallel; ntt_pass_u32.cu / ntt_pass_u64.cu dispatch to them.

}  // namespace ntt
