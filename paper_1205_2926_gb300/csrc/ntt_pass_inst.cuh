// ntt_pass_inst.cuh -- instantiation and launch of the pass kernels for one
// word type; included by ntt_pass_u32.cu and ntt_pass_u64.cu so that the two
// word types compile in parallel.
#pragma once

#include "ntt_internal.hpp"
#include "ntt_kernels.cuh"

namespace ntt {

template <typename W>
static PassArgs<W> to_args(const LaunchSpec &s) {
    PassArgs<W> a;
    a.data = static_cast<W *>(s.data);
    a.stride = s.stride;
    a.batch = s.batch;
    a.logL = s.logL;
    a.logR = s.logR;
    a.logS = s.logS;
    a.per_cta = s.per_cta;
    a.logTV = s.logTV;
    a.logTA = s.logTA;
    a.flags = s.flags;
    a.tw = static_cast<const W *>(s.tw);
    a.ma = static_cast<const W *>(s.ma);
    a.mb = static_cast<const W *>(s.mb);
    a.p = (W)s.p;
    a.nrows = s.nrows;
    a.rowptrs = nullptr;
    return a;
}

template <typename W, int DIR, int VAR, bool ROW>
static cudaError_t launch_one(const LaunchSpec &s, cudaStream_t st) {
    auto kern = k_pass<W, DIR, VAR, ROW>;
    // Opt in to large dynamic shared memory once per device and kernel.
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    kern<<<s.grid, kThreads, s.smem, st>>>(to_args<W>(s));
    return cudaGetLastError();
}

template <typename W, int DIR, int VAR>
static cudaError_t launch_kind(const LaunchSpec &s, int kind, cudaStream_t st) {
    if (kind == 0) return launch_one<W, DIR, VAR, false>(s, st);
    if (kind == 1) return launch_one<W, DIR, VAR, true>(s, st);
    k_tiny<W, DIR, VAR><<<s.grid, 128, 0, st>>>(to_args<W>(s));
    return cudaGetLastError();
}

template <typename W>
static cudaError_t launch_pass_t(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st) {
    if (dir == DIR_FWD)
        return var == VAR_LAZY ? launch_kind<W, DIR_FWD, VAR_LAZY>(s, kind, st)
                               : launch_kind<W, DIR_FWD, VAR_NTL>(s, kind, st);
    return var == VAR_LAZY ? launch_kind<W, DIR_INV, VAR_LAZY>(s, kind, st)
                           : launch_kind<W, DIR_INV, VAR_NTL>(s, kind, st);
}

}  // namespace ntt
