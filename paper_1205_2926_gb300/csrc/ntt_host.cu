// ntt_host.cu -- transforms of batches that live in host memory.
//
// The batch is cut into chunks of whole transforms; chunk i is copied in on
// the plan's copy-in stream, transformed on the caller's stream once its copy
// has landed, and copied out on the copy-out stream once its transform is
// done.  Copies of later chunks therefore overlap the transforms and the
// copy-out of earlier ones (both copy directions run at once on the
// host-device link).  A single transform, or a batch under the chunk size,
// goes through one copy-in, transform, copy-out sequence on the caller's
// stream.  The device copy of the batch is owned by the plan and grows on
// demand; the call returns after the caller's stream has finished.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ntt_internal.hpp"

namespace ntt {

constexpr int kHostChunksMax = 16;             // copy/transform chunks per call
constexpr size_t kHostChunkBytes = 2u << 20;   // aim for chunks of about this size

static int ensure_pipeline(ntt_plan_s *pl) {
    if (pl->hs_in) return NTT_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&pl->hs_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->hs_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->hev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->hev_end, cudaEventDisableTiming);
    for (int i = 0; i < kHostChunksMax && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&pl->hev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->hev_done[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release_host_pipeline(pl);
        return cuda_fail(e, "host pipeline streams");
    }
    return NTT_OK;
}

void release_host_pipeline(ntt_plan_s *pl) {
    if (pl->stage) cudaFree(pl->stage);
    pl->stage = nullptr;
    pl->stage_bytes = 0;
    if (pl->hs_in) cudaStreamDestroy(pl->hs_in);
    if (pl->hs_out) cudaStreamDestroy(pl->hs_out);
    pl->hs_in = pl->hs_out = nullptr;
    if (pl->hev_start) cudaEventDestroy(pl->hev_start);
    if (pl->hev_end) cudaEventDestroy(pl->hev_end);
    pl->hev_start = pl->hev_end = nullptr;
    for (int i = 0; i < kHostChunksMax; ++i) {
        if (pl->hev_in[i]) cudaEventDestroy(pl->hev_in[i]);
        if (pl->hev_done[i]) cudaEventDestroy(pl->hev_done[i]);
        pl->hev_in[i] = pl->hev_done[i] = nullptr;
    }
}

}  // namespace ntt

using namespace ntt;

extern "C" int ntt_transform_host(ntt_plan_t pl, int inverse, void *h_data, size_t batch, size_t stride_words,
                                  void *stream) {
    if (!pl || !h_data || batch == 0 || (inverse != 0 && inverse != 1)) return NTT_ERR_ARG;
    if (stride_words < pl->L || ((stride_words * pl->wbytes) & 15)) return NTT_ERR_ALIGN;
    std::lock_guard<std::mutex> lk(pl->mu);
    const size_t per = stride_words * pl->wbytes;  // bytes per transform
    const size_t bytes = batch * per;
    cudaStream_t st = (cudaStream_t)stream;
    if (pl->stage_bytes < bytes) {
        if (pl->stage) {
            cudaStreamSynchronize(st);
            cudaFree(pl->stage);
        }
        pl->stage = nullptr;
        pl->stage_bytes = 0;
        cudaError_t e = cudaMalloc(&pl->stage, bytes);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "cudaMalloc");
        pl->stage_bytes = bytes;
    }
    char *dev = static_cast<char *>(pl->stage);
    char *host = static_cast<char *>(h_data);
    const size_t nc = std::min<size_t>({batch, (size_t)kHostChunksMax, std::max<size_t>(1, bytes / kHostChunkBytes)});
    cudaError_t e;
    if (nc <= 1) {
        e = cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "H2D");
        int rc = enqueue_transform(pl, inverse, dev, batch, stride_words, st);
        if (rc) return rc;
        e = cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "D2H");
    } else {
        int rc = ensure_pipeline(pl);
        if (rc) return rc;
        // work already queued on the caller's stream comes first
        e = cudaEventRecord(pl->hev_start, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->hs_in, pl->hev_start, 0);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline start");
        for (size_t i = 0; i < nc; ++i) {
            const size_t b0 = i * batch / nc, b1 = (i + 1) * batch / nc;
            const size_t off = b0 * per, n = (b1 - b0) * per;
            e = cudaMemcpyAsync(dev + off, host + off, n, cudaMemcpyHostToDevice, pl->hs_in);
            if (e == cudaSuccess) e = cudaEventRecord(pl->hev_in[i], pl->hs_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, pl->hev_in[i], 0);
            if (e != cudaSuccess) return cuda_fail(e, "H2D chunk");
            rc = enqueue_transform(pl, inverse, dev + off, b1 - b0, stride_words, st);
            if (rc) return rc;
            e = cudaEventRecord(pl->hev_done[i], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(pl->hs_out, pl->hev_done[i], 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(host + off, dev + off, n, cudaMemcpyDeviceToHost, pl->hs_out);
            if (e != cudaSuccess) return cuda_fail(e, "D2H chunk");
        }
        e = cudaEventRecord(pl->hev_end, pl->hs_out);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, pl->hev_end, 0);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline end");
    }
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "sync");
}
