// ntt_server.cu -- continuous-batching server for polynomial products mod p
// (the application of Section 1 of Harvey, arXiv:1205.2926, under load).
//
// A scheduler thread owns the GPU work.  Submitted requests wait in a FIFO
// queue; the scheduler admits them in order while their device memory fits
// in the budget, groups the admitted ones by transform length L, and runs
// each group as one batch on the CUDA stream with the least outstanding work
// (butterflies of the batches still running on it), so that small requests
// do not queue behind a large one:
//   gather the operands into a zero-padded slab, forward transforms (2n
//   vectors), pointwise product times L^-1, inverse transforms (n vectors),
//   scatter the na+nb-1 result words of each request to its host buffer.
// Operands and results in page-locked host memory are read and written by
// the gather and scatter kernels themselves (the device reaches them
// through unified addressing), so a batch costs a fixed handful of CUDA
// calls whatever its size; other host memory goes through one copy per
// operand and result.  The scheduler releases the server lock while it
// issues a batch, so submitters never wait for the launches.
// Requests that arrive while batches are on the GPU are admitted as soon as
// memory frees up, into new batches on other streams, so their work overlaps
// with the running ones.  Plans and twiddle tables stay resident on the
// device (one cached plan per (p, L)).  A batch is the same arithmetic as a
// lone polymul_mod_p call, so each result is identical alone or in a mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "modarith.cuh"
#include "ntt_internal.hpp"
#include "ntt_polymul.hpp"

namespace ntt {

template <typename W>
__global__ void k_pointwise_batch(W *__restrict__ A, const W *__restrict__ B, uint64_t n, W p, W J, W K, W Kq) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        W y = mont_mul(A[i], B[i], J, p);
        // fully reduced: the inverse transform's input interval is [0, p)
        // for the fully reduced butterflies (Algorithm 2)
        A[i] = csub(shoup_mul(y, K, Kq, p), p);
    }
}

// Gather / scatter between the host buffers of up to kGather requests and
// the slab: blockIdx.y is the request, blockIdx.z the operand (gather).
constexpr int kGather = 32;
struct GatherTable {
    const void *a[kGather];
    const void *b[kGather];
    void *c[kGather];
    uint32_t na[kGather], nb[kGather];
};

template <typename W>
__global__ void k_gather(const GatherTable t, W *__restrict__ slab, uint64_t L, uint64_t row_a, uint64_t row_b) {
    const int r = blockIdx.y;
    const bool second = blockIdx.z != 0;
    const W *__restrict__ src = static_cast<const W *>(second ? t.b[r] : t.a[r]);
    const uint64_t cnt = second ? t.nb[r] : t.na[r];
    W *__restrict__ dst = slab + ((second ? row_b : row_a) + r) * L;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < L; j += (uint64_t)gridDim.x * blockDim.x)
        dst[j] = j < cnt ? src[j] : (W)0;
}

template <typename W>
__global__ void k_scatter(const GatherTable t, const W *__restrict__ slab, uint64_t L, uint64_t row0) {
    const int r = blockIdx.y;
    const uint64_t cnt = (uint64_t)t.na[r] + t.nb[r] - 1;
    const W *__restrict__ src = slab + (row0 + r) * L;
    W *__restrict__ dst = static_cast<W *>(t.c[r]);
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (uint64_t)gridDim.x * blockDim.x)
        dst[j] = src[j];
}

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id;
    const void *a, *b;
    void *c;
    const void *da = nullptr, *db = nullptr;  // device views of page-locked operands (else null)
    void *dc = nullptr;                       // device view of a page-locked result buffer (else null)
    size_t na, nb;
    uint64_t L;
    Clock::time_point t_submit, t_done;
    int status;  // NTT_ERR_PENDING while queued or running
};

struct Batch {
    std::vector<uint64_t> ids;
    ntt_plan_s *plan = nullptr;
    void *slab = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    int stream = 0;
    int status = NTT_OK;
    double work = 0;  // butterflies of the batch (stream load balancing)
    bool direct = false;  // operands gathered and results scattered by kernels
};

}  // namespace ntt

struct ntt_server_s {
    ntt_server_config_t cfg;
    int device = 0;
    size_t wbytes = 4;
    std::vector<cudaStream_t> streams;
    std::vector<double> stream_work;  // outstanding butterflies per stream
    cudaMemPool_t pool = nullptr;     // the server's own stream-ordered pool
    int next_stream = 0;              // where the next tie-break starts
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, ntt::Request> reqs;
    std::vector<ntt::Batch> inflight;
    size_t inflight_bytes = 0;
    int launching = 0;  // batches being issued with the lock released
    uint64_t next_id = 1;
    bool stop = false;
    int fail_next = 0;
    // statistics
    std::vector<double> lat_us;
    uint64_t n_done = 0, n_refused = 0, n_cancelled = 0, n_failed = 0, n_batches = 0, n_direct = 0;
    double butterflies = 0;
    ntt::Clock::time_point t_first, t_last;
    bool any = false;
    std::thread worker;
};

namespace ntt {

static uint64_t bfly_count(uint64_t L) {
    uint64_t l = 0;
    while ((1ull << l) < L) ++l;
    return 3 * l * (L / 2);  // two forward transforms and one inverse
}

// Launch one batch (scheduler thread, server lock released).
template <typename W>
static int launch_batch_t(ntt_server_s *sv, Batch &bt, const std::vector<Request *> &rs, cudaStream_t st) {
    ntt_plan_s *pl = bt.plan;
    const uint64_t L = pl->L, n = rs.size();
    const size_t wb = sizeof(W);
    cudaError_t e = cudaMallocFromPoolAsync(&bt.slab, bt.bytes, sv->pool, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "server slab");
    W *slab = (W *)bt.slab;
    bool direct = true;  // every operand and result buffer reachable from the device
    for (const Request *r : rs) direct = direct && r->da && r->db && r->dc;
    bt.direct = direct;
    const unsigned gx = (unsigned)std::min<uint64_t>((L + 255) / 256, 64);
    if (direct) {
        for (uint64_t i0 = 0; i0 < n; i0 += kGather) {
            const int m = (int)std::min<uint64_t>(kGather, n - i0);
            GatherTable t;
            for (int j = 0; j < m; ++j) {
                t.a[j] = rs[i0 + j]->da;
                t.b[j] = rs[i0 + j]->db;
                t.c[j] = rs[i0 + j]->dc;
                t.na[j] = (uint32_t)rs[i0 + j]->na;
                t.nb[j] = (uint32_t)rs[i0 + j]->nb;
            }
            k_gather<W><<<dim3(gx, m, 2), 256, 0, st>>>(t, slab, L, i0, n + i0);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "server gather");
    } else {
        e = cudaMemsetAsync(slab, 0, bt.bytes, st);
        if (e != cudaSuccess) return cuda_fail(e, "server memset");
        for (uint64_t i = 0; i < n; ++i) {
            e = cudaMemcpyAsync(slab + i * L, rs[i]->a, rs[i]->na * wb, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slab + (n + i) * L, rs[i]->b, rs[i]->nb * wb, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "server H2D");
        }
    }
    int rc = enqueue_transform(pl, 0, slab, 2 * n, L, st);
    if (rc) return rc;
    const int bits = pl->wbytes * 8;
    uint64_t J = 1;
    for (int i = 0; i < 7; ++i) J *= 2 - pl->p * J;
    const uint64_t K = (uint64_t)(((unsigned __int128)pl->L_inv << bits) % pl->p);
    const uint64_t Kq = nt::shoup_quotient(K, pl->p, bits);
    const uint64_t total = n * L;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 152 * 16);
    k_pointwise_batch<W><<<grid, 256, 0, st>>>(slab, slab + total, total, (W)pl->p, (W)J, (W)K, (W)Kq);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "server pointwise");
    rc = enqueue_transform(pl, 1, slab, n, L, st);
    if (rc) return rc;
    if (direct) {
        for (uint64_t i0 = 0; i0 < n; i0 += kGather) {
            const int m = (int)std::min<uint64_t>(kGather, n - i0);
            GatherTable t;
            for (int j = 0; j < m; ++j) {
                t.a[j] = rs[i0 + j]->da;
                t.b[j] = rs[i0 + j]->db;
                t.c[j] = rs[i0 + j]->dc;
                t.na[j] = (uint32_t)rs[i0 + j]->na;
                t.nb[j] = (uint32_t)rs[i0 + j]->nb;
            }
            k_scatter<W><<<dim3(gx, m, 1), 256, 0, st>>>(t, slab, L, i0);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "server scatter");
    } else {
        for (uint64_t i = 0; i < n; ++i) {
            e = cudaMemcpyAsync(rs[i]->c, slab + i * L, (rs[i]->na + rs[i]->nb - 1) * wb, cudaMemcpyDeviceToHost,
                                st);
            if (e != cudaSuccess) return cuda_fail(e, "server D2H");
        }
    }
    e = cudaFreeAsync(bt.slab, st);
    bt.slab = nullptr;
    if (e != cudaSuccess) return cuda_fail(e, "server free");
    e = cudaEventRecord(bt.done, st);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "server event");
}

static void finish_request(ntt_server_s *sv, Request &r, int status) {
    r.status = status;
    r.t_done = Clock::now();
    if (status == NTT_OK) {
        sv->n_done++;
        sv->lat_us.push_back(std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count());
        sv->butterflies += (double)bfly_count(r.L);
        sv->t_last = r.t_done;
    } else if (status == NTT_ERR_FAILED) {
        sv->n_failed++;
    }
}

static void scheduler(ntt_server_s *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        // 1. completions (batches on one stream finish in order: once one
        //    is still running, the later ones on its stream are not queried)
        bool progressed = false;
        uint64_t busy = 0;  // streams with a batch still running (bit per stream)
        for (size_t i = 0; i < sv->inflight.size();) {
            Batch &bt = sv->inflight[i];
            if (busy >> bt.stream & 1) {
                ++i;
                continue;
            }
            cudaError_t q = cudaEventQuery(bt.done);
            if (q == cudaErrorNotReady) {
                busy |= 1ull << bt.stream;
                ++i;
                continue;
            }
            const int st = (q == cudaSuccess && bt.status == NTT_OK) ? NTT_OK : NTT_ERR_FAILED;
            if (q != cudaSuccess && q != cudaErrorNotReady) cudaGetLastError();
            for (uint64_t id : bt.ids) finish_request(sv, sv->reqs[id], st);
            sv->inflight_bytes -= bt.bytes;
            sv->stream_work[bt.stream] -= bt.work;
            cudaEventDestroy(bt.done);
            sv->inflight.erase(sv->inflight.begin() + i);
            progressed = true;
        }
        if (progressed) sv->done_cv.notify_all();
        if (sv->stop && sv->queue.empty() && sv->inflight.empty()) break;  // (launching is 0 here)
        // 2. admission in FIFO order while memory allows
        std::map<uint64_t, std::vector<uint64_t>> by_len;
        size_t admitted_bytes = 0;
        while (!sv->queue.empty()) {
            Request &r = sv->reqs[sv->queue.front()];
            const size_t need = 2 * r.L * sv->wbytes;
            if (sv->inflight_bytes + admitted_bytes + need > sv->cfg.mem_budget_bytes) break;
            auto &v = by_len[r.L];
            if ((int)v.size() >= sv->cfg.max_batch) break;
            v.push_back(r.id);
            admitted_bytes += need;
            sv->queue.pop_front();
        }
        // 3. launch one batch per length class
        for (auto &kv : by_len) {
            Batch bt;
            bt.ids = kv.second;
            bt.bytes = 2 * kv.first * sv->wbytes * bt.ids.size();
            bt.work = (double)bfly_count(kv.first) * (double)bt.ids.size();
            {
                // least outstanding work; ties go round-robin so that small
                // batches spread over the idle streams
                const int ns = (int)sv->streams.size();
                int best = sv->next_stream;
                for (int k = 1; k < ns; ++k) {
                    const int c = (sv->next_stream + k) % ns;
                    if (sv->stream_work[c] < sv->stream_work[best]) best = c;
                }
                bt.stream = best;
                sv->next_stream = (best + 1) % ns;
            }
            cudaEventCreateWithFlags(&bt.done, cudaEventDisableTiming);
            std::vector<Request *> rs;
            for (uint64_t id : bt.ids) rs.push_back(&sv->reqs[id]);
            int rc = polymul_plan(sv->cfg.p, kv.first, &bt.plan, sv->cfg.variant);
            if (rc == NTT_OK && sv->fail_next > 0) {
                sv->fail_next--;
                rc = NTT_ERR_FAILED;  // host-side failure injection
            }
            if (rc == NTT_OK) {
                // issue the batch without the lock: submitters go on queueing
                // meanwhile (admitted requests are neither cancelled nor
                // erased, and the request map keeps their addresses)
                cudaStream_t st = sv->streams[bt.stream];
                sv->launching++;
                lk.unlock();
                rc = sv->wbytes == 4 ? launch_batch_t<uint32_t>(sv, bt, rs, st) : launch_batch_t<uint64_t>(sv, bt, rs, st);
                lk.lock();
                sv->launching--;
            }
            if (rc != NTT_OK) {
                // this batch fails; the others are unaffected
                if (bt.slab) cudaFreeAsync(bt.slab, sv->streams[bt.stream]);
                cudaStreamSynchronize(sv->streams[bt.stream]);
                cudaGetLastError();
                for (Request *r : rs) finish_request(sv, *r, NTT_ERR_FAILED);
                cudaEventDestroy(bt.done);
                sv->done_cv.notify_all();
                continue;
            }
            sv->n_batches++;
            sv->n_direct += bt.direct ? 1 : 0;
            sv->inflight_bytes += bt.bytes;
            sv->stream_work[bt.stream] += bt.work;
            sv->inflight.push_back(bt);
        }
        // 4. wait for work: short sleeps while batches run (requests that
        //    arrive meanwhile are admitted together), block when idle
        if (!sv->inflight.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else if (sv->queue.empty() && !sv->stop) {
            sv->cv.wait(lk, [sv] { return sv->stop || !sv->queue.empty(); });
        } else if (!sv->queue.empty() && by_len.empty()) {
            // head of the queue cannot be admitted yet and nothing runs: it
            // can never fit (guarded at submit), so this is unreachable; yield
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

}  // namespace ntt

using namespace ntt;

extern "C" {

int ntt_server_create(const ntt_server_config_t *cfg, ntt_server_t *out) {
    if (!cfg || !out) return NTT_ERR_ARG;
    *out = nullptr;
    if (cfg->p < 3 || cfg->p >= (1ull << 62) || !nt::is_prime(cfg->p)) return NTT_ERR_MODULUS;
    if (cfg->max_coeffs == 0 || cfg->mem_budget_bytes == 0 || cfg->n_streams < 1 || cfg->n_streams > 64 ||
        cfg->max_batch < 1 || (cfg->variant != NTT_VARIANT_LAZY && cfg->variant != NTT_VARIANT_NTL))
        return NTT_ERR_ARG;
    uint64_t L = 0;
    int rc = polymul_validate(cfg->p, cfg->max_coeffs, cfg->max_coeffs, &L);
    if (rc) return rc;
    ntt_server_s *sv = new (std::nothrow) ntt_server_s();
    if (!sv) return NTT_ERR_NOMEM;
    sv->cfg = *cfg;
    sv->wbytes = cfg->p < (1ull << 30) ? 4 : 8;
    cudaGetDevice(&sv->device);
    for (int i = 0; i < cfg->n_streams; ++i) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return cuda_fail(e, "server stream");
        }
        sv->streams.push_back(s);
    }
    sv->stream_work.assign(sv->streams.size(), 0.0);
    {
        // slabs come from a pool of the server's own that keeps up to the
        // memory budget reserved between batches instead of returning it to
        // the driver at every synchronisation (remapping costs milliseconds)
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = sv->device;
        cudaError_t e = cudaMemPoolCreate(&sv->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = cfg->mem_budget_bytes;
            e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if (e != cudaSuccess) {
            if (sv->pool) cudaMemPoolDestroy(sv->pool);
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return cuda_fail(e, "server pool");
        }
    }
    {
        // map the pool's memory up front (the budget, at most 4 GiB): batches
        // then never wait for the pool to grow while requests are served
        void *p = nullptr;
        const size_t reserve = std::min<size_t>(cfg->mem_budget_bytes, (size_t)4 << 30);
        if (cudaMallocFromPoolAsync(&p, reserve, sv->pool, sv->streams[0]) == cudaSuccess) {
            cudaFreeAsync(p, sv->streams[0]);
            cudaStreamSynchronize(sv->streams[0]);
        }
        cudaGetLastError();  // a reservation that does not fit is not an error
    }
    // the plan (twiddle tables, and with them the pass kernels) of every
    // length class the server accepts, and the server's own kernels, made and
    // loaded now: a plan made while requests are served allocates and
    // uploads its tables and loads kernels, which stalls the batches in flight
    {
        cudaFuncAttributes fa;
        cudaError_t e = sv->wbytes == 4 ? cudaFuncGetAttributes(&fa, k_gather<uint32_t>) : cudaFuncGetAttributes(&fa, k_gather<uint64_t>);
        if (e == cudaSuccess)
            e = sv->wbytes == 4 ? cudaFuncGetAttributes(&fa, k_scatter<uint32_t>) : cudaFuncGetAttributes(&fa, k_scatter<uint64_t>);
        if (e == cudaSuccess)
            e = sv->wbytes == 4 ? cudaFuncGetAttributes(&fa, k_pointwise_batch<uint32_t>)
                                : cudaFuncGetAttributes(&fa, k_pointwise_batch<uint64_t>);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(sv->pool);
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return cuda_fail(e, "server kernels");
        }
    }
    for (uint64_t l = 2; l <= L; l <<= 1) {
        ntt_plan_s *pl = nullptr;
        rc = polymul_plan(cfg->p, l, &pl, cfg->variant);
        if (rc) {
            cudaMemPoolDestroy(sv->pool);
            for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
            delete sv;
            return rc;
        }
    }
    sv->worker = std::thread(scheduler, sv);
    *out = sv;
    return NTT_OK;
}

// Device view of a host buffer: page-locked (registered or cudaHostAlloc)
// memory is reachable from the server's device at attr.devicePointer; any
// other memory gives null (the batch then copies it).
static void *device_view(const void *p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return (at.device == device || at.device < 0) ? at.devicePointer : nullptr;
}

int ntt_server_submit(ntt_server_t sv, const void *h_a, size_t na, const void *h_b, size_t nb, void *h_c,
                      uint64_t *req_id) {
    if (!sv || !h_a || !h_b || !h_c || !req_id) return NTT_ERR_ARG;
    uint64_t L = 0;
    int rc = polymul_validate(sv->cfg.p, na, nb, &L);
    void *da = nullptr, *db = nullptr, *dc = nullptr;
    if (rc == NTT_OK) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != sv->device) cudaSetDevice(sv->device);
        da = device_view(h_a, sv->device);
        db = da ? device_view(h_b, sv->device) : nullptr;
        dc = db ? device_view(h_c, sv->device) : nullptr;
        if (cur >= 0 && cur != sv->device) cudaSetDevice(cur);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    Request r;
    r.da = da;
    r.db = db;
    r.dc = dc;
    r.id = sv->next_id++;
    r.a = h_a;
    r.b = h_b;
    r.c = h_c;
    r.na = na;
    r.nb = nb;
    r.L = L;
    r.t_submit = Clock::now();
    if (!sv->any) {
        sv->any = true;
        sv->t_first = r.t_submit;
    }
    *req_id = r.id;
    if (rc != NTT_OK || na > sv->cfg.max_coeffs || nb > sv->cfg.max_coeffs ||
        2 * L * sv->wbytes > sv->cfg.mem_budget_bytes) {
        r.status = NTT_ERR_REFUSED;
        sv->n_refused++;
        sv->reqs[r.id] = r;
        return NTT_ERR_REFUSED;
    }
    r.status = NTT_ERR_PENDING;
    sv->reqs[r.id] = r;
    sv->queue.push_back(r.id);
    sv->cv.notify_one();
    return NTT_OK;
}

int ntt_server_poll(ntt_server_t sv, uint64_t id, int *status) {
    if (!sv || !status) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return NTT_ERR_ARG;
    *status = it->second.status;
    return NTT_OK;
}

int ntt_server_wait(ntt_server_t sv, uint64_t id, int timeout_ms, int *status) {
    if (!sv || !status) return NTT_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return NTT_ERR_ARG;
    auto ready = [&] { return sv->reqs[id].status != NTT_ERR_PENDING; };
    if (timeout_ms < 0)
        sv->done_cv.wait(lk, ready);
    else
        sv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    *status = sv->reqs[id].status;
    return NTT_OK;
}

int ntt_server_cancel(ntt_server_t sv, uint64_t id) {
    if (!sv) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(id);
    if (it == sv->reqs.end()) return NTT_ERR_ARG;
    auto q = std::find(sv->queue.begin(), sv->queue.end(), id);
    if (q == sv->queue.end()) return NTT_ERR_PENDING;  // already admitted or finished
    sv->queue.erase(q);
    it->second.status = NTT_ERR_CANCELLED;
    sv->n_cancelled++;
    sv->done_cv.notify_all();
    return NTT_OK;
}

int ntt_server_drain(ntt_server_t sv, int timeout_ms) {
    if (!sv) return NTT_ERR_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto idle = [sv] { return sv->queue.empty() && sv->inflight.empty() && sv->launching == 0; };
    if (timeout_ms < 0) {
        sv->done_cv.wait(lk, idle);
        return NTT_OK;
    }
    return sv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle) ? NTT_OK : NTT_ERR_PENDING;
}

int ntt_server_stats(ntt_server_t sv, ntt_server_stats_t *out) {
    if (!sv || !out) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->completed = sv->n_done;
    out->refused = sv->n_refused;
    out->cancelled = sv->n_cancelled;
    out->failed = sv->n_failed;
    out->batches = sv->n_batches;
    out->direct_batches = sv->n_direct;
    out->butterflies = sv->butterflies;
    std::vector<double> v = sv->lat_us;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double s = 0;
        for (double x : v) s += x;
        out->mean_us = s / v.size();
    }
    if (sv->any && sv->n_done) out->wall_s = std::chrono::duration<double>(sv->t_last - sv->t_first).count();
    return NTT_OK;
}

int ntt_server_reset_stats(ntt_server_t sv) {
    if (!sv) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat_us.clear();
    sv->n_done = sv->n_refused = sv->n_cancelled = sv->n_failed = sv->n_batches = sv->n_direct = 0;
    sv->butterflies = 0;
    sv->any = false;
    for (auto it = sv->reqs.begin(); it != sv->reqs.end();) {
        if (it->second.status != NTT_ERR_PENDING)
            it = sv->reqs.erase(it);
        else
            ++it;
    }
    return NTT_OK;
}

int ntt_server_inject_failures(ntt_server_t sv, int n_batches) {
    if (!sv || n_batches < 0) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->fail_next = n_batches;
    return NTT_OK;
}

int ntt_server_destroy(ntt_server_t sv) {
    if (!sv) return NTT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    sv->worker.join();
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    if (sv->pool) cudaMemPoolDestroy(sv->pool);
    delete sv;
    return NTT_OK;
}

}  // extern "C"
