// ntt_uneven.cu -- many transforms of different lengths, primes and
// directions in ONE persistent kernel launch.
//
// Host side: descriptors are grouped by (plan, direction).  A group whose
// plan runs in a single pass (L <= 2^11) becomes one "class task" whose rows
// are the transforms themselves (row addresses gathered in a device table),
// so one CTA packs many short transforms that share twiddles.  Every
// transform of a multi-pass plan becomes its own task with one stage per
// pass.  Work items (one CTA's worth of one stage of one task) are listed in
// dependency order as a pipeline over chunks of multi-pass tasks: stage s of
// chunk k beside stage 0 of chunk k + s, so that a later stage reads what the
// previous one wrote shortly before (from L2), with the single-pass items
// spread over the steps.
//
// Device side (ntt_uneven_kernel.cuh; one kernel per butterfly variant,
// compiled in ntt_uneven_lazy.cu and ntt_uneven_ntl.cu): each CTA of the
// persistent grid takes the next item from an atomic counter.  An item of stage s > 0 waits until every item of stage
// s-1 of its task has finished (a per-(task, stage) completion counter).  It
// only ever waits for items with a smaller index, which were taken by CTAs
// already running, so the waits cannot deadlock whatever the residency.
// Every wait is bounded by a clock budget; on expiry the CTA records
// NTT_ERR_TIMEOUT in a status word, raises an abort flag that makes every
// other CTA stop at its next check, and returns.  Inputs of later stages are
// read with L1-bypassing loads because other CTAs of the same launch wrote
// them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <mutex>
#include <vector>

#include "ntt_uneven_kernel.cuh"

namespace ntt {

// What a prepared batch copied from a plan: its split, variant and table
// addresses.  A plan re-split (or given other tables) after the batch was
// prepared no longer matches, and the batch is prepared again instead of
// reading freed tables.
struct PlanSig {
    const ntt_plan_s *plan;
    int npass, variant;
    int logr[kMaxPasses];
    const void *tw[2];
    const void *mid[kMaxPasses][2][2];
    bool operator==(const PlanSig &o) const { return memcmp(this, &o, sizeof(PlanSig)) == 0; }
};

static PlanSig plan_sig(const ntt_plan_s *pl) {
    PlanSig g;
    memset(&g, 0, sizeof(g));
    g.plan = pl;
    g.npass = pl->npass;
    g.variant = pl->variant;
    for (int d = 0; d < 2; ++d) g.tw[d] = pl->tw[d];
    for (int q = 0; q < kMaxPasses; ++q) {
        g.logr[q] = pl->pass[q].logR;
        for (int d = 0; d < 2; ++d) {
            g.mid[q][d][0] = pl->pass[q].ma[d];
            g.mid[q][d][1] = pl->pass[q].mb[d];
        }
    }
    return g;
}

struct Prepared {
    std::vector<ntt_desc_t> key;
    std::vector<PlanSig> sigs;  // one per distinct plan of the batch
    UTask *d_tasks = nullptr;
    UItem *d_items = nullptr;
    uint32_t **d_rowptrs = nullptr;
    unsigned int *d_done = nullptr;
    UCtl *d_ctl = nullptr;
    uint32_t n_items = 0, n_done = 0;
    size_t smem = 0;
    uint32_t buf_chunks = 0;
    unsigned grid = 0;
    int device = -1;
    int variant = NTT_VARIANT_LAZY;  // of every plan in the batch
    void release() {
        cudaFree(d_tasks);
        cudaFree(d_items);
        cudaFree(d_rowptrs);
        cudaFree(d_done);
        cudaFree(d_ctl);
        d_tasks = nullptr;
        d_items = nullptr;
        d_rowptrs = nullptr;
        d_done = nullptr;
        d_ctl = nullptr;
    }
};

static std::mutex g_mu;
// Every batch prepared on a device stays prepared (its work list is small)
// until ntt_uneven_release: graphs that captured different batches then stay
// valid side by side, and preparing one batch never frees another's lists.
static std::map<int, std::vector<Prepared *>> g_preps;
static std::map<int, Prepared *> g_last;  // the batch launched last on each device
static long long g_wait_budget = 2000000000LL;  // clock cycles (about 1 s)
static int g_stall_stage = -1;

static std::vector<PlanSig> batch_sigs(const ntt_desc_t *d, size_t n) {
    std::vector<PlanSig> v;
    std::vector<const ntt_plan_s *> seen;
    for (size_t i = 0; i < n; ++i)
        if (d[i].plan && std::find(seen.begin(), seen.end(), d[i].plan) == seen.end()) {
            seen.push_back(d[i].plan);
            v.push_back(plan_sig(d[i].plan));
        }
    return v;
}

static bool same_key(const Prepared &pr, const ntt_desc_t *d, size_t n) {
    if (pr.key.size() != n) return false;
    if (n && memcmp(pr.key.data(), d, n * sizeof(ntt_desc_t)) != 0) return false;
    return pr.sigs == batch_sigs(d, n);
}

// Stage geometry of pass q of a plan, executed in direction dir as step i.
static UStage make_stage(const ntt_plan_s *pl, int dir, int i, uint32_t nrows_class, size_t *smem) {
    const int n = pl->npass;
    const int q = dir == 0 ? i : n - 1 - i;
    const PassPlan &ps = pl->pass[q];
    LaunchSpec s;
    memset(&s, 0, sizeof(s));
    s.nrows = nrows_class;
    // a large batch count: no tile narrowing (the batch itself fills the GPU)
    tile_params(pl, q, 1u << 20, s, true);
    s.nrows = nrows_class ? nrows_class : (1ull << (pl->logL - ps.logR));
    s.ntiles = (uint32_t)((s.nrows + ((uint64_t)s.per_cta << 2) - 1) / ((uint64_t)s.per_cta << 2));
    if (q != n - 1) {
        const int logV = 2;
        const uint64_t sub = 1ull << (pl->logL - ps.logR - s.logTV - logV);
        s.ntiles = (uint32_t)((sub + s.per_cta - 1) / s.per_cta);
        // the persistent kernel carries column tiles of the default width only
        if (s.logTV != std::min(3, 11 - ps.logR)) *smem = (size_t)-1;
    }
    UStage sg;
    memset(&sg, 0, sizeof(sg));
    sg.logR = (int8_t)ps.logR;
    sg.logS = (int8_t)ps.logS;
    sg.flags = (i == n - 1) ? F_NORMALIZE : 0;
    sg.row = q == n - 1 ? 1 : 0;
    sg.logTV = (int8_t)s.logTV;
    sg.per_cta = (uint16_t)s.per_cta;
    sg.units = s.ntiles;
    sg.buf_chunks = s.buf_chunks;
    if (!sg.row) {
        sg.logTA = (int8_t)ps.logTA;
        sg.flags |= F_MIDDLE | (ps.has_mb ? F_MB : 0);
        sg.ma = (const uint32_t *)ps.ma[dir];
        sg.mb = (const uint32_t *)ps.mb[dir];
    }
    if (*smem != (size_t)-1) *smem = std::max(*smem, (size_t)s.buf_chunks * 16);
    return sg;
}

// The persistent kernel for a batch's butterfly variant.
static UnevenKernel kernel_for(int variant) {
    return variant == NTT_VARIANT_NTL ? uneven_kernel<VAR_NTL>() : uneven_kernel<VAR_LAZY>();
}

static int prepare(const ntt_desc_t *descs, size_t n, Prepared &pr) {
    pr.release();
    pr.key.assign(descs, descs + n);
    pr.sigs = batch_sigs(descs, n);
    cudaGetDevice(&pr.device);
    // group by (plan, direction), preserving first appearance
    std::map<std::pair<ntt_plan_s *, int>, std::vector<size_t>> groups;
    std::vector<std::pair<ntt_plan_s *, int>> order;
    for (size_t i = 0; i < n; ++i) {
        ntt_plan_s *pl = descs[i].plan;
        if (!pl || !descs[i].d_data || (descs[i].inverse != 0 && descs[i].inverse != 1)) return NTT_ERR_ARG;
        if (pl->wbytes != 4 || pl->logL > 22 || pl->logL < 3) return NTT_ERR_RANGE;
        if (pl->variant != NTT_VARIANT_LAZY && pl->variant != NTT_VARIANT_NTL) return NTT_ERR_RANGE;
        if (i == 0) pr.variant = pl->variant;
        if (pl->variant != pr.variant) return NTT_ERR_ARG;  // one butterfly variant per launch
        if ((uintptr_t)descs[i].d_data & 15) return NTT_ERR_ALIGN;
        auto k = std::make_pair(pl, descs[i].inverse);
        if (!groups.count(k)) order.push_back(k);
        groups[k].push_back(i);
    }
    std::vector<UTask> tasks;
    std::vector<uint32_t *> rowptrs;
    std::vector<size_t> rowptr_off;  // per class task: offset into rowptrs
    std::vector<int> is_class;
    size_t smem = 0;
    uint32_t done = 0;
    // multi-pass tasks first (longest first), then class tasks
    std::stable_sort(order.begin(), order.end(), [](const std::pair<ntt_plan_s *, int> &x,
                                                    const std::pair<ntt_plan_s *, int> &y) {
        return x.first->logL > y.first->logL;
    });
    for (auto &k : order) {
        ntt_plan_s *pl = k.first;
        const int dir = k.second;
        const auto &idx = groups[k];
        if (pl->npass == 1) {
            UTask t;
            memset(&t, 0, sizeof(t));
            t.tw = (const uint32_t *)pl->tw[dir];
            t.p = (uint32_t)pl->p;
            t.logL = (int8_t)pl->logL;
            t.nstages = 1;
            t.dir = (int8_t)dir;
            t.nrows = idx.size();
            t.done_base = done;
            done += 1;
            t.st[0] = make_stage(pl, dir, 0, (uint32_t)idx.size(), &smem);
            rowptr_off.push_back(rowptrs.size());
            for (size_t i : idx) rowptrs.push_back((uint32_t *)descs[i].d_data);
            tasks.push_back(t);
            is_class.push_back(1);
        } else {
            for (size_t i : idx) {
                UTask t;
                memset(&t, 0, sizeof(t));
                t.data = (uint32_t *)descs[i].d_data;
                t.tw = (const uint32_t *)pl->tw[dir];
                t.p = (uint32_t)pl->p;
                t.logL = (int8_t)pl->logL;
                t.nstages = (int8_t)pl->npass;
                t.dir = (int8_t)dir;
                t.done_base = done;
                done += pl->npass;
                for (int s = 0; s < pl->npass; ++s) t.st[s] = make_stage(pl, dir, s, 0, &smem);
                rowptr_off.push_back(0);
                tasks.push_back(t);
                is_class.push_back(0);
            }
        }
    }
    if (smem == (size_t)-1) return NTT_ERR_RANGE;  // a plan with a narrow column tile
    // items: stage 0 of multi-pass tasks, class tasks, then later stages
    // Item order: a pipeline over chunks of multi-pass tasks (about
    // kChunkBytes of transform data each).  Step k lists stage s of chunk
    // k - s for every s, so a task's later stage follows its previous stage
    // by one step: its inputs were written recently (still in L2; the whole
    // batch's intermediate data would not be) and its dependencies are
    // normally met when it is claimed.  The single-pass items, which depend
    // on nothing, are spread evenly over the steps.  Every item still comes
    // after all items it waits for, so the queue always drains.
    std::vector<UItem> items;
    {
        // 16 MB measured best of 8, 12, 16, 24 and 48 MB on the 4096-transform
        // workload (24 MB: 1 % slower, 8 and 48 MB: 4-8 % slower)
        const uint64_t kChunkBytes = 16ull << 20;
        std::vector<std::vector<uint32_t>> chunks(1);
        uint64_t acc = 0;
        int max_stages = 1;
        for (size_t ti = 0; ti < tasks.size(); ++ti) {
            if (is_class[ti]) continue;
            const uint64_t bytes = 4ull << tasks[ti].logL;
            if (acc > 0 && acc + bytes > kChunkBytes) {
                chunks.emplace_back();
                acc = 0;
            }
            chunks.back().push_back((uint32_t)ti);
            acc += bytes;
            max_stages = std::max<int>(max_stages, tasks[ti].nstages);
        }
        if (chunks.back().empty()) chunks.pop_back();
        std::vector<UItem> class_items;
        for (size_t ti = 0; ti < tasks.size(); ++ti)
            if (is_class[ti])
                for (uint32_t c = 0; c < tasks[ti].st[0].units; ++c) class_items.push_back({(uint32_t)ti, 0, c});
        const size_t nsteps = chunks.size() + (size_t)max_stages - 1;
        size_t next_class = 0;
        for (size_t k = 0; k < nsteps; ++k) {
            for (int sg = 0; sg < max_stages; ++sg) {
                if (k < (size_t)sg || k - sg >= chunks.size()) continue;
                for (uint32_t ti : chunks[k - sg])
                    if (sg < tasks[ti].nstages)
                        for (uint32_t c = 0; c < tasks[ti].st[sg].units; ++c) items.push_back({ti, (uint32_t)sg, c});
            }
            const size_t upto = nsteps ? class_items.size() * (k + 1) / nsteps : class_items.size();
            for (; next_class < upto; ++next_class) items.push_back(class_items[next_class]);
        }
        for (; next_class < class_items.size(); ++next_class) items.push_back(class_items[next_class]);
    }
    // device copies
    cudaError_t e;
    if (!rowptrs.empty()) {
        e = cudaMalloc(&pr.d_rowptrs, rowptrs.size() * sizeof(uint32_t *));
        if (e != cudaSuccess) return NTT_ERR_NOMEM;
        e = cudaMemcpy(pr.d_rowptrs, rowptrs.data(), rowptrs.size() * sizeof(uint32_t *), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uneven rowptrs");
        for (size_t ti = 0; ti < tasks.size(); ++ti)
            if (is_class[ti]) tasks[ti].rowptrs = pr.d_rowptrs + rowptr_off[ti];
    }
    e = cudaMalloc(&pr.d_tasks, std::max<size_t>(1, tasks.size()) * sizeof(UTask));
    if (e != cudaSuccess) return NTT_ERR_NOMEM;
    e = cudaMalloc(&pr.d_items, std::max<size_t>(1, items.size()) * sizeof(UItem));
    if (e != cudaSuccess) return NTT_ERR_NOMEM;
    e = cudaMalloc(&pr.d_done, std::max<uint32_t>(1, done) * sizeof(unsigned int));
    if (e != cudaSuccess) return NTT_ERR_NOMEM;
    e = cudaMalloc(&pr.d_ctl, sizeof(UCtl));
    if (e != cudaSuccess) return NTT_ERR_NOMEM;
    if (!tasks.empty()) {
        e = cudaMemcpy(pr.d_tasks, tasks.data(), tasks.size() * sizeof(UTask), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uneven tasks");
    }
    if (!items.empty()) {
        e = cudaMemcpy(pr.d_items, items.data(), items.size() * sizeof(UItem), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uneven items");
    }
    pr.n_items = (uint32_t)items.size();
    pr.n_done = done;
    pr.buf_chunks = (uint32_t)(std::max<size_t>(smem, 16) / 16);
    pr.smem = (size_t)pr.buf_chunks * 16;  // one tile buffer
    // persistent grid: as many CTAs as fit on the device at once
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pr.device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pr.device);
    const UnevenKernel kern = kernel_for(pr.variant);
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern.func);
    if (e != cudaSuccess) return cuda_fail(e, "uneven attr");
    if (pr.smem + fa.sharedSizeBytes > (size_t)optin) return NTT_ERR_RANGE;
    e = cudaFuncSetAttribute(kern.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pr.smem);
    if (e != cudaSuccess) return cuda_fail(e, "uneven attr");
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern.func, kThreads, pr.smem);
    if (e != cudaSuccess) return cuda_fail(e, "uneven occupancy");
    pr.grid = (unsigned)std::max<long long>(1, std::min<long long>((long long)sms * std::max(per_sm, 1), pr.n_items));
    return NTT_OK;
}

// Free the prepared batches whose transforms lie in [lo, hi) (a scratch
// layout, such as the autotuner's, that nothing else launches).
void uneven_release_range(const void *lo, const void *hi) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<Prepared *> &list = g_preps[dev];
    std::vector<Prepared *> keep;
    for (Prepared *pr : list) {
        bool inside = !pr->key.empty();
        for (const ntt_desc_t &d : pr->key)
            inside = inside && (uintptr_t)d.d_data >= (uintptr_t)lo && (uintptr_t)d.d_data < (uintptr_t)hi;
        if (inside) {
            if (g_last[dev] == pr) g_last.erase(dev);
            pr->release();
            delete pr;
        } else {
            keep.push_back(pr);
        }
    }
    list.swap(keep);
}

}  // namespace ntt

using namespace ntt;

extern "C" {

int ntt_execute_uneven(const ntt_desc_t *descs, size_t n, void *stream) {
    if (!descs || n == 0) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<Prepared *> &list = g_preps[dev];
    Prepared *pr = nullptr;
    for (Prepared *q : list)
        if (q->d_ctl && q->device == dev && same_key(*q, descs, n)) {
            pr = q;
            break;
        }
    if (!pr) {
        pr = new (std::nothrow) Prepared();
        if (!pr) return NTT_ERR_NOMEM;
        int rc = prepare(descs, n, *pr);
        if (rc) {
            pr->release();
            delete pr;
            return rc;
        }
        list.push_back(pr);
    }
    g_last[dev] = pr;
    cudaError_t e = cudaMemsetAsync(pr->d_done, 0, std::max<uint32_t>(1, pr->n_done) * sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr->d_ctl, 0, sizeof(UCtl), st);
    if (e != cudaSuccess) return cuda_fail(e, "uneven memset");
    e = kernel_for(pr->variant).launch(pr->grid, pr->smem, st, pr->d_tasks, pr->d_items, pr->n_items, pr->d_done,
                                       pr->d_ctl, g_wait_budget, g_stall_stage);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "k_uneven");
}

int ntt_uneven_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceSynchronize();  // launches of these batches may still run
    for (Prepared *pr : g_preps[dev]) {
        pr->release();
        delete pr;
    }
    g_preps[dev].clear();
    g_last.erase(dev);
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "uneven release");
}

int ntt_uneven_status(int *status) {
    if (!status) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaGetDevice(&dev);
    auto it = g_last.find(dev);
    if (it == g_last.end() || !it->second || !it->second->d_ctl) {
        *status = NTT_OK;
        return NTT_OK;
    }
    UCtl c;
    cudaError_t e = cudaMemcpy(&c, it->second->d_ctl, sizeof(UCtl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "uneven status");
    *status = c.status;
    return NTT_OK;
}

int ntt_uneven_set_wait_budget(long long cycles, int stall_stage) {
    if (cycles <= 0) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    g_wait_budget = cycles;
    g_stall_stage = stall_stage;
    return NTT_OK;
}

}  // extern "C"
