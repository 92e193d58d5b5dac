// ntt_autotune.cu -- picks the pass split of a plan (and the body of its row
// pass) by timing candidates on the device, and remembers the choice in a
// small JSON cache file.
//
// A candidate is a split of log L into passes (the radix of each on-chip
// sub-transform); the kernel geometry of each pass (tile width, rows per
// CTA) follows from it.  Every candidate runs forward + inverse on a scratch
// batch, timed with CUDA events after warm-up; the fastest is kept.  The
// cache key is (GPU name, word size, log L, log2 of the batch rounded down),
// so one tuning serves every plan of that shape on that GPU model.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ntt_internal.hpp"

namespace ntt {

static std::mutex g_tune_mu;

static std::string cache_path() {
    const char *p = getenv("NTT_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/ntt_gb300_autotune.json";
}

// The cache is a flat JSON object {"key": [l0, l1, ...], ...}.
static std::map<std::string, std::vector<int>> load_cache() {
    std::map<std::string, std::vector<int>> m;
    std::ifstream f(cache_path());
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while (true) {
        size_t k0 = s.find('"', i);
        if (k0 == std::string::npos) break;
        size_t k1 = s.find('"', k0 + 1);
        size_t a0 = s.find('[', k1), a1 = s.find(']', a0);
        if (k1 == std::string::npos || a0 == std::string::npos || a1 == std::string::npos) break;
        std::vector<int> v;
        std::stringstream vs(s.substr(a0 + 1, a1 - a0 - 1));
        std::string tok;
        while (std::getline(vs, tok, ',')) v.push_back(atoi(tok.c_str()));
        m[s.substr(k0 + 1, k1 - k0 - 1)] = v;
        i = a1 + 1;
    }
    return m;
}

static void save_cache(const std::map<std::string, std::vector<int>> &m) {
    const std::string path = cache_path();
    // create the parent directories (mkdir -p)
    for (size_t pos = path.find('/', 1); pos != std::string::npos; pos = path.find('/', pos + 1))
        mkdir(path.substr(0, pos).c_str(), 0755);
    const std::string tmp = path + ".tmp";
    std::ofstream f(tmp);
    if (!f) return;
    f << "{\n";
    size_t n = 0;
    for (auto &kv : m) {
        f << "  \"" << kv.first << "\": [";
        for (size_t i = 0; i < kv.second.size(); ++i) f << (i ? ", " : "") << kv.second[i];
        f << "]" << (++n < m.size() ? "," : "") << "\n";
    }
    f << "}\n";
    f.close();
    rename(tmp.c_str(), path.c_str());
}

static std::string tune_key(const ntt_plan_s *pl, size_t batch) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, pl->device);
    int lb = 0;
    while ((2ull << lb) <= batch) ++lb;
    std::string name = prop.name;
    for (char &c : name)
        if (c == '"' || c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof(buf), "%s/w%d/l%d/b%d", name.c_str(), pl->wbytes * 8, pl->logL, lb);
    return buf;
}

// Candidate splits: one pass when it fits, every two-pass split, and a few
// balanced three-pass splits for long transforms.
static std::vector<std::vector<int>> candidates(const ntt_plan_s *pl) {
    std::vector<std::vector<int>> c;
    const int l = pl->logL;
    auto push = [&](std::vector<int> v) {
        int n = (int)v.size();
        if (split_allowed(l, pl->wbytes, n, v.data())) c.push_back(v);
    };
    if (l <= kMaxRowLog) push({l});
    for (int a = 3; a <= kMaxColLog; ++a) push({a, l - a});
    for (int a = 3; a <= kMaxColLog; ++a)
        for (int b = 3; b <= kMaxColLog; ++b)
            if (l - a - b >= 6 && l - a - b <= kMaxRowLog && std::abs(a - b) <= 1) push({a, b, l - a - b});
    return c;
}

}  // namespace ntt

using namespace ntt;

extern "C" int ntt_plan_autotune(ntt_plan_t pl, size_t batch, int use_cache, int *log_r_out) {
    if (!pl || batch == 0) return NTT_ERR_ARG;
    if (pl->logL <= 2) return NTT_OK;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::string key = tune_key(pl, batch);
    // the row pass's body (radix-8 CTA rows, or one warp per row) is cached
    // beside the split under key + "/warp"; an entry without it means CTA rows
    const std::string wkey = key + "/warp";
    if (use_cache) {
        auto m = load_cache();
        auto it = m.find(key);
        if (it != m.end() && split_allowed(pl->logL, pl->wbytes, (int)it->second.size(), it->second.data())) {
            int rc = ntt_plan_set_split(pl, (int)it->second.size(), it->second.data());
            auto wt = m.find(wkey);
            pl->warp_rows = wt != m.end() && !wt->second.empty() && wt->second[0] != 0;
            if (rc == NTT_OK && log_r_out)
                for (size_t i = 0; i < it->second.size(); ++i) log_r_out[i] = it->second[i];
            return rc;
        }
    }
    const size_t words = batch * pl->L;
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, words * pl->wbytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "autotune buffer");
    cudaMemset(buf, 0, words * pl->wbytes);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_variant = pl->variant;
    const bool saved_warp = pl->warp_rows;
    pl->warp_rows = false;  // splits are timed with the radix-8 rows
    // time the lazy butterflies where the modulus allows them (the splits'
    // relative cost is the same for every variant), else the plan's own
    if (variant_fits(pl, NTT_VARIANT_LAZY)) pl->variant = NTT_VARIANT_LAZY;
    std::vector<int> best;
    float best_ms = 1e30f;
    int rc = NTT_OK;
    for (const auto &cand : candidates(pl)) {
        rc = ntt_plan_set_split(pl, (int)cand.size(), cand.data());
        if (rc) break;
        for (int w = 0; w < 2; ++w) {
            enqueue_transform(pl, 0, buf, batch, pl->L, st);
            enqueue_transform(pl, 1, buf, batch, pl->L, st);
        }
        cudaEventRecord(e0, st);
        const int reps = 5;
        for (int r = 0; r < reps; ++r) {
            enqueue_transform(pl, 0, buf, batch, pl->L, st);
            enqueue_transform(pl, 1, buf, batch, pl->L, st);
        }
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    // then the row pass's body for the chosen split: one warp per row against
    // the radix-8 rows, when the rows are 2^5..2^10 words (measured: warp
    // rows win for short rows in small, latency-bound launches)
    bool warp = false;
    const int row_log = best.empty() ? 0 : best.back();
    if (rc == NTT_OK && row_log >= 5 && row_log <= 10) {
        rc = ntt_plan_set_split(pl, (int)best.size(), best.data());
        float ms[2] = {0, 0};
        for (int w = 0; w < 2 && rc == NTT_OK; ++w) {
            pl->warp_rows = w != 0;
            for (int r = 0; r < 2; ++r) {
                enqueue_transform(pl, 0, buf, batch, pl->L, st);
                enqueue_transform(pl, 1, buf, batch, pl->L, st);
            }
            cudaEventRecord(e0, st);
            for (int r = 0; r < 5; ++r) {
                enqueue_transform(pl, 0, buf, batch, pl->L, st);
                enqueue_transform(pl, 1, buf, batch, pl->L, st);
            }
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotune timing");
                break;
            }
            cudaEventElapsedTime(&ms[w], e0, e1);
        }
        warp = rc == NTT_OK && ms[1] < ms[0];
    }
    pl->variant = saved_variant;
    pl->warp_rows = saved_warp;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(buf);
    if (rc) return rc;
    if (best.empty()) return NTT_ERR_ARG;
    rc = ntt_plan_set_split(pl, (int)best.size(), best.data());
    if (rc) return rc;
    pl->warp_rows = warp;
    if (log_r_out)
        for (size_t i = 0; i < best.size(); ++i) log_r_out[i] = best[i];
    auto m = load_cache();
    m[key] = best;
    m[wkey] = std::vector<int>{warp ? 1 : 0};
    save_cache(m);
    return NTT_OK;
}

// ------------------------------------------------------------ uneven batches

// The pass split of each multi-pass length class of an uneven batch, tuned
// inside the persistent launch itself (the classes share the GPU, so the best
// split of a class alone is not necessarily its best in the mix).  A class is
// one transform length: every multi-pass plan of that length (whatever its
// prime) takes the class's split.  One round of coordinate descent: classes
// in order of decreasing length, every allowed two-pass split of the class
// timed with the others fixed.  Timed on a scratch copy of the batch's
// layout, so the caller's data are not touched.
extern "C" int ntt_uneven_autotune(const ntt_desc_t *descs, size_t n, int use_cache, void *stream) {
    if (!descs || n == 0) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    struct Class {
        int logL;
        size_t count = 0;
        std::vector<ntt_plan_s *> plans;
        std::string key;
    };
    std::vector<Class> classes;
    for (size_t i = 0; i < n; ++i) {
        ntt_plan_s *pl = descs[i].plan;
        if (!pl) return NTT_ERR_ARG;
        if (pl->logL <= kMaxRowLog) continue;
        auto it = std::find_if(classes.begin(), classes.end(),
                               [&](const Class &c) { return c.logL == pl->logL && c.plans[0]->wbytes == pl->wbytes; });
        if (it == classes.end()) {
            classes.emplace_back();
            classes.back().logL = pl->logL;
            it = classes.end() - 1;
        }
        ++it->count;
        if (std::find(it->plans.begin(), it->plans.end(), pl) == it->plans.end()) it->plans.push_back(pl);
    }
    if (classes.empty()) return NTT_OK;
    std::stable_sort(classes.begin(), classes.end(), [](const Class &a, const Class &b) { return a.logL > b.logL; });
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (Class &c : classes) c.key = "uneven/" + tune_key(c.plans[0], c.count);
    auto apply = [&](Class &c, const std::vector<int> &v) -> int {
        for (ntt_plan_s *pl : c.plans) {
            bool same = (int)v.size() == pl->npass;
            for (size_t q = 0; same && q < v.size(); ++q) same = pl->pass[q].logR == v[q];
            if (!same) {
                int rc = ntt_plan_set_split(pl, (int)v.size(), v.data());
                if (rc) return rc;
            }
        }
        return NTT_OK;
    };
    if (use_cache) {
        auto m = load_cache();
        bool all = true;
        for (size_t i = 0; i < classes.size() && all; ++i) {
            auto it = m.find(classes[i].key);
            all = it != m.end() && split_allowed(classes[i].logL, classes[i].plans[0]->wbytes,
                                                 (int)it->second.size(), it->second.data());
        }
        if (all) {
            for (Class &c : classes) {
                int rc = apply(c, m[c.key]);
                if (rc) return rc;
            }
            return NTT_OK;
        }
    }
    // scratch copy of the layout: each transform at a 16-byte-aligned offset
    std::vector<ntt_desc_t> sd(descs, descs + n);
    size_t words = 0;
    for (size_t i = 0; i < n; ++i) words += (descs[i].plan->L + 3) & ~3ull;
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, std::max<size_t>(words, 4) * 4);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "uneven autotune buffer");
    cudaMemsetAsync(buf, 0, std::max<size_t>(words, 4) * 4, st);
    size_t off = 0;
    for (size_t i = 0; i < n; ++i) {
        sd[i].d_data = static_cast<uint32_t *>(buf) + off;
        off += (descs[i].plan->L + 3) & ~3ull;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_batch = [&](float *ms) -> int {
        for (int w = 0; w < 2; ++w) {
            int rc = ntt_execute_uneven(sd.data(), n, st);
            if (rc) return rc;
        }
        cudaEventRecord(e0, st);
        const int reps = 5;
        for (int r = 0; r < reps; ++r) {
            int rc = ntt_execute_uneven(sd.data(), n, st);
            if (rc) return rc;
        }
        cudaEventRecord(e1, st);
        cudaError_t ee = cudaEventSynchronize(e1);
        if (ee != cudaSuccess) return cuda_fail(ee, "uneven autotune timing");
        int status = 0;
        int rc = ntt_uneven_status(&status);
        if (rc || status) return rc ? rc : status;
        cudaEventElapsedTime(ms, e0, e1);
        return NTT_OK;
    };
    int rc = NTT_OK;
    for (size_t ci = 0; ci < classes.size() && rc == NTT_OK; ++ci) {
        Class &c = classes[ci];
        const ntt_plan_s *p0 = c.plans[0];
        std::vector<int> cur(p0->npass);
        for (int q = 0; q < p0->npass; ++q) cur[q] = p0->pass[q].logR;
        rc = apply(c, cur);  // every plan of the class on one split to start
        if (rc) break;
        std::vector<int> best = cur;
        float best_ms = 1e30f;
        rc = time_batch(&best_ms);
        if (rc) break;
        for (int a = 3; a <= kMaxColLog; ++a) {
            std::vector<int> cand = {a, c.logL - a};
            if (cand == cur || cand[1] > kMaxRowLog || !split_allowed(c.logL, p0->wbytes, 2, cand.data())) continue;
            rc = apply(c, cand);
            if (rc) break;
            float ms = 0;
            const int trc = time_batch(&ms);
            if (trc == NTT_ERR_RANGE) continue;  // a split the persistent kernel does not carry
            if (trc) {
                rc = trc;
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        if (rc) break;
        rc = apply(c, best);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    // the work lists prepared for the scratch layout (one per candidate) go with it
    uneven_release_range(buf, static_cast<uint32_t *>(buf) + std::max<size_t>(words, 4));
    cudaFree(buf);
    if (rc) return rc;
    auto m = load_cache();
    for (const Class &c : classes) {
        std::vector<int> v(c.plans[0]->npass);
        for (int q = 0; q < c.plans[0]->npass; ++q) v[q] = c.plans[0]->pass[q].logR;
        m[c.key] = v;
    }
    save_cache(m);
    return NTT_OK;
}
