// ntt_plan.cu -- host side of the library: number theory, plans and their
// device tables, the pass schedule, and the transform entry points of the C ABI.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "ntt_internal.hpp"
#include "ntt_kernels.cuh"

namespace ntt {

static thread_local std::string g_last_cuda_error;

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t pool = nullptr;
            e = cudaMemPoolCreate(&pool, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = 4ull << 30;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(pool);
                return e;
            }
            pools[dev] = pool;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, pools[dev], st);
}

int cuda_fail(cudaError_t e, const char *where) {
    g_last_cuda_error = std::string(where) + ": " + cudaGetErrorString(e);
    return NTT_ERR_CUDA;
}

// ------------------------------------------------------------ number theory
namespace nt {

typedef unsigned __int128 u128;

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t result = 1 % p, base = a % p;
    while (e) {
        if (e & 1) result = mulmod(result, base, p);
        base = mulmod(base, base, p);
        e >>= 1;
    }
    return result;
}

// Strong-probable-prime test to each of the first twelve prime bases; this
// set has no 64-bit strong pseudoprime, so the answer is exact.
bool is_prime(uint64_t n) {
    const uint64_t small[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t q : small) {
        if (n % q == 0) return n == q;
    }
    uint64_t d = n - 1;
    int s = __builtin_ctzll(d);
    d >>= s;
    for (uint64_t a : small) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < s && witness; ++i) {
            x = mulmod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

uint64_t smallest_qnr(uint64_t p) {
    const uint64_t half = (p - 1) / 2;
    for (uint64_t g = 2; g < p; ++g)
        if (powmod(g, half, p) == p - 1) return g;
    return 0;
}

uint64_t shoup_quotient(uint64_t w, uint64_t p, int word_bits) {
    return (uint64_t)(((u128)w << word_bits) / p);
}

uint32_t bitrev(uint32_t k, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1u) << (bits - 1 - i);
    return r;
}

}  // namespace nt

// ------------------------------------------------------------ pass schedule

static int ilog2u(uint64_t x) { return 63 - __builtin_clzll(x); }

// Default split of log L into passes: one row pass of at most 2^11
// elements, preceded by as few column passes (each at most 2^11) as needed,
// balanced.
static int default_split(int logL, int wbytes, int *logr) {
    (void)wbytes;
    if (logL <= kMaxRowLog) {
        logr[0] = logL;
        return 1;
    }
    if (logL <= 2 * kMaxRowLog) {
        int c = std::max(logL - kMaxRowLog, std::min((logL + 1) / 2, 9));
        logr[0] = c;
        logr[1] = logL - c;
        return 2;
    }
    int rest = logL - kMaxRowLog;  // two column passes
    logr[0] = (rest + 1) / 2;
    logr[1] = rest - logr[0];
    logr[2] = kMaxRowLog;
    return 3;
}

bool split_allowed(int logL, int wbytes, int n, const int *logr) {
    if (n < 1 || n > kMaxPasses) return false;
    if (logL <= 2) return n == 1 && logr[0] == logL;
    int sum = 0;
    const int logT = wbytes == 4 ? 5 : 4;  // narrowest column tile is 16 bytes; need S >= 8 vectors
    for (int i = 0; i < n; ++i) {
        if (logr[i] < 3 || logr[i] > std::max(kMaxRowLog, kMaxColLog)) return false;
        sum += logr[i];
    }
    if (sum != logL) return false;
    int after = logL;
    for (int i = 0; i < n - 1; ++i) {
        after -= logr[i];
        if (logr[i] > kMaxColLog) return false;
        if (after < logT) return false;
    }
    return true;
}

// Widest column tile: 8 vectors (128-byte rows), or the whole column stride.
static int max_logtv(int logS, int wbytes) {
    const int logV = wbytes == 4 ? 2 : 1;
    return std::min(3, logS - logV);
}

static void free_tables(ntt_plan_s *pl) {
    for (int d = 0; d < 2; ++d) {
        for (void **t : {&pl->tw[d], &pl->twm[d]}) {
            if (*t) cudaFree(*t);
            *t = nullptr;
        }
        for (int q = 0; q < kMaxPasses; ++q)
            for (void **t : {&pl->pass[q].ma[d], &pl->pass[q].mb[d], &pl->pass[q].mam[d], &pl->pass[q].mbm[d]}) {
                if (*t) cudaFree(*t);
                *t = nullptr;
            }
    }
    pl->mont = false;
    pl->table_bytes = 0;
}

// Upload a host vector of (W, W') pairs (as uint64) in the plan's word type.
static int upload_pairs(ntt_plan_s *pl, const std::vector<uint64_t> &pairs, void **dst) {
    const size_t n = pairs.size();
    const size_t bytes = n * pl->wbytes;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "cudaMalloc");
    if (pl->wbytes == 4) {
        std::vector<uint32_t> h(n);
        for (size_t i = 0; i < n; ++i) h[i] = (uint32_t)pairs[i];
        e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
    } else {
        e = cudaMemcpy(d, pairs.data(), bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy tables");
    }
    *dst = d;
    pl->table_bytes += bytes;
    return NTT_OK;
}

// Second word of a twiddle pair: Shoup's quotient floor(W beta / p)
// (Algorithms 2-4) or the Montgomery form beta W mod p (Algorithm 5).
static inline uint64_t second_word(uint64_t w, uint64_t p, int bits, bool mont) {
    if (!mont) return nt::shoup_quotient(w, p, bits);
    return (uint64_t)(((unsigned __int128)w << bits) % p);
}

static inline void push_pair(std::vector<uint64_t> &v, uint64_t w, uint64_t p, int bits, bool mont) {
    v.push_back(w);
    v.push_back(second_word(w, p, bits, mont));
}

// Build the device tables of the plan for its current split, in Shoup form
// (tw, ma, mb) or in Montgomery form (twm, mam, mbm).
static int build_tables_form(ntt_plan_s *pl, bool mont) {
    const uint64_t p = pl->p;
    const int bits = pl->wbytes * 8;
    int maxr = 0;
    for (int q = 0; q < pl->npass; ++q) maxr = std::max(maxr, pl->pass[q].logR);
    pl->tw_log = std::max(2, maxr);  // lane stages read entries 1..3
    for (int d = 0; d < 2; ++d) {
        const uint64_t root = d == 0 ? pl->omega : pl->omega_inv;
        // stage table: entry m+k = root^(k L / 2m), for m = 1, 2, ..., 2^(tw_log-1);
        // entry 0 is unused (set to W = 1)
        std::vector<uint64_t> tw;
        tw.reserve(2 * ((size_t)1 << pl->tw_log));
        push_pair(tw, 1, p, bits, mont);
        for (int b = 0; b < pl->tw_log; ++b) {
            const uint64_t m = 1ull << b;
            const uint64_t step = nt::powmod(root, pl->L / (2 * m), p);
            uint64_t w = 1;
            for (uint64_t k = 0; k < m; ++k) {
                push_pair(tw, w, p, bits, mont);
                w = nt::mulmod(w, step, p);
            }
        }
        tw.resize(2 * ((size_t)1 << pl->tw_log));  // 2^tw_log entries: [0] + m in [1, 2^tw_log)
        int rc = upload_pairs(pl, tw, mont ? &pl->twm[d] : &pl->tw[d]);
        if (rc) return rc;
        // middle tables of the column passes
        int logB = pl->logL;
        for (int q = 0; q < pl->npass - 1; ++q) {
            ntt::PassPlan &ps = pl->pass[q];
            const int logR = ps.logR, logS = logB - logR;
            const uint64_t R = 1ull << logR;
            const uint64_t u = pl->L >> logB;  // middle twiddle omega^(u c rev(s))
            std::vector<uint64_t> ma, mb;
            ma.reserve(2 * (R << ps.logTA));
            for (uint64_t s = 0; s < R; ++s) {
                const uint64_t z = nt::powmod(root, (u * nt::bitrev((uint32_t)s, logR)) % pl->L, p);
                uint64_t w = 1;
                for (uint64_t c = 0; c < (1ull << ps.logTA); ++c) {
                    push_pair(ma, w, p, bits, mont);
                    w = nt::mulmod(w, z, p);
                }
            }
            rc = upload_pairs(pl, ma, mont ? &ps.mam[d] : &ps.ma[d]);
            if (rc) return rc;
            if (ps.has_mb) {
                const uint64_t nhi = 1ull << (logS - ps.logTA);
                mb.assign(2 * nhi * R, 0);
                for (uint64_t s = 0; s < R; ++s) {
                    const uint64_t zt = nt::powmod(root, ((u * nt::bitrev((uint32_t)s, logR)) << ps.logTA) % pl->L, p);
                    uint64_t w = 1;
                    for (uint64_t chi = 0; chi < nhi; ++chi) {
                        mb[2 * (chi * R + s)] = w;
                        mb[2 * (chi * R + s) + 1] = second_word(w, p, bits, mont);
                        w = nt::mulmod(w, zt, p);
                    }
                }
                rc = upload_pairs(pl, mb, mont ? &ps.mbm[d] : &ps.mb[d]);
                if (rc) return rc;
            }
            logB -= logR;
        }
    }
    if (mont) pl->mont = true;
    return NTT_OK;
}

static int build_tables(ntt_plan_s *pl) {
    const bool mont = pl->mont;
    free_tables(pl);
    int rc = build_tables_form(pl, false);
    if (rc == NTT_OK && (mont || pl->variant == NTT_VARIANT_MONT)) rc = build_tables_form(pl, true);
    return rc;
}

// Pass geometry of a split (no device work): radix, stride, tile width and
// middle-table shape of every pass.
static void set_geometry(ntt_plan_s *pl, int n, const int *logr) {
    pl->npass = n;
    const int logV = pl->wbytes == 4 ? 2 : 1;
    int logB = pl->logL;
    for (int q = 0; q < kMaxPasses; ++q) pl->pass[q] = PassPlan();
    for (int q = 0; q < n; ++q) {
        PassPlan &ps = pl->pass[q];
        ps.logR = logr[q];
        ps.logS = q == n - 1 ? 0 : logB - logr[q];
        if (q < n - 1) {
            ps.logTV = max_logtv(ps.logS, pl->wbytes);
            const int logT = ps.logTV + logV;
            // One middle-twiddle table MA of B pairs (a single Shoup product per
            // element) while it stays small enough to live in L2 (<= 2 MiB);
            // beyond that MA and MB of about 2 R sqrt(S) pairs.
            const bool full = ((uint64_t)2 * pl->wbytes << (ps.logR + ps.logS)) <= (2u << 20);
            ps.logTA = full ? ps.logS : std::min(ps.logS, std::max(logT, (ps.logS + 1) / 2));
            ps.has_mb = ps.logTA < ps.logS;
        }
        logB -= logr[q];
    }
}

static int apply_split(ntt_plan_s *pl, int n, const int *logr) {
    set_geometry(pl, n, logr);
    return build_tables(pl);
}

// ---------------------------------------------------------------- launches

// Input-range check (checked mode): the smallest flat index b*L + i whose
// word is >= bound, by an atomic minimum over a grid-stride scan.
template <typename W>
__global__ void k_check_input(const W *__restrict__ d, uint64_t stride, int logL, uint64_t total, W bound,
                              unsigned long long *first) {
    const uint64_t mask = (1ull << logL) - 1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x)
        if (d[(i >> logL) * stride + (i & mask)] >= bound) atomicMin(first, (unsigned long long)i);
}

// Wait budget of the pass kernels' tile copies and the test hook of
// ntt_pass_set_wait_budget.
static std::atomic<long long> g_pass_budget{2000000000LL};
static std::atomic<uint32_t> g_pass_extra{0};

// Device status word of the pass kernels: a file-scope __device__ word (zero
// when the module loads), so no transform ever allocates for it.  Host code
// cannot use the variable's name as a device address; its address on each
// device is looked up once with cudaGetSymbolAddress, with that device
// current (ntt_plan does it for the plan's device, so the first transform
// does no lookup either).
static __device__ int g_pass_status_word;

static cudaError_t pass_status(int **out) {
    static std::mutex m;
    static int *words[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(m);
    if (!words[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pass_status_word);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        words[dev] = static_cast<int *>(p);
    }
    *out = words[dev];
    return cudaSuccess;
}

// Tensor map of a column pass's view of the batch: dimension 0 the S words of
// a row, 1 the L/S rows of a transform, 2 the transforms; the box is one
// 128-byte tile row wide and up to 256 rows high.  False when the layout does
// not allow tensor copies (16-byte alignment of the base and the strides).
static bool tma_map(const ntt_plan_s *pl, LaunchSpec &s, size_t batch) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode enc = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<Encode>(fn);
    });
    if (!enc) return false;
    const uint64_t w = (uint64_t)pl->wbytes;
    const uint64_t S = 1ull << s.logS;
    if ((reinterpret_cast<uintptr_t>(s.data) & 15u) != 0 || (S * w) % 16 != 0 || (s.stride * w) % 16 != 0) return false;
    if (S * w < 128) return false;
    const cuuint64_t dims[3] = {S, pl->L / S, batch};
    const cuuint64_t strides[2] = {S * w, s.stride * w};
    const cuuint32_t box[3] = {(cuuint32_t)(128 / w), (cuuint32_t)std::min(256, 1 << s.logR), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&s.map, w == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, s.data, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

static_assert(NTT_VARIANT_LAZY == VAR_LAZY && NTT_VARIANT_NTL == VAR_NTL && NTT_VARIANT_MONT == VAR_MONT &&
                  NTT_VARIANT_MOLLER == VAR_MOLLER,
              "the C-ABI variant numbers select the kernel variants directly");

static cudaError_t launch(const ntt_plan_s *pl, const LaunchSpec &s, int kind, int dir, cudaStream_t st) {
    const int var = pl->variant;  // NTT_VARIANT_LAZY, _NTL, _MONT or _MOLLER: 0, 1, 2, 3
    return pl->wbytes == 4 ? launch_pass_u32(s, kind, dir, var, st) : launch_pass_u64(s, kind, dir, var, st);
}

int enqueue_transform(ntt_plan_s *pl, int dir, void *data, size_t batch, size_t stride, cudaStream_t st) {
    return enqueue_steps(pl, dir, data, batch, stride, st, 0, pl->logL <= 2 ? 1 : pl->npass);
}

int enqueue_steps(ntt_plan_s *pl, int dir, void *data, size_t batch, size_t stride, cudaStream_t st, int first,
                  int count) {
    return enqueue_steps_roots(pl, dir, dir, data, batch, stride, st, first, count);
}

int enqueue_steps_roots(ntt_plan_s *pl, int dir, int roots, void *data, size_t batch, size_t stride,
                        cudaStream_t st, int first, int count) {
    LaunchSpec s;
    memset(&s, 0, sizeof(s));
    s.data = data;
    s.stride = stride;
    s.batch = (uint32_t)batch;
    s.logL = pl->logL;
    s.p = pl->p;
    s.J = pl->J;
    s.wait_budget = g_pass_budget.load();
    s.tx_extra = g_pass_extra.load();
    const bool mont = pl->variant == NTT_VARIANT_MONT;
    s.tw = mont ? pl->twm[roots] : pl->tw[roots];
    if (pl->logL <= 2) {
        s.grid = (unsigned)((batch + 127) / 128);
        cudaError_t e = launch(pl, s, 2, dir, st);
        return e == cudaSuccess ? NTT_OK : cuda_fail(e, "launch tiny");
    }
    const int n = pl->npass;
    for (int i = first; i < first + count && i < n; ++i) {
        const int q = dir == 0 ? i : n - 1 - i;  // inverse runs the passes backwards
        const PassPlan &ps = pl->pass[q];
        s.logR = ps.logR;
        s.logS = ps.logS;
        s.flags = (i == n - 1) ? 1 : 0;  // F_NORMALIZE on the last executed pass
        tile_params(pl, q, batch, s);
        int kind = q == n - 1 ? 1 : 0;
        if (kind == 1 && pl->warp_rows && ps.logR >= 5 && ps.logR <= 10) kind = 3;  // one warp per row
        if (kind == 0) {
            s.logTA = ps.logTA;
            s.flags |= 2 | (ps.has_mb ? 4 : 0);  // F_MIDDLE, F_MB
            s.ma = mont ? ps.mam[roots] : ps.ma[roots];
            s.mb = mont ? ps.mbm[roots] : ps.mb[roots];
        } else {
            s.ma = s.mb = nullptr;
        }
        // prefetching passes (64-bit column passes) double-buffer their tiles
        s.smem = (size_t)(kind == 0 && pl->wbytes == 8 ? 2 : 1) * s.buf_chunks * 16;
        // 64-bit column passes with 128-byte tile rows fetch their tiles by
        // tensor copies (measured 2-5 % faster than the cp.async copies);
        // 32-bit column passes load their first round directly (tensor
        // copies cost them a resident CTA per SM and measured 3-7 % slower)
        if (kind == 0 && s.logTV == 3 && pl->wbytes == 8 && tma_map(pl, s, batch)) {
            s.flags |= 8;  // F_TMA: tiles by tensor copies, double buffered
            s.smem = (size_t)2 * s.buf_chunks * 16 + 16;  // two buffers and their two mbarriers
        }
        if (!s.status) {
            cudaError_t es = pass_status(&s.status);
            if (es != cudaSuccess) return cuda_fail(es, "status word");
        }
        cudaError_t e = launch(pl, s, kind, dir, st);
        if (e != cudaSuccess) return cuda_fail(e, "launch pass");
    }
    return NTT_OK;
}

void tile_params(const ntt_plan_s *pl, int q, uint64_t batch, LaunchSpec &s, bool persistent) {
    const PassPlan &ps = pl->pass[q];
    const int logV = pl->wbytes == 4 ? 2 : 1;
    const int logR = ps.logR;
    if (q == pl->npass - 1) {  // row pass: groups of V rows, one per vector lane
        const uint32_t units_per_group = (1u << logR) >> 3;
        const uint32_t nsp = (1u << logR) + ((1u << logR) >> 3);
        s.logTV = 0;
        s.per_cta = (int)std::max<uint32_t>(1, kThreads / units_per_group);
        s.nrows = s.nrows ? s.nrows : (batch << (pl->logL - logR));
        const uint64_t rows_per_iter = (uint64_t)s.per_cta << logV;
        s.ntiles = (uint32_t)((s.nrows + rows_per_iter - 1) / rows_per_iter);
        s.buf_chunks = (uint32_t)s.per_cta * nsp;
    } else {  // column pass: R rows x TV vectors per sub-tile
        // R * TV <= 4096 vectors in the one buffer of a directly loading
        // (32-bit) column pass with R >= 2^10, <= 2048 otherwise
        const int logmax = (pl->wbytes == 4 && !persistent && logR >= 10) ? 12 : 11;
        int logTV = std::min(ps.logTV, std::max(0, logmax - logR));
        while (logTV > 1 && (batch << (pl->logL - logR - logTV - logV)) < 4 * 152) --logTV;
        const uint32_t units = (1u << (logR + logTV)) >> 3;
        // tiles with 128-byte rows are unpadded (see the kernels' layout)
        const uint32_t nsp = (1u << logR) + (logTV == 3 ? 0u : (1u << logR >> 3));
        s.logTV = logTV;
        s.per_cta = (int)std::max<uint32_t>(1, kThreads / units);
        const uint64_t sub = batch << (pl->logL - logR - logTV - logV);
        s.ntiles = (uint32_t)((sub + s.per_cta - 1) / s.per_cta);
        s.buf_chunks = ((uint32_t)s.per_cta * nsp) << logTV;
        s.nrows = 0;
    }
}

// Host-only self-test of the launch geometry against the kernels' compile-time
// layout, for every allowed split of every length 2^3..2^26, both word sizes
// and a range of batch sizes (see the header).
template <typename W, int LOGR>
static int tvf_t() {
    return ColWidth<LOGR, ColTileLog<W, LOGR>::MAX>::LOGTV;
}
template <typename W>
static int tvf(int logR) {
    static const int t[12] = {0, 0, 0, tvf_t<W, 3>(), tvf_t<W, 4>(), tvf_t<W, 5>(), tvf_t<W, 6>(), tvf_t<W, 7>(),
                              tvf_t<W, 8>(), tvf_t<W, 9>(), tvf_t<W, 10>(), tvf_t<W, 11>()};
    return t[logR];
}

static bool geometry_ok(const ntt_plan_s &pl, int q, uint64_t batch, bool persistent, char *msg, int msg_len) {
    LaunchSpec s;
    memset(&s, 0, sizeof(s));
    tile_params(&pl, q, batch, s, persistent);
    const PassPlan &ps = pl.pass[q];
    const int logV = pl.wbytes == 4 ? 2 : 1;
    const uint64_t R = 1ull << ps.logR;
    const bool row = q == pl.npass - 1;
    const size_t smem_max = 232448;  // 227 KiB of shared memory per CTA
    auto fail = [&](const char *what) {
        if (msg && msg_len > 0)
            snprintf(msg, msg_len, "w%d L=2^%d pass %d/%d log R=%d batch=%llu%s: %s", pl.wbytes * 8, pl.logL, q,
                     pl.npass, ps.logR, (unsigned long long)batch, persistent ? " (uneven)" : "", what);
        return false;
    };
    if (s.per_cta < 1 || s.ntiles < 1) return fail("empty tiling");
    if (row) {
        const uint64_t units = (uint64_t)s.per_cta * (R >> 3);
        if (units != (uint64_t)kThreads) return fail("row tile is not one unit per thread");
        const uint64_t nrows = batch << (pl.logL - ps.logR), per = (uint64_t)s.per_cta << logV;
        if (s.nrows != nrows) return fail("row count");
        if ((uint64_t)s.ntiles * per < nrows || (uint64_t)(s.ntiles - 1) * per >= nrows) return fail("row tiles");
        if (s.buf_chunks != (uint32_t)s.per_cta * (R + R / 8)) return fail("row buffer");
        if ((size_t)s.buf_chunks * 16 > smem_max) return fail("row buffer exceeds shared memory");
        return true;
    }
    const int ltb = ps.logS - s.logTV - logV, lbt = pl.logL - ps.logR - ps.logS;
    if (s.logTV < 0 || ltb < 0 || lbt < 0) return fail("column geometry");
    const uint64_t sub = batch << (ltb + lbt);
    if ((uint64_t)s.ntiles * s.per_cta < sub || (uint64_t)(s.ntiles - 1) * s.per_cta >= sub) return fail("column tiles");
    const int logT = ps.logR - 3 + s.logTV;  // threads (units) of one sub-tile
    const uint64_t units = (uint64_t)s.per_cta << logT;
    if (logT < 8 ? units != (uint64_t)kThreads : units % kThreads != 0)
        return fail("sub-tiles are not contiguous thread blocks");
    // the kernel's shared layout: unpadded exactly when its compile-time width is 8 vectors
    const int tv_kernel = pl.wbytes == 4 ? tvf<uint32_t>(ps.logR) : tvf<uint64_t>(ps.logR);
    if (!persistent && s.logTV > tv_kernel) return fail("tile wider than the kernel's widest");
    const bool dense = s.logTV == 3;
    if (dense && tv_kernel != 3) return fail("unpadded tile for a padded kernel layout");
    const uint64_t nsp = dense ? R : R + R / 8;
    if (s.buf_chunks != ((uint32_t)s.per_cta * nsp << s.logTV)) return fail("column buffer");
    const bool two = pl.wbytes == 8;  // prefetching passes hold two buffers (tensor copies add two mbarriers)
    if ((size_t)(two ? 2 : 1) * s.buf_chunks * 16 + 16 > smem_max) return fail("column buffers exceed shared memory");
    if (two && dense && (((uint64_t)pl.wbytes << ps.logS) < 128 || (R > 256 && R % 256)))
        return fail("tensor-copy box");
    return true;
}

// Whether a butterfly variant's modulus bound holds for the plan's p and word
// (beta = 2^(8 wbytes)): p < beta/4 for the redundant-residue variants
// (Theorems 2-4), p < beta/2 for Algorithm 2 (Theorem 1), p < beta/phi for
// Moeller's form (end of Section 2).
bool variant_fits(const ntt_plan_s *pl, int variant) {
    const int bits = pl->wbytes * 8;
    const uint64_t quarter = 1ull << (bits - 2), half = 1ull << (bits - 1);
    const uint64_t golden = bits == 32 ? (uint64_t)NTT_P_MAX_W32 : (uint64_t)NTT_P_MAX_W64;
    switch (variant) {
        case NTT_VARIANT_LAZY:
        case NTT_VARIANT_MONT: return pl->p < quarter;
        case NTT_VARIANT_NTL: return pl->p < half;
        case NTT_VARIANT_MOLLER: return pl->p <= golden;
        default: return false;
    }
}

}  // namespace ntt

using namespace ntt;

// ------------------------------------------------------------------- C ABI

extern "C" {

int ntt_version(void) { return 100; }

int ntt_pass_status(int reset, int *status) {
    if (!status) return NTT_ERR_ARG;
    int *w = nullptr;
    cudaError_t e = pass_status(&w);
    if (e == cudaSuccess) e = cudaMemcpy(status, w, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(w, 0, sizeof(int));
    return e == cudaSuccess ? NTT_OK : cuda_fail(e, "pass status");
}

int ntt_pass_set_wait_budget(long long cycles, unsigned int stall_bytes) {
    if (cycles <= 0 || stall_bytes % 16 != 0 || stall_bytes > (1u << 16)) return NTT_ERR_ARG;
    g_pass_budget = cycles;
    g_pass_extra = stall_bytes;
    return NTT_OK;
}

const char *ntt_strerror(int code) {
    switch (code) {
        case NTT_OK: return "ok";
        case NTT_ERR_MODULUS: return "modulus is not a prime below 2^62";
        case NTT_ERR_LENGTH: return "length is not a power of two >= 2 dividing p-1";
        case NTT_ERR_ROOT: return "omega is not a primitive L-th root of unity";
        case NTT_ERR_ARG: return "invalid argument";
        case NTT_ERR_CUDA: return "CUDA runtime error";
        case NTT_ERR_NOMEM: return "out of memory";
        case NTT_ERR_TIMEOUT: return "device-side wait timed out";
        case NTT_ERR_ALIGN: return "pointer or stride not 16-byte aligned";
        case NTT_ERR_RANGE: return "size beyond the supported maximum";
        case NTT_ERR_REFUSED: return "request refused by admission control";
        case NTT_ERR_CANCELLED: return "request cancelled";
        case NTT_ERR_PENDING: return "request pending";
        case NTT_ERR_FAILED: return "request failed";
        case NTT_ERR_INPUT: return "input residue outside the accepted range";
        default: return "unknown status";
    }
}

const char *ntt_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int ntt_is_prime(uint64_t n, int *is_prime) {
    if (!is_prime) return NTT_ERR_ARG;
    *is_prime = nt::is_prime(n) ? 1 : 0;
    return NTT_OK;
}

int ntt_root_of_unity(uint64_t p, uint64_t L, uint64_t *omega) {
    if (!omega) return NTT_ERR_ARG;
    if (p < 3 || !nt::is_prime(p)) return NTT_ERR_MODULUS;
    if (L < 1 || (L & (L - 1)) || (p - 1) % L) return NTT_ERR_LENGTH;
    const uint64_t g = nt::smallest_qnr(p);
    *omega = nt::powmod(g, (p - 1) / L, p);
    return NTT_OK;
}

int ntt_find_prime(uint64_t lo, int k, uint64_t *q) {
    if (!q || k < 1 || k > 62) return NTT_ERR_ARG;
    const uint64_t step = 1ull << k;
    uint64_t c = (lo / step) * step + 1;
    while (c <= lo) c += step;
    for (; c > lo; c += step) {
        if (nt::is_prime(c)) {
            *q = c;
            return NTT_OK;
        }
    }
    return NTT_ERR_RANGE;
}

// Load every pass kernel of the plan's word size and current variant, both
// directions, at set-up time: under CUDA's lazy module loading a kernel is
// otherwise loaded at its first launch, inside whatever latency-sensitive
// call (a server batch, an allocation-free product) makes it.
static int preload_kernels(const ntt_plan_s *pl) {
    LaunchSpec s;
    memset(&s, 0, sizeof(s));
    for (int dir = 0; dir < 2; ++dir) {
        cudaError_t e = launch(pl, s, KIND_PRELOAD, dir, 0);
        if (e != cudaSuccess) return cuda_fail(e, "kernel preload");
    }
    return NTT_OK;
}

int ntt_plan_words(ntt_plan_t *out, uint64_t p, uint64_t omega, uint64_t L, int word_bytes) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    if (word_bytes != 4 && word_bytes != 8) return NTT_ERR_ARG;
    const uint64_t pmax = word_bytes == 4 ? (uint64_t)NTT_P_MAX_W32 : (uint64_t)NTT_P_MAX_W64;
    if (p < 3 || p > pmax || !nt::is_prime(p)) return NTT_ERR_MODULUS;
    if (L < 2 || (L & (L - 1))) return NTT_ERR_LENGTH;
    if (L > (1ull << 26)) return NTT_ERR_RANGE;
    if ((p - 1) % L) return NTT_ERR_LENGTH;
    if (omega == 0 || omega >= p || nt::powmod(omega, L / 2, p) != p - 1) return NTT_ERR_ROOT;
    ntt_plan_s *pl = new (std::nothrow) ntt_plan_s();
    if (!pl) return NTT_ERR_NOMEM;
    pl->p = p;
    pl->omega = omega;
    pl->omega_inv = nt::powmod(omega, p - 2, p);
    pl->L = L;
    pl->L_inv = nt::powmod(L % p, p - 2, p);
    pl->logL = ilog2u(L);
    pl->wbytes = word_bytes;
    pl->variant = variant_fits(pl, NTT_VARIANT_LAZY)  ? NTT_VARIANT_LAZY
                  : variant_fits(pl, NTT_VARIANT_NTL) ? NTT_VARIANT_NTL
                                                      : NTT_VARIANT_MOLLER;
    {
        uint64_t inv = 1;  // p^-1 mod 2^64 by Newton's iteration (p odd); its low word is p^-1 mod 2^32
        for (int i = 0; i < 6; ++i) inv *= 2 - p * inv;
        pl->J = pl->wbytes == 4 ? (inv & 0xffffffffu) : inv;
    }
    cudaGetDevice(&pl->device);
    {
        int *word = nullptr;  // the pass kernels' status word on this device (a lookup, no allocation)
        cudaError_t e = pass_status(&word);
        if (e != cudaSuccess) {
            delete pl;
            return cuda_fail(e, "status word");
        }
    }
    int logr[kMaxPasses];
    int n = default_split(pl->logL, pl->wbytes, logr);
    int rc = apply_split(pl, n, logr);
    if (rc == NTT_OK) rc = preload_kernels(pl);
    if (rc) {
        free_tables(pl);
        delete pl;
        return rc;
    }
    *out = pl;
    return NTT_OK;
}

int ntt_plan(ntt_plan_t *out, uint64_t p, uint64_t omega, uint64_t L) {
    return ntt_plan_words(out, p, omega, L, p < (1ull << 30) ? 4 : 8);
}

int ntt_plan_destroy(ntt_plan_t pl) {
    if (!pl) return NTT_ERR_ARG;
    cudaDeviceSynchronize();
    free_tables(pl);
    release_host_pipeline(pl);
    if (pl->check_word) cudaFree(pl->check_word);
    delete pl;
    return NTT_OK;
}

int ntt_plan_set_variant(ntt_plan_t pl, int variant) {
    if (!pl || variant < NTT_VARIANT_LAZY || variant > NTT_VARIANT_MOLLER) return NTT_ERR_ARG;
    if (!variant_fits(pl, variant)) return NTT_ERR_MODULUS;
    if (variant == NTT_VARIANT_MONT && !pl->mont) {
        std::lock_guard<std::mutex> lk(pl->mu);
        int rc = build_tables_form(pl, true);
        if (rc) return rc;
    }
    const bool changed = pl->variant != variant;
    pl->variant = variant;
    return changed ? preload_kernels(pl) : NTT_OK;
}

int ntt_plan_get_info(ntt_plan_t pl, ntt_plan_info_t *info) {
    if (!pl || !info) return NTT_ERR_ARG;
    memset(info, 0, sizeof(*info));
    info->p = pl->p;
    info->omega = pl->omega;
    info->omega_inv = pl->omega_inv;
    info->L = pl->L;
    info->L_inv = pl->L_inv;
    info->log_L = pl->logL;
    info->word_bytes = pl->wbytes;
    info->variant = pl->variant;
    info->n_passes = pl->npass;
    for (int q = 0; q < pl->npass && q < 4; ++q) info->log_r[q] = pl->pass[q].logR;
    info->table_bytes = pl->table_bytes;
    return NTT_OK;
}

int ntt_plan_set_split(ntt_plan_t pl, int n_passes, const int *log_r) {
    if (!pl || !log_r) return NTT_ERR_ARG;
    if (!split_allowed(pl->logL, pl->wbytes, n_passes, log_r)) return NTT_ERR_ARG;
    cudaDeviceSynchronize();
    return apply_split(pl, n_passes, log_r);
}

static int check_batch_args(ntt_plan_t pl, const void *d, size_t batch, size_t stride) {
    if (!pl || !d || batch == 0) return NTT_ERR_ARG;
    if (stride < pl->L) return NTT_ERR_ARG;
    if (((uintptr_t)d & 15) || ((stride * pl->wbytes) & 15)) return NTT_ERR_ALIGN;
    if (batch > (1ull << 31) / std::max<uint64_t>(1, pl->L / 8)) return NTT_ERR_RANGE;
    return NTT_OK;
}

int ntt_check_input(ntt_plan_t pl, int inverse, const void *d_data, size_t batch, size_t stride_words, void *stream,
                    long long *first_bad) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc) return rc;
    if ((inverse != 0 && inverse != 1) || !first_bad) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(pl->mu);
    cudaError_t e = cudaSuccess;
    if (!pl->check_word) {
        e = cudaMalloc(&pl->check_word, sizeof(unsigned long long));
        if (e != cudaSuccess) {
            pl->check_word = nullptr;
            return e == cudaErrorMemoryAllocation ? NTT_ERR_NOMEM : cuda_fail(e, "check word");
        }
    }
    unsigned long long *word = static_cast<unsigned long long *>(pl->check_word);
    const bool reduced = pl->variant == NTT_VARIANT_NTL || pl->variant == NTT_VARIANT_MOLLER;
    const uint64_t bound = reduced ? pl->p : (inverse ? 4 : 2) * pl->p;
    const uint64_t total = (uint64_t)batch * pl->L;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, 152 * 8);
    e = cudaMemsetAsync(word, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "check memset");
    if (pl->wbytes == 4)
        k_check_input<uint32_t><<<grid, 256, 0, st>>>(static_cast<const uint32_t *>(d_data), stride_words, pl->logL,
                                                      total, (uint32_t)bound, word);
    else
        k_check_input<uint64_t><<<grid, 256, 0, st>>>(static_cast<const uint64_t *>(d_data), stride_words, pl->logL,
                                                      total, bound, word);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "check launch");
    unsigned long long h = ~0ull;
    e = cudaMemcpyAsync(&h, word, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "check result");
    *first_bad = h == ~0ull ? -1 : (long long)h;
    return NTT_OK;
}

int ntt_plan_set_warp_rows(ntt_plan_t pl, int on) {
    if (!pl) return NTT_ERR_ARG;
    pl->warp_rows = on != 0;
    return NTT_OK;
}

int ntt_plan_set_checked(ntt_plan_t pl, int on) {
    if (!pl) return NTT_ERR_ARG;
    pl->checked = on != 0;
    return NTT_OK;
}

// Checked mode: the input-range check before a transform.
static int checked_gate(ntt_plan_t pl, int inverse, const void *d, size_t batch, size_t stride, void *stream) {
    if (!pl->checked) return NTT_OK;
    long long bad = -1;
    int rc = ntt_check_input(pl, inverse, d, batch, stride, stream, &bad);
    if (rc) return rc;
    return bad < 0 ? NTT_OK : NTT_ERR_INPUT;
}

int ntt_forward_batch(ntt_plan_t pl, void *d_data, size_t batch, size_t stride_words, void *stream) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc == NTT_OK) rc = checked_gate(pl, 0, d_data, batch, stride_words, stream);
    if (rc) return rc;
    return enqueue_transform(pl, 0, d_data, batch, stride_words, (cudaStream_t)stream);
}

int ntt_inverse_batch(ntt_plan_t pl, void *d_data, size_t batch, size_t stride_words, void *stream) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc == NTT_OK) rc = checked_gate(pl, 1, d_data, batch, stride_words, stream);
    if (rc) return rc;
    return enqueue_transform(pl, 1, d_data, batch, stride_words, (cudaStream_t)stream);
}

int ntt_selftest_geometry(long long *n_checked, char *msg, int msg_len) {
    if (!n_checked) return NTT_ERR_ARG;
    *n_checked = 0;
    if (msg && msg_len > 0) msg[0] = 0;
    for (int wb : {4, 8}) {
        for (int logL = 3; logL <= 26; ++logL) {
            std::vector<std::vector<int>> splits;
            for (int a = 3; a <= 11; ++a) {
                splits.push_back({a, logL - a});
                for (int b = 3; b <= 11; ++b) {
                    splits.push_back({a, b, logL - a - b});
                    for (int c = 3; c <= 11; ++c) splits.push_back({a, b, c, logL - a - b - c});
                }
            }
            splits.push_back({logL});
            for (const auto &sp : splits) {
                if (!split_allowed(logL, wb, (int)sp.size(), sp.data())) continue;
                ntt_plan_s pl;
                pl.logL = logL;
                pl.L = 1ull << logL;
                pl.wbytes = wb;
                set_geometry(&pl, (int)sp.size(), sp.data());
                for (uint64_t batch : {1ull, 2ull, 3ull, 5ull, 64ull, 1000ull, 1ull << 14}) {
                    if (batch > (1ull << 31) / std::max<uint64_t>(1, pl.L / 8)) continue;  // the API's batch limit
                    for (int q = 0; q < pl.npass; ++q) {
                        for (bool persistent : {false, true}) {
                            if (persistent && (wb != 4 || logL > 16 || batch != 1)) continue;  // uneven batches
                            ++*n_checked;
                            if (!geometry_ok(pl, q, batch, persistent, msg, msg_len)) return NTT_ERR_RANGE;
                        }
                    }
                }
            }
        }
    }
    return NTT_OK;
}

int ntt_forward_dit_batch(ntt_plan_t pl, void *d_data, size_t batch, size_t stride_words, void *stream) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc == NTT_OK) rc = checked_gate(pl, 1, d_data, batch, stride_words, stream);  // Algorithm 4's input range
    if (rc) return rc;
    return enqueue_steps_roots(pl, 1, 0, d_data, batch, stride_words, (cudaStream_t)stream, 0,
                               pl->logL <= 2 ? 1 : pl->npass);
}

int ntt_inverse_dif_batch(ntt_plan_t pl, void *d_data, size_t batch, size_t stride_words, void *stream) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc == NTT_OK) rc = checked_gate(pl, 0, d_data, batch, stride_words, stream);  // Algorithm 3's input range
    if (rc) return rc;
    return enqueue_steps_roots(pl, 0, 1, d_data, batch, stride_words, (cudaStream_t)stream, 0,
                               pl->logL <= 2 ? 1 : pl->npass);
}

int ntt_execute_step(ntt_plan_t pl, int inverse, int step, void *d_data, size_t batch, size_t stride_words,
                     void *stream) {
    int rc = check_batch_args(pl, d_data, batch, stride_words);
    if (rc) return rc;
    const int n = pl->logL <= 2 ? 1 : pl->npass;
    if ((inverse != 0 && inverse != 1) || step < 0 || step >= n) return NTT_ERR_ARG;
    return enqueue_steps(pl, inverse, d_data, batch, stride_words, (cudaStream_t)stream, step, 1);
}

}  // extern "C"
