// ntt_internal.hpp -- host-side structures shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/ntt_gb300.h"

namespace ntt {

constexpr int kMaxPasses = 4;
constexpr int kMaxRowLog = 11;  // longest on-chip sub-transform of a row pass
constexpr int kMaxColLog = 11;  // longest column-pass sub-transform

// Host number theory (the library's own; independent of any test code).
namespace nt {
uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p);
uint64_t powmod(uint64_t a, uint64_t e, uint64_t p);
bool is_prime(uint64_t n);
uint64_t smallest_qnr(uint64_t p);
uint64_t shoup_quotient(uint64_t w, uint64_t p, int word_bits);  // floor(w * beta / p)
uint32_t bitrev(uint32_t k, int bits);
}  // namespace nt

struct PassPlan {
    int logR = 0;   // sub-transform length
    int logS = 0;   // column stride (0: row pass)
    int logTV = 3;  // column pass: 16-byte vectors per tile row
    int logTA = 0;  // column pass: MA table width
    bool has_mb = false;
    void *ma[2] = {nullptr, nullptr};  // [direction] middle tables
    void *mb[2] = {nullptr, nullptr};
    void *mam[2] = {nullptr, nullptr};  // the same in Montgomery form (second word beta W mod p)
    void *mbm[2] = {nullptr, nullptr};
};

}  // namespace ntt

struct ntt_plan_s {
    uint64_t p = 0, omega = 0, omega_inv = 0, L = 0, L_inv = 0;
    int logL = 0;
    int wbytes = 4;
    int variant = NTT_VARIANT_LAZY;
    int device = 0;
    int npass = 0;
    ntt::PassPlan pass[ntt::kMaxPasses];
    void *tw[2] = {nullptr, nullptr};  // stage tables per direction
    void *twm[2] = {nullptr, nullptr}; // the same in Montgomery form (built on first use)
    bool mont = false;                 // Montgomery tables present
    uint64_t J = 0;                    // p^-1 mod beta
    int tw_log = 0;                    // tables cover distances m < 2^tw_log
    uint64_t table_bytes = 0;
    // host-buffer staging (ntt_transform_host): a device copy of the batch,
    // and the copy-in / copy-out streams and events of its chunk pipeline
    void *stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t hs_in = nullptr, hs_out = nullptr;
    cudaEvent_t hev_start = nullptr, hev_end = nullptr;
    cudaEvent_t hev_in[16] = {}, hev_done[16] = {};
    bool warp_rows = false;      // row passes of 2^5..2^10 words run one warp per row (ntt_plan_set_warp_rows)
    bool checked = false;        // checked mode: validate input ranges before each transform
    void *check_word = nullptr;  // device word of ntt_check_input (allocated on first use)
    std::mutex mu;
};

namespace ntt {

// Launch of one pass (kind: 0 column pass, 1 row pass, 2 tiny length 2/4,
// 3 row pass with one warp per row).
// Defined per word type in ntt_pass_u32.cu / ntt_pass_u64.cu.
struct LaunchSpec {
    void *data;
    uint64_t stride;
    uint32_t batch;
    int logL, logR, logS, logTV, logTA;
    int per_cta;          // column pass: sub-tiles per CTA iteration; row pass: rows per iteration
    uint32_t ntiles;      // CTA iterations of the pass
    uint32_t buf_chunks;  // 16-byte chunks of one shared-memory tile buffer
    uint32_t flags;
    const void *tw, *ma, *mb;
    uint64_t p;
    uint64_t J;           // p^-1 mod beta (Montgomery variant)
    uint64_t nrows;
    unsigned grid;  // tiny kernel only
    size_t smem;    // dynamic shared memory of the launch
    int *status;    // device status word of the pass kernels
    long long wait_budget;  // clock cycles a pass kernel waits for one tile copy
    uint32_t tx_extra;      // extra bytes each tile copy expects (a test hook; 0)
    CUtensorMap map;  // column tiles by tensor copies (flag 8): the column view of the data
};

// Tile geometry of pass q of a plan for a batch (or, for a row pass over
// single-row transforms, `rows` rows): fills logTV, per_cta, ntiles,
// buf_chunks and nrows of the spec.
// persistent: geometry for the uneven-batch kernel (column tiles of at most
// 2048 vectors, its two buffers); otherwise for k_pass.
void tile_params(const ntt_plan_s *pl, int q, uint64_t batch, LaunchSpec &s, bool persistent = false);
// kind: 0 column pass, 1 row pass, 2 tiny transform, 3 row pass with one
// warp per row; KIND_PRELOAD loads every pass kernel of (word, dir, var).
constexpr int KIND_PRELOAD = -1;
cudaError_t launch_pass_u32(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st);
cudaError_t launch_pass_u64(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st);

// Enqueue a whole forward or inverse transform of a batch (all passes).
int enqueue_transform(ntt_plan_s *plan, int dir, void *data, size_t batch, size_t stride, cudaStream_t st);

// Enqueue execution steps first .. first+count-1 of a transform (a step is
// one pass; the inverse executes the passes in reverse order).
// The same with the twiddle tables of root direction `roots` (0: omega,
// 1: omega^-1) in the schedule of direction `dir`: dir = 1, roots = 0 is the
// forward transform from bit-reversed to natural order (DIT), dir = 0,
// roots = 1 the inverse from natural to bit-reversed order (DIF).
int enqueue_steps_roots(ntt_plan_s *plan, int dir, int roots, void *data, size_t batch, size_t stride,
                        cudaStream_t st, int first, int count);

int enqueue_steps(ntt_plan_s *plan, int dir, void *data, size_t batch, size_t stride, cudaStream_t st, int first,
                  int count);

// Whether a pass split is allowed for a transform of 2^logL words of wbytes.
bool split_allowed(int logL, int wbytes, int n, const int *logr);

// Whether a butterfly variant's modulus bound holds for the plan's p and word.
bool variant_fits(const ntt_plan_s *pl, int variant);

// Free the prepared uneven batches whose transforms all lie in [lo, hi).
void uneven_release_range(const void *lo, const void *hi);

// Free the staging buffer, streams and events of ntt_transform_host.
void release_host_pipeline(ntt_plan_s *plan);

// Stream-ordered scratch for the library's own calls (polymul_mod_p,
// bigint_mul): a memory pool per device that keeps up to 4 GiB reserved
// between calls instead of returning it to the driver at every
// synchronisation (re-mapping a large slab costs milliseconds).
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st);

// Record a CUDA failure for ntt_last_cuda_error(); returns NTT_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *where);

}  // namespace ntt
