/*
 * ntt_gb300.h -- C ABI of the GB300 (sm_103a) batched number-theoretic
 * transform library.
 *
 * The transform (Harvey, "Faster arithmetic for number-theoretic transforms",
 * arXiv:1205.2926, Section 1): for a word-sized prime p with p = 1 mod L,
 * L = 2^l, and a primitive L-th root of unity omega,
 *      b_j = sum_{i<L} omega^(i j) a_i  (mod p),   0 <= j < L,
 * computed by the radix-2 schedule of Algorithm 1, whose output is in
 * bit-reversed order: position k holds b_{rev_l(k)}.
 *
 * Arithmetic (Sections 2-4): butterflies use Shoup's product with a
 * precomputed quotient W' = floor(W beta / p) and keep residues redundant,
 * in [0, 2p) for the forward butterfly (Algorithm 3) and [0, 4p) for the
 * inverse butterfly (Algorithm 4); one final reduction returns [0, p).  The
 * fully reduced butterfly of Algorithm 2 is available as a comparison
 * variant.  The word size beta follows from p:
 *      p < 2^30  ->  beta = 2^32, data words are uint32_t;
 *      p < 2^62  ->  beta = 2^64, data words are uint64_t.
 * (Algorithms 3 and 4 need p < beta/4.)
 *
 * Conventions for every entry point:
 *  - Return value: NTT_OK (0) or a negative NTT_ERR_* code; nothing throws and
 *    nothing aborts.  ntt_strerror() names a code.
 *  - Device pointers are CUDA device (or managed) memory on the device that
 *    was current when the plan was made; the caller owns them.  They must be
 *    16-byte aligned (NTT_ERR_ALIGN otherwise).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Transform calls are asynchronous on that stream: they return
 *    after enqueueing, and errors of the kernels themselves surface at the
 *    caller's next synchronisation.
 *  - Plans own their device tables; a plan may be used from one host thread
 *    at a time and by any number of streams (the tables are read-only).
 */
#ifndef NTT_GB300_H
#define NTT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define NTT_OK 0
#define NTT_ERR_MODULUS -1   /* p not prime, p >= 2^62, or p even */
#define NTT_ERR_LENGTH -2    /* L not a power of two, L < 2, or L does not divide p-1 */
#define NTT_ERR_ROOT -3      /* omega^L != 1 or omega^(L/2) != p-1 */
#define NTT_ERR_ARG -4       /* null pointer, zero size, stride < L, bad enum */
#define NTT_ERR_CUDA -5      /* a CUDA runtime call failed (see ntt_last_cuda_error) */
#define NTT_ERR_NOMEM -6     /* device or host allocation failed */
#define NTT_ERR_TIMEOUT -7   /* a bounded device-side wait gave up */
#define NTT_ERR_ALIGN -8     /* pointer or stride not 16-byte aligned */
#define NTT_ERR_RANGE -9     /* size beyond a documented maximum */
#define NTT_ERR_REFUSED -10  /* server: request refused by admission (too large for the memory budget) */
#define NTT_ERR_CANCELLED -11 /* server: request was cancelled */
#define NTT_ERR_PENDING -12  /* server: request not finished yet */
#define NTT_ERR_FAILED -13   /* server: request failed */
#define NTT_ERR_INPUT -14    /* checked mode: an input residue lies outside the accepted range */

/* Butterfly variants (ntt_plan_set_variant). */
#define NTT_VARIANT_LAZY 0 /* Algorithms 3 (forward) and 4 (inverse), redundant residues */
#define NTT_VARIANT_NTL 1  /* Algorithm 2 and its fully reduced inverse (comparison baseline) */
#define NTT_VARIANT_MONT 2 /* Algorithm 5 (Montgomery's product, lazy ranges) and its inverse
                              counterpart (Algorithm 4 with Montgomery's product) */
#define NTT_VARIANT_MOLLER 3 /* Algorithm 2 in Moeller's form (end of Section 2): fully reduced,
                                valid for any p < beta/phi */

/* Largest modulus of each word size: p < beta/phi, phi = (1 + sqrt 5)/2 (Moeller's bound for
 * the fully reduced butterfly; the redundant-residue variants need p < beta/4 and Algorithm 2
 * as printed p < beta/2).  beta/phi is irrational, so p < beta/phi means p <= these values. */
#define NTT_P_MAX_W32 2654435769u                /* floor(2^32 / phi) */
#define NTT_P_MAX_W64 11400714819323198485ull    /* floor(2^64 / phi) */

typedef struct ntt_plan_s *ntt_plan_t;

/* ---------------------------------------------------------- number theory */

/* Deterministic Miller-Rabin test of n (bases: the first twelve primes, exact
 * for every 64-bit n).  *is_prime receives 1 or 0.  Host only. */
int ntt_is_prime(uint64_t n, int *is_prime);

/* Section 1 fixes "one of" the primitive L-th roots; this library's choice is
 * omega = g^((p-1)/L) with g the smallest quadratic non-residue mod p (any
 * odd prime p < 2^64).
 * Errors: NTT_ERR_MODULUS, NTT_ERR_LENGTH.  Host only. */
int ntt_root_of_unity(uint64_t p, uint64_t L, uint64_t *omega);

/* Smallest prime q > lo with q = 1 mod 2^k (deterministic search).  Host only. */
int ntt_find_prime(uint64_t lo, int k, uint64_t *q);

/* ------------------------------------------------------------------ plans */

/* Make a plan for length-L transforms over F_p with root omega (Section 1).
 * Validates p (prime, <= NTT_P_MAX_W64), L (power of two, 2 <= L, L | p-1)
 * and omega (omega^(L/2) = p-1, hence order exactly L), computes omega^-1 and
 * L^-1, and uploads the twiddle tables (W, W') of Algorithms 2-4 for both
 * directions to the current device.  Word size: 32-bit words for p < 2^30
 * (beta/4 at beta = 2^32), 64-bit words otherwise.  The variant starts as
 * NTT_VARIANT_LAZY when p < beta/4, else NTT_VARIANT_NTL when p < beta/2,
 * else NTT_VARIANT_MOLLER.  *out receives the plan; the library owns its
 * memory until ntt_plan_destroy.
 * Errors: NTT_ERR_ARG, NTT_ERR_MODULUS, NTT_ERR_LENGTH, NTT_ERR_ROOT,
 * NTT_ERR_RANGE (L > 2^26), NTT_ERR_NOMEM, NTT_ERR_CUDA. */
int ntt_plan(ntt_plan_t *out, uint64_t p, uint64_t omega, uint64_t L);

/* ntt_plan with the word size chosen by the caller: word_bytes 4 (beta =
 * 2^32, p <= NTT_P_MAX_W32) or 8 (beta = 2^64, p <= NTT_P_MAX_W64).  This is
 * what Moeller's bound buys (end of Section 2): a prime between 2^30 and
 * 2^32/phi still runs on 32-bit words with NTT_VARIANT_MOLLER (or
 * NTT_VARIANT_NTL below 2^31), where the redundant-residue variants would need
 * 64-bit words.  Default variant as for ntt_plan.
 * Errors: as ntt_plan; NTT_ERR_ARG for another word_bytes, NTT_ERR_MODULUS
 * for p beyond the word's bound. */
int ntt_plan_words(ntt_plan_t *out, uint64_t p, uint64_t omega, uint64_t L, int word_bytes);

/* Free a plan and its device tables (synchronises the device first). */
int ntt_plan_destroy(ntt_plan_t plan);

/* Select NTT_VARIANT_LAZY, NTT_VARIANT_NTL, NTT_VARIANT_MONT or
 * NTT_VARIANT_MOLLER for later calls on this plan.  The first selection of
 * NTT_VARIANT_MONT builds the plan's tables in Montgomery form (W' = beta W
 * mod p, Algorithm 5's input), kept beside the Shoup tables until the plan is
 * destroyed or re-split; the variant's input and output ranges are those of
 * NTT_VARIANT_LAZY.  NTT_VARIANT_MOLLER takes and returns fully reduced
 * residues like NTT_VARIANT_NTL.  Each variant's modulus bound (beta the
 * plan's word): LAZY and MONT p < beta/4 (Theorems 2-4), NTL p < beta/2
 * (Theorem 1), MOLLER p < beta/phi.
 * Errors: NTT_ERR_ARG, NTT_ERR_MODULUS (p beyond the variant's bound),
 * NTT_ERR_NOMEM. */
int ntt_plan_set_variant(ntt_plan_t plan, int variant);

/* Choose the kernel of the plan's row pass (the last pass of the forward
 * transform, the first of the inverse; the only pass when L <= 2^11) when its
 * rows have 2^5..2^10 words: on != 0 runs one warp per row, each thread
 * holding R/32 words in registers (stages of distance >= 32 inside a thread,
 * one transpose through the warp's shared memory, the distances from R/32
 * to 16 across lanes by warp shuffles, the rest inside a thread again; in
 * passes of many rows a warp owns several rows at once); 0 (the default)
 * runs the radix-8 CTA rows of the other passes.  Results are identical
 * (Algorithm 1's stages, the same butterflies).  Shorter or longer rows
 * ignore the setting; ntt_plan_autotune sets it by timing.  Errors:
 * NTT_ERR_ARG. */
int ntt_plan_set_warp_rows(ntt_plan_t plan, int on);

/* Read-only description of a plan.  word_bytes is 4 or 8; n_passes is the
 * number of on-chip passes the transform is split into (four-step split of
 * Algorithm 1's stages); log_r[i] is log2 of pass i's sub-transform length;
 * table_bytes counts the plan's device tables. */
typedef struct {
    uint64_t p, omega, omega_inv, L, L_inv;
    int log_L, word_bytes, variant, n_passes;
    int log_r[4];
    uint64_t table_bytes;
} ntt_plan_info_t;
int ntt_plan_get_info(ntt_plan_t plan, ntt_plan_info_t *info);

/* Override the pass split (autotuning; n_passes 1..4, sum of log_r = log L,
 * every log_r[i] in [3, 11], and every column pass (all but the last)
 * followed by at least 2^5 (32-bit words) or 2^4 (64-bit words) elements).
 * Rebuilds the plan's middle-twiddle tables.  NTT_ERR_ARG if the split is not
 * allowed. */
int ntt_plan_set_split(ntt_plan_t plan, int n_passes, const int *log_r);

/* Autotuner: time every allowed pass split of this plan (forward + inverse
 * on a scratch batch of `batch` vectors, CUDA events, after warm-up), keep
 * the fastest; then, when that split's row pass has 2^5..2^10 words, time
 * it once with the radix-8 CTA rows and once with one warp per row
 * (ntt_plan_set_warp_rows) and keep the faster body.  Both choices are
 * stored in a JSON cache keyed by GPU name, word size, log L and
 * log2(batch) ($NTT_AUTOTUNE_CACHE, default ~/.cache/ntt_gb300_autotune.json;
 * the row body under the key + "/warp").  With use_cache != 0 a cached choice
 * for the same key is applied without timing (no "/warp" entry: CTA rows).  log_r_out (may be NULL, else
 * room for 4 ints) receives the chosen split.  Allocates a scratch batch
 * and synchronises; call at set-up time.  Errors: NTT_ERR_ARG, NTT_ERR_NOMEM,
 * NTT_ERR_CUDA. */
int ntt_plan_autotune(ntt_plan_t plan, size_t batch, int use_cache, int *log_r_out);

/* ------------------------------------------------------------- transforms */

/* Forward transform of `batch` vectors in place (Section 1, Algorithm 1 with
 * Algorithm 3 butterflies).  Vector b starts at word b*stride_words of d_data
 * (words are uint32_t or uint64_t per the plan).  Input residues may lie in
 * [0, 2p) for the lazy variant (Algorithm 3's input range) and must lie in
 * [0, p) for NTT_VARIANT_NTL; the output is in [0, p), bit-reversed order.
 * stride_words >= L and stride_words*word_bytes a multiple of 16.
 * 64-bit column passes fetch their tiles by tensor copies whose waits are
 * bounded: a copy that never lands ends the pass early with NTT_ERR_TIMEOUT
 * in the device status word (ntt_pass_status), never a hang.
 * Errors: NTT_ERR_ARG, NTT_ERR_ALIGN, NTT_ERR_CUDA (launch failure). */
int ntt_forward_batch(ntt_plan_t plan, void *d_data, size_t batch, size_t stride_words, void *stream);

/* Inverse transform in place: Algorithm 1 run backwards (Section 4) with the
 * Algorithm 4 butterfly and the inverse root.  Input in bit-reversed order,
 * residues in [0, 4p) (lazy) or [0, p) (NTL); output in natural order in
 * [0, p), UNNORMALISED: inverse(forward(a)) = L * a.  Layout and errors as
 * ntt_forward_batch. */
int ntt_inverse_batch(ntt_plan_t plan, void *d_data, size_t batch, size_t stride_words, void *stream);

/* Input-range check (the checked mode of the library; Algorithms 3 and 4
 * state their input intervals, and outside them the redundant-residue bounds
 * of Theorems 2 and 3 do not hold).  Scans the `batch` vectors of L words at
 * d_data (layout as ntt_forward_batch) for a word >= the bound the plan's
 * variant accepts: 2p for a forward and 4p for an inverse transform with the
 * lazy or Montgomery variant, p with NTT_VARIANT_NTL.  *first_bad receives
 * the smallest flat index b*L + i of such a word, or -1.  Synchronous: runs
 * one kernel on `stream` and waits for it.  Errors: NTT_ERR_ARG,
 * NTT_ERR_ALIGN, NTT_ERR_RANGE, NTT_ERR_NOMEM, NTT_ERR_CUDA. */
int ntt_check_input(ntt_plan_t plan, int inverse, const void *d_data, size_t batch, size_t stride_words,
                    void *stream, long long *first_bad);

/* Checked mode on (on != 0) or off for a plan: ntt_forward_batch and
 * ntt_inverse_batch then run ntt_check_input first (synchronously) and
 * return NTT_ERR_INPUT, leaving the data untouched, when a word is out of
 * range.  Off by default: the unchecked calls are asynchronous and leave
 * out-of-range inputs undefined.  Errors: NTT_ERR_ARG. */
int ntt_plan_set_checked(ntt_plan_t plan, int on);

/* Forward transform from bit-reversed input to natural-order output: the
 * schedule of ntt_inverse_batch (Algorithm 1 run backwards, Section 4, with
 * the Algorithm 4 butterfly) driven by the forward root's tables, so
 * out[i] = sum_j omega^(i j) x[rev(j)]: applied to the bit-reversal of a, the
 * DFT of a in natural order.  The pair ntt_inverse_dif_batch /
 * ntt_forward_dit_batch mirrors ntt_forward_batch / ntt_inverse_batch with
 * the roots exchanged.  Input residues in [0, 4p) (lazy, Montgomery) or [0, p) (NTL);
 * output in [0, p).  Layout and errors as ntt_forward_batch (plus
 * NTT_ERR_INPUT in checked mode). */
int ntt_forward_dit_batch(ntt_plan_t plan, void *d_data, size_t batch, size_t stride_words, void *stream);

/* Inverse transform from natural-order input to bit-reversed output: the
 * schedule of ntt_forward_batch (Algorithm 1, Algorithm 3 butterflies) driven
 * by the inverse root's tables, so position k holds
 * sum_i omega^(-i rev(k)) x[i] (unnormalised).  Input residues in [0, 2p)
 * (lazy, Montgomery) or [0, p) (NTL); output in [0, p).  Layout and errors
 * as ntt_forward_batch. */
int ntt_inverse_dif_batch(ntt_plan_t plan, void *d_data, size_t batch, size_t stride_words, void *stream);

/* Host-only self-test of the launch geometry (no device needed): for every
 * pass split that ntt_plan_set_split accepts, for every length 2^3..2^26, both
 * word sizes and batches of 1 .. 16384 vectors (within the batch limit of the
 * transform calls), checks that the tiles of each pass cover its data
 * exactly once, that each sub-tile's threads form the contiguous block the
 * kernels synchronise, that the shared-memory buffers match the kernels'
 * compile-time layout (padded or not) and fit in 227 KiB, and that 64-bit
 * tensor-copy boxes are well formed.  *n_checked receives the number of
 * (split, pass, batch) cases; on the first violation returns NTT_ERR_RANGE
 * with a description in msg (msg_len bytes, may be NULL).  Returns NTT_OK or
 * NTT_ERR_ARG. */
int ntt_selftest_geometry(long long *n_checked, char *msg, int msg_len);

/* One execution step (one pass, one kernel launch) of a transform: steps
 * 0 .. n_passes-1 run in order are exactly ntt_forward_batch (inverse = 0) or
 * ntt_inverse_batch (inverse = 1); intermediate contents between steps are
 * residues in the redundant range and in the four-step intermediate order.
 * For profiling and per-kernel timing.  Errors as ntt_forward_batch, plus
 * NTT_ERR_ARG for a step outside [0, n_passes). */
int ntt_execute_step(ntt_plan_t plan, int inverse, int step, void *d_data, size_t batch, size_t stride_words,
                     void *stream);

/* Same transforms on HOST buffers (Algorithm 1 / its inverse as above).
 * h_data holds batch*stride_words words.  The batch is copied to a device
 * buffer owned by the plan (grown on demand), transformed on `stream`, and
 * copied back; the call returns after `stream` has finished.  A batch of
 * several transforms is cut into chunks of whole transforms (at most 16,
 * about 2 MiB each) so that copy-in, transform and copy-out of different
 * chunks overlap on the plan's two copy streams.  Work queued earlier on
 * `stream` completes before the first copy.  `inverse` is 0 or 1.  With
 * pinned host memory the copies are asynchronous DMA; any host memory works.
 * Calls on one plan serialise (a plan mutex); calls on different plans from
 * different threads run concurrently.
 * Errors: as above plus NTT_ERR_NOMEM. */
int ntt_transform_host(ntt_plan_t plan, int inverse, void *h_data, size_t batch, size_t stride_words,
                       void *stream);

/* ------------------------------------------------- polynomial products */

/* c = a * b in F_p[x] (the polynomial-multiplication application, Section 1):
 * zero-pad both operands to L = nextpow2(na + nb - 1), forward transforms,
 * pointwise product times L^-1 (Montgomery reduction as in Algorithm 5, then
 * a Shoup product by L^-1, reduced to [0, p)), inverse transform.  a, b, c are DEVICE arrays of
 * natural-order coefficients in [0, p) in the word type of p; c receives
 * na + nb - 1 words.  omega is the library's root for (p, L).  Plans are
 * cached per (device, p, L); device scratch of 2*L words is allocated per
 * call (stream-ordered, from a library pool per device that keeps up to
 * 4 GiB reserved between calls) and released on the stream.  Asynchronous on
 * `stream`.
 * Errors: NTT_ERR_ARG (null, na or nb zero), NTT_ERR_LENGTH (L does not divide
 * p-1), NTT_ERR_MODULUS, NTT_ERR_ALIGN, NTT_ERR_NOMEM, NTT_ERR_CUDA. */
int polymul_mod_p(uint64_t p, const void *d_a, size_t na, const void *d_b, size_t nb, void *d_c, void *stream);

/* Size of the fixed device scratch of polymul_mod_p_noalloc, in bytes. */
#define NTT_NOALLOC_SCRATCH_BYTES (8u << 20)

/* polymul_mod_p for callers that must not allocate device memory while they
 * run.  The paper has no counterpart; this is a library-level variant.  Who
 * needs it: code whose device memory belongs to another allocator (a
 * framework's caching allocator or a fixed arena) and may not allocate
 * behind its back, and latency-critical paths where a cudaMalloc or
 * cudaMallocAsync could block, synchronise or fail under memory pressure.
 * This call allocates nothing: its scratch (the two zero-padded operands,
 * 2 L words) is a file-scope __device__ array of NTT_NOALLOC_SCRATCH_BYTES
 * (8 MiB) that every GPU loading the library holds until the process exits.
 * Sizes: 2 * L * word_bytes must fit, i.e. L <= 2^20 for 32-bit words and
 * L <= 2^19 for 64-bit words; larger requests return NTT_ERR_RANGE.
 * `plan` is made beforehand with ntt_plan (that call does allocate, so make
 * it at set-up time) for the modulus, any primitive L-th root and a length
 * L >= na + nb - 1; it must use NTT_VARIANT_LAZY and belong to the current
 * device.  a, b, c are device arrays as for polymul_mod_p; the result equals
 * polymul_mod_p's.  What the first call on a device does: it looks up the
 * address of the scratch array on that device with cudaGetSymbolAddress
 * (set-up done once per device, no allocation; under CUDA's lazy module
 * loading that lookup is when the driver places the library's module, array
 * included, in device memory); make that first call before any stream
 * capture.  The transform kernels' status word is likewise a __device__
 * word, looked up by ntt_plan, so no later call allocates it.  Every call
 * on a device shares the
 * one scratch array and leaves its contents behind (each call rewrites all
 * of it before use): calls whose work overlaps on the GPU -- different
 * streams, or different host threads -- race and give wrong results, so
 * serialise them (one stream, or events).  Asynchronous on `stream`.
 * Errors: NTT_ERR_ARG (null pointer, na or nb zero, NTL plan, plan of
 * another device, device index 64 or above), NTT_ERR_LENGTH
 * (L < na + nb - 1), NTT_ERR_RANGE (scratch too small), NTT_ERR_ALIGN,
 * NTT_ERR_CUDA. */
int polymul_mod_p_noalloc(ntt_plan_t plan, const void *d_a, size_t na, const void *d_b, size_t nb, void *d_c,
                          void *stream);

/* ----------------------------------------------------- big-integer products */

/* c = a * b for non-negative integers given as little-endian arrays of
 * 32-bit limbs (device pointers; the application named in Section 1:
 * integers multiplied as polynomials evaluated at 2^32).  The coefficients of
 * the polynomial product are below min(na, nb) (2^32 - 1)^2 < 2^86; they are
 * computed by three polynomial products modulo 998244353, 167772161 and
 * 469762049 (forward transforms with Algorithm 3, pointwise product,
 * inverse transform with Algorithm 4), combined by Chinese remaindering
 * (Garner's form), and their words summed with a parallel carry scan.
 * c receives na + nb limbs (the top one may be 0); a and b are not modified
 * and may not overlap c.  Limits: na + nb - 1 <= 2^23.  Device scratch of
 * 24 (nextpow2(na + nb - 1)) bytes comes stream-ordered from the same
 * library pool as polymul_mod_p's.
 * Asynchronous on `stream`.
 * Errors: NTT_ERR_ARG (null pointer or zero length), NTT_ERR_RANGE, NTT_ERR_NOMEM,
 * NTT_ERR_CUDA. */
int bigint_mul(const uint32_t *d_a, size_t na, const uint32_t *d_b, size_t nb, uint32_t *d_c, void *stream);

/* ------------------------------------------------------------- uneven batch */

/* One transform of an uneven batch: its plan, its device vector (L words of
 * the plan's word type, 16-byte aligned) and its direction (0 forward,
 * 1 inverse).  Plans may differ in p and L; all must use 32-bit words and one
 * butterfly variant, NTT_VARIANT_LAZY (Algorithms 3-4) or NTT_VARIANT_NTL
 * (Algorithm 2), and live on the current device. */
typedef struct {
    ntt_plan_t plan;
    void *d_data;
    int inverse;
} ntt_desc_t;

/* Run every transform of `descs` in ONE persistent kernel launch: the work is
 * cut into tiles of every pass of every transform, tiles are handed out by a
 * device-side atomic counter in dependency order, and a tile of a later pass
 * waits (bounded by a clock budget) for the tiles of the earlier pass of the
 * same transform.  Results are those of ntt_forward_batch/ntt_inverse_batch
 * on each transform alone.  Host-side preparation (the work list's upload,
 * synchronous) is cached per distinct batch (descs array contents and the
 * plans' splits): calling again with the same batch reuses it, so the call
 * can be captured in a CUDA graph after a first call outside the capture.
 * Every batch prepared on a device stays prepared (a few bytes of device
 * memory per work item) until ntt_uneven_release, so graphs that captured
 * different batches stay valid side by side.
 * Errors: NTT_ERR_ARG (also plans of different variants in one batch),
 * NTT_ERR_RANGE (a 64-bit plan, a variant other than LAZY or NTL, L > 2^22),
 * NTT_ERR_CUDA, NTT_ERR_TIMEOUT (reported by ntt_uneven_status when a wait
 * gave up). */
int ntt_execute_uneven(const ntt_desc_t *descs, size_t n, void *stream);

/* Autotuner for uneven batches: pick the pass split of every multi-pass
 * length class (one class per length L > 2^11: every plan of that length,
 * whatever its prime) by timing the persistent launch of this batch's layout,
 * one class at a time (longest first) over every two-pass split the
 * persistent kernel carries, the other classes fixed.  The chosen splits are
 * applied to the plans (ntt_plan_set_split: later calls on those plans use
 * them) and cached per (GPU model, word size, log L, log2 of the class's
 * transform count) under "uneven/..." keys of the autotune cache
 * file (NTT_AUTOTUNE_CACHE, else ~/.cache/ntt_gb300_autotune.json).  With
 * use_cache != 0 and every class cached, the cached splits are applied
 * without timing.  Timing runs on a scratch copy of the batch's layout
 * (allocated and freed here; the caller's data are not touched) on `stream`,
 * and synchronises it.  A prepared batch whose plans changed split since it
 * was prepared is prepared again by the next ntt_execute_uneven.
 * Errors: NTT_ERR_ARG, NTT_ERR_NOMEM, NTT_ERR_CUDA, and those of
 * ntt_execute_uneven. */
int ntt_uneven_autotune(const ntt_desc_t *descs, size_t n, int use_cache, void *stream);

/* Free every batch prepared by ntt_execute_uneven on the current device
 * (synchronises the device first).  Graphs that captured one of them must not
 * be replayed afterwards.  Errors: NTT_ERR_CUDA. */
int ntt_uneven_release(void);

/* Status word of the last ntt_execute_uneven on this device, read after the
 * stream has been synchronised: NTT_OK or NTT_ERR_TIMEOUT. */
int ntt_uneven_status(int *status);

/* Failure-detection hook for tests and operators: set the clock-cycle budget
 * of every device-side wait of ntt_execute_uneven (default 2e9, about one
 * second) and, when stall_stage >= 1, make every wait of that stage ask for
 * one completion more than can ever arrive, so that the wait runs out and
 * the launch ends with status NTT_ERR_TIMEOUT instead of hanging.
 * stall_stage = -1 restores normal waits.  Takes effect at the next launch
 * (a prepared batch keeps no copy of these values). */
int ntt_uneven_set_wait_budget(long long cycles, int stall_stage);

/* Status word of the pass kernels on the current device (synchronous read):
 * NTT_OK, or NTT_ERR_TIMEOUT when a pass kernel gave up waiting for one of
 * its tile copies (64-bit column passes fetch tiles by tensor copies that
 * complete on an mbarrier; every wait is bounded, after which the kernel
 * records the timeout and returns instead of hanging; its output is then
 * invalid).  reset != 0 clears the word after reading it.  Returns NTT_OK or
 * NTT_ERR_ARG / NTT_ERR_CUDA. */
int ntt_pass_status(int reset, int *status);

/* Failure-detection hook for tests and operators: set the clock-cycle budget
 * of each tile-copy wait of the pass kernels (default 2e9, about one second)
 * and, with stall_bytes > 0 (a multiple of 16, at most 65536), make every
 * tile copy expect that many bytes more than can ever arrive, so that its
 * wait runs out and ntt_pass_status reports NTT_ERR_TIMEOUT instead of the
 * kernel hanging.  stall_bytes = 0 restores normal waits.  Takes effect at
 * the next launch; a captured CUDA graph keeps the values it was captured
 * with. */
int ntt_pass_set_wait_budget(long long cycles, unsigned int stall_bytes);

/* -------------------------------------------------- polymul serving loop */

/* A continuous-batching server of polynomial products mod p (the Section 1
 * application under a request stream).  A scheduler thread admits queued
 * requests in FIFO order while their device memory (2 L words each) fits in
 * mem_budget_bytes, groups them by L = nextpow2(na+nb-1), and runs each group
 * as one batch (forward transforms of both operands, pointwise product times
 * L^-1, inverse transform) on the one of n_streams CUDA streams with the
 * least outstanding work (butterflies of its running batches).  Requests
 * arriving while batches run are admitted as memory frees up, and their
 * batches overlap with the running ones on the device.  Each result is the
 * same as polymul_mod_p on that request alone.
 * Host buffers: when both operands and the result of every request of a
 * batch are in page-locked memory (cudaHostAlloc, cudaHostRegister, torch
 * pin_memory), kernels gather the operands into the device slab and scatter
 * the results back through unified addressing, with no per-request copy
 * call; otherwise each operand and result is one cudaMemcpyAsync.  The
 * server's memory pool maps min(mem_budget_bytes, 4 GiB) at creation and
 * keeps up to mem_budget_bytes mapped between batches. */
typedef struct ntt_server_s *ntt_server_t;

typedef struct {
    uint64_t p;              /* prime modulus (word type as for plans) */
    size_t max_coeffs;       /* largest accepted na or nb */
    size_t mem_budget_bytes; /* device bytes for admitted, unfinished requests */
    int n_streams;           /* concurrent CUDA streams, 1..64 */
    int max_batch;           /* most requests of one length per batch */
    int variant;             /* butterflies of the server's transforms: NTT_VARIANT_LAZY (0, the
                                default, Algorithms 3-4) or NTT_VARIANT_NTL (Algorithm 2) */
} ntt_server_config_t;

typedef struct {
    uint64_t completed, refused, cancelled, failed, batches;
    double butterflies;                      /* transform butterflies of completed requests */
    double p50_us, p99_us, mean_us, max_us;  /* submit-to-result latency of completed requests */
    double wall_s;                           /* first submit to last completion */
    uint64_t direct_batches;                 /* batches whose operands and results were all in
                                                page-locked host memory: gathered and scattered
                                                by kernels, with no per-request copy calls */
} ntt_server_stats_t;

/* Start a server on the current device.  Makes the plan of every transform
 * length it accepts (2 .. nextpow2(2 max_coeffs - 1)) before returning, so
 * that no table upload or kernel load happens while requests are served.
 * Errors: NTT_ERR_ARG (also a variant other than LAZY or NTL), NTT_ERR_MODULUS,
 * NTT_ERR_LENGTH (p has no root of order nextpow2(2*max_coeffs-1)),
 * NTT_ERR_CUDA. */
int ntt_server_create(const ntt_server_config_t *cfg, ntt_server_t *out);

/* Queue c = a * b.  h_a, h_b, h_c are HOST arrays (na, nb and na+nb-1 words
 * of the word type of p, coefficients in [0, p)) that must stay valid and
 * untouched until the request finishes; pinned memory gives asynchronous
 * copies.  *req_id receives the request id even when the request is refused.
 * Returns NTT_OK, or NTT_ERR_REFUSED for a request too large for max_coeffs
 * or the memory budget (or with a length p does not support), or NTT_ERR_ARG. */
int ntt_server_submit(ntt_server_t sv, const void *h_a, size_t na, const void *h_b, size_t nb, void *h_c,
                      uint64_t *req_id);

/* Status of a request: NTT_ERR_PENDING (queued or running), NTT_OK (result
 * written to h_c), NTT_ERR_REFUSED, NTT_ERR_CANCELLED or NTT_ERR_FAILED. */
int ntt_server_poll(ntt_server_t sv, uint64_t req_id, int *status);

/* Block until the request is no longer pending or timeout_ms passes (< 0:
 * no limit); *status as ntt_server_poll. */
int ntt_server_wait(ntt_server_t sv, uint64_t req_id, int timeout_ms, int *status);

/* Cancel a request that is still queued (not yet admitted): NTT_OK; a request
 * already admitted runs to completion and this returns NTT_ERR_PENDING. */
int ntt_server_cancel(ntt_server_t sv, uint64_t req_id);

/* Wait until nothing is queued or running (timeout_ms < 0: no limit);
 * NTT_ERR_PENDING on timeout. */
int ntt_server_drain(ntt_server_t sv, int timeout_ms);

/* Counters and latency percentiles since creation or the last reset. */
int ntt_server_stats(ntt_server_t sv, ntt_server_stats_t *out);
int ntt_server_reset_stats(ntt_server_t sv);

/* Failure injection on the host: the next n_batches batches fail before
 * launch; their requests end NTT_ERR_FAILED and other batches are unaffected. */
int ntt_server_inject_failures(ntt_server_t sv, int n_batches);

/* Finish queued and running work, stop the scheduler, free the server. */
int ntt_server_destroy(ntt_server_t sv);

/* ------------------------------------------------------------------ misc */

/* Human-readable name of a status code (static storage). */
const char *ntt_strerror(int code);

/* The last CUDA error string seen by the library on this host thread. */
const char *ntt_last_cuda_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int ntt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NTT_GB300_H */
