// ntt_polymul.hpp -- internal entry points of the polynomial product, shared
// with the serving loop.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ntt_internal.hpp"

namespace ntt {

// Check (p, na, nb); on success *L_out = max(2, nextpow2(na + nb - 1)).
int polymul_validate(uint64_t p, size_t na, size_t nb, uint64_t *L_out);

// Cached plan for (current device, p, L) with the library's root of unity,
// set to butterfly variant `variant` (-1: the plan's default choice).
int polymul_plan(uint64_t p, uint64_t L, ntt_plan_s **out, int variant = -1);

// Enqueue A <- A B L^-1 mod p over L words (transforms in [0, 2p) from the
// forward pass; result in [0, 2p), the inverse pass's input range).
int enqueue_pointwise(ntt_plan_s *pl, void *A, const void *B, uint64_t L, cudaStream_t st);

// Enqueue c = a * b on `st` using `buf` (2 L words of device scratch).
int enqueue_polymul(ntt_plan_s *pl, const void *a, size_t na, const void *b, size_t nb, void *c, void *buf,
                    cudaStream_t st);

}  // namespace ntt
