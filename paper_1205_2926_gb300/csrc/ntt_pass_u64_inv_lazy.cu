// Pass kernels for 64-bit words, inverse direction, lazy butterflies.
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u64_inv_lazy(const LaunchSpec &s, int kind, cudaStream_t st) {
    return launch_kind<uint64_t, DIR_INV, VAR_LAZY>(s, kind, st);
}
}  // namespace ntt
