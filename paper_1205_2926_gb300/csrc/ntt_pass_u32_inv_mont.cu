// Pass kernels for 32-bit words, inverse direction, mont butterflies.
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u32_inv_mont(const LaunchSpec &s, int kind, cudaStream_t st) {
    return launch_kind<uint32_t, DIR_INV, VAR_MONT>(s, kind, st);
}
}  // namespace ntt
