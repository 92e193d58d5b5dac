// Pass kernels for 32-bit words, inverse direction (own translation
// unit so that the instantiations compile in parallel).
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u32_inv(const LaunchSpec &s, int kind, int var, cudaStream_t st) {
    return launch_pass_dir<uint32_t, DIR_INV>(s, kind, var, st);
}
}  // namespace ntt
