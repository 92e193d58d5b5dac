// Pass kernels for 32-bit words (beta = 2^32, p < 2^30).
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u32(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st) {
    return launch_pass_t<uint32_t>(s, kind, dir, var, st);
}
}  // namespace ntt
