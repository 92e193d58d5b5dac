// Pass kernels for 64-bit words (beta = 2^64, p < 2^62).
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u64(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st) {
    return launch_pass_t<uint64_t>(s, kind, dir, var, st);
}
}  // namespace ntt
