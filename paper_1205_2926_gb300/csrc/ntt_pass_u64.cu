// Dispatch of the pass kernels for 64-bit words to the per-direction units.
#include "ntt_internal.hpp"

namespace ntt {
cudaError_t launch_pass_u64_fwd(const LaunchSpec &s, int kind, int var, cudaStream_t st);
cudaError_t launch_pass_u64_inv(const LaunchSpec &s, int kind, int var, cudaStream_t st);

cudaError_t launch_pass_u64(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st) {
    return dir == 0 ? launch_pass_u64_fwd(s, kind, var, st) : launch_pass_u64_inv(s, kind, var, st);
}
}  // namespace ntt
