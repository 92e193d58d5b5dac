// Dispatch of the pass kernels for 32-bit words to the per-(direction, variant) units.
#include "ntt_internal.hpp"

namespace ntt {
cudaError_t launch_pass_u32_fwd_lazy(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_fwd_ntl(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_fwd_mont(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_inv_lazy(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_inv_ntl(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_inv_mont(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_fwd_moller(const LaunchSpec &s, int kind, cudaStream_t st);
cudaError_t launch_pass_u32_inv_moller(const LaunchSpec &s, int kind, cudaStream_t st);

cudaError_t launch_pass_u32(const LaunchSpec &s, int kind, int dir, int var, cudaStream_t st) {
    switch (var) {
        case 0: return dir == 0 ? launch_pass_u32_fwd_lazy(s, kind, st) : launch_pass_u32_inv_lazy(s, kind, st);
        case 1: return dir == 0 ? launch_pass_u32_fwd_ntl(s, kind, st) : launch_pass_u32_inv_ntl(s, kind, st);
        case 2: return dir == 0 ? launch_pass_u32_fwd_mont(s, kind, st) : launch_pass_u32_inv_mont(s, kind, st);
        case 3: return dir == 0 ? launch_pass_u32_fwd_moller(s, kind, st) : launch_pass_u32_inv_moller(s, kind, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace ntt
