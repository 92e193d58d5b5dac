// Pass kernels for 32-bit words, forward direction, ntl butterflies.
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u32_fwd_ntl(const LaunchSpec &s, int kind, cudaStream_t st) {
    return launch_kind<uint32_t, DIR_FWD, VAR_NTL>(s, kind, st);
}
}  // namespace ntt
