// Pass kernels for 32-bit words, forward direction (own translation
// unit so that the instantiations compile in parallel).
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u32_fwd(const LaunchSpec &s, int kind, int var, cudaStream_t st) {
    return launch_pass_dir<uint32_t, DIR_FWD>(s, kind, var, st);
}
}  // namespace ntt
