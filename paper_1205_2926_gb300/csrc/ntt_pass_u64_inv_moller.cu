// Pass kernels for 64-bit words, inverse direction, Moeller's fully reduced butterflies.
#include "ntt_pass_inst.cuh"

namespace ntt {
cudaError_t launch_pass_u64_inv_moller(const LaunchSpec &s, int kind, cudaStream_t st) {
    return launch_kind<uint64_t, DIR_INV, VAR_MOLLER>(s, kind, st);
}
}  // namespace ntt
