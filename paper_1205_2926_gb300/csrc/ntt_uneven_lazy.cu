// ntt_uneven_lazy.cu -- k_uneven with the lazy butterflies (Algorithms 3 and 4).
#include "ntt_uneven_kernel.cuh"

namespace ntt {

template <>
UnevenKernel uneven_kernel<VAR_LAZY>() {
    return {reinterpret_cast<const void *>(&k_uneven<VAR_LAZY>), &launch_uneven<VAR_LAZY>};
}

}  // namespace ntt
