// ntt_uneven_ntl.cu -- k_uneven with the NTL-style fully reduced butterflies (Algorithm 2).
#include "ntt_uneven_kernel.cuh"

namespace ntt {

template <>
UnevenKernel uneven_kernel<VAR_NTL>() {
    return {reinterpret_cast<const void *>(&k_uneven<VAR_NTL>), &launch_uneven<VAR_NTL>};
}

}  // namespace ntt
