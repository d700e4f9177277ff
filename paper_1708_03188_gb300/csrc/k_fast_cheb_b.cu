// k_fast_cheb_b.cu - instantiations of cheb_mode (see k_fast_cheb.cuh).
#include "k_fast_cheb.cuh"

namespace sgm {

template cudaError_t cheb_mode<float, kChebScalar, double>(const void*, void*, int, long, int, bool, const float2*,
                                                 const float2*, cudaStream_t);
template cudaError_t cheb_mode<float, kChebBackward, double>(const void*, void*, int, long, int, bool, const float2*,
                                                 const float2*, cudaStream_t);

}  // namespace sgm
