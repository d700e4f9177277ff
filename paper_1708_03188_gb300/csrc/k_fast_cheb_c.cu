// k_fast_cheb_c.cu - instantiations of cheb_mode (see k_fast_cheb.cuh).
#include "k_fast_cheb.cuh"

namespace sgm {

template cudaError_t cheb_mode<double, kChebScalar, double>(const void*, void*, int, long, int, bool, const double2*,
                                                 const double2*, cudaStream_t);
template cudaError_t cheb_mode<double, kChebBackward, double>(const void*, void*, int, long, int, bool, const double2*,
                                                 const double2*, cudaStream_t);
template cudaError_t cheb_mode<double, kChebForwardT, double>(const void*, void*, int, long, int, bool, const double2*,
                                                 const double2*, cudaStream_t);

}  // namespace sgm
