// k_gl_f64.cu - double instantiation of the Ginzburg-Landau kernels (k_gl.cuh).
#include "k_gl.cuh"

namespace sgm {
template cudaError_t gl_launch<double>(int, int, bool, bool, const double2*, double2*, double2*, double2*, const double2*, double2*, double2*, const GlParams&,
                                   const double2*, cudaStream_t);
}  // namespace sgm
