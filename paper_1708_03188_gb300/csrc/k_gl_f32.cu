// k_gl_f32.cu - float instantiation of the Ginzburg-Landau kernels (k_gl.cuh).
#include "k_gl.cuh"

namespace sgm {
template cudaError_t gl_launch<float>(int, int, bool, bool, const float2*, float2*, float2*, float2*, const float2*, float2*, float2*, const GlParams&,
                                   const float2*, cudaStream_t);
}  // namespace sgm
