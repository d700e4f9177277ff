// k_fast_cheb.cu - dispatch of the compile-time-length Chebyshev-axis transforms (k_fast.cuh).
#include "k_fast.cuh"

namespace sgm {

template <typename T, int MODE, typename TS>
cudaError_t cheb_mode(const void* in, void* out, int N, long inner, int basis, bool real,
                      const cplx<T>* twf, const cplx<T>* dctw, cudaStream_t s);

template <typename T>
cudaError_t launch_cheb_fast(int mode, int basis, bool real, const void* in, void* out, int N, long inner,
                             const cplx<T>* twf, const cplx<T>* dctw, cudaStream_t s, bool wide) {
  if (inner <= 0) return cudaSuccess;
  const bool w = wide && sizeof(T) == 4;
  switch (mode) {
    case kChebScalar:
      return w ? cheb_mode<T, kChebScalar, double>(in, out, N, inner, basis, real, twf, dctw, s)
               : cheb_mode<T, kChebScalar, T>(in, out, N, inner, basis, real, twf, dctw, s);
    case kChebBackward:
      return w ? cheb_mode<T, kChebBackward, double>(in, out, N, inner, basis, real, twf, dctw, s)
               : cheb_mode<T, kChebBackward, T>(in, out, N, inner, basis, real, twf, dctw, s);
    case kChebForwardT:
      return cheb_mode<T, kChebForwardT, T>(in, out, N, inner, basis, real, twf, dctw, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_cheb_fast<float>(int, int, bool, const void*, void*, int, long, const float2*,
                                             const float2*, cudaStream_t, bool);
template cudaError_t launch_cheb_fast<double>(int, int, bool, const void*, void*, int, long, const double2*,
                                              const double2*, cudaStream_t, bool);

}  // namespace sgm
