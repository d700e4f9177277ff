// k_fast_cheb.cuh - launch of one (precision, mode, spectral storage) family of the
// compile-time-length Chebyshev kernels; instantiated in k_fast_cheb_{a,b,c}.cu so the
// build compiles the families in parallel.
#pragma once
#include "k_fast.cuh"

namespace sgm {

template <typename T, int MODE, typename TS>
cudaError_t cheb_mode(const void* in, void* out, int N, long inner, int basis, bool real,
                             const cplx<T>* twf, const cplx<T>* dctw, cudaStream_t s) {
  constexpr int TW = fast_tw_cols<T>();
  const unsigned grid = (unsigned)((inner + TW - 1) / TW);
  auto go = [&](auto kernel, int n) -> cudaError_t {
    const size_t smem = sizeof(cplx<T>) * (size_t)TW * pad_ld(n);
    cudaError_t e = fast_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, kFastThreads, smem, s>>>(in, out, inner, basis, real ? 1 : 0, twf, dctw);
    return cudaGetLastError();
  };
  switch (N) {
#define SGM_FC(n) case n: return go(k_cheb_fast<T, MODE, TS, n>, n);
    SGM_FC(16) SGM_FC(32) SGM_FC(64) SGM_FC(128) SGM_FC(256) SGM_FC(512) SGM_FC(1024) SGM_FC(2048)
    SGM_FC(192) SGM_FC(384) SGM_FC(768) SGM_FC(1536)
#undef SGM_FC
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sgm
