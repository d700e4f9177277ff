// k_fast_strided.cu - dispatch of the compile-time-length strided-axis transforms (k_fast.cuh).
#include "k_fast.cuh"

namespace sgm {

template <typename T, bool INV>
static cudaError_t strided_dir(const void* in, void* out, long outer, int L, long inner, const cplx<T>* twf,
                               cudaStream_t s) {
  constexpr int TW = fast_tw_cols<T>();
  dim3 grid((unsigned)((inner + TW - 1) / TW), (unsigned)outer);
  auto go = [&](auto kernel, int l) -> cudaError_t {
    const size_t smem = sizeof(cplx<T>) * (size_t)TW * pad_ld(l);
    cudaError_t e = fast_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, kFastThreads, smem, s>>>((const cplx<T>*)in, (cplx<T>*)out, inner, twf);
    return cudaGetLastError();
  };
  switch (L) {
#define SGM_FS(n) case n: return go(k_strided_fast<T, INV, n>, n);
    SGM_FS(16) SGM_FS(32) SGM_FS(64) SGM_FS(128) SGM_FS(256) SGM_FS(512) SGM_FS(1024) SGM_FS(2048)
    SGM_FS(192) SGM_FS(384) SGM_FS(768) SGM_FS(1536)
#undef SGM_FS
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_strided_fast(bool inverse, const void* in, void* out, long outer, int L, long inner,
                                const cplx<T>* twf, cudaStream_t s) {
  if (outer <= 0 || inner <= 0) return cudaSuccess;
  return inverse ? strided_dir<T, true>(in, out, outer, L, inner, twf, s)
                 : strided_dir<T, false>(in, out, outer, L, inner, twf, s);
}

template cudaError_t launch_strided_fast<float>(bool, const void*, void*, long, int, long, const float2*, cudaStream_t);
template cudaError_t launch_strided_fast<double>(bool, const void*, void*, long, int, long, const double2*,
                                                 cudaStream_t);

}  // namespace sgm
