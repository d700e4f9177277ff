// k_fast_rows.cu - dispatch of the compile-time-length row transforms (k_fast.cuh).
#include "k_fast.cuh"

namespace sgm {

bool fast_compiled(int L) {
  switch (L) {
    case 16: case 32: case 64: case 128: case 256: case 512: case 1024: case 2048:
    case 192: case 384: case 768: case 1536: return true;
    default: return false;
  }
}

template <typename T, int MODE>
static cudaError_t rows_mode(const void* in, void* out, long nrows, int L, int LF, const cplx<T>* twf,
                             const cplx<T>* tw_L, cudaStream_t s) {
  auto go = [&](auto kernel, int lf) -> cudaError_t {
    const int lines = std::max(1, fast_elems<T>() / lf);
    const size_t smem = sizeof(cplx<T>) * (size_t)lines * pad_ld(lf);
    cudaError_t e = fast_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    kernel<<<(unsigned)((nrows + lines - 1) / lines), kFastThreads, smem, s>>>(in, out, nrows, L, twf, tw_L);
    return cudaGetLastError();
  };
  switch (LF) {
#define SGM_FR(n) case n: return go(k_rows_fast<T, MODE, n>, n);
    SGM_FR(16) SGM_FR(32) SGM_FR(64) SGM_FR(128) SGM_FR(256) SGM_FR(512) SGM_FR(1024) SGM_FR(2048)
    SGM_FR(192) SGM_FR(384) SGM_FR(768) SGM_FR(1536)
#undef SGM_FR
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_rows_fast(int mode, const void* in, void* out, long nrows, int L, const cplx<T>* twf,
                             const cplx<T>* tw_L, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const bool packed = (mode == kRowR2C || mode == kRowC2R);
  const int LF = packed ? L / 2 : L;
  switch (mode) {
    case kRowR2C: return rows_mode<T, kRowR2C>(in, out, nrows, L, LF, twf, tw_L, s);
    case kRowC2R: return rows_mode<T, kRowC2R>(in, out, nrows, L, LF, twf, tw_L, s);
    case kRowC2CFwd: return rows_mode<T, kRowC2CFwd>(in, out, nrows, L, LF, twf, tw_L, s);
    case kRowC2CInv: return rows_mode<T, kRowC2CInv>(in, out, nrows, L, LF, twf, tw_L, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_rows_fast<float>(int, const void*, void*, long, int, const float2*, const float2*,
                                             cudaStream_t);
template cudaError_t launch_rows_fast<double>(int, const void*, void*, long, int, const double2*, const double2*,
                                              cudaStream_t);

}  // namespace sgm
