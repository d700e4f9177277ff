// k_fourier.cu - Fourier-axis transforms (Sec. 3.4.1 of the paper):
//   forward  u_hat_l = (1/M) sum_j u_j exp(-i l X_j),  backward  u_j = sum_l u_hat_l exp(i l X_j).
//
// k_rows     the contiguous last axis, a CTA holding several whole rows in shared memory.
//            R2C of even length M packs the real row as M/2 complex numbers
//            z_n = u_{2n} + i u_{2n+1}, transforms them with one length-M/2 FFT and
//            separates the even/odd half-spectra (E_k, O_k) to form
//            u_hat_k = (E_k + w^k O_k) / M, w = exp(-2 pi i / M), k = 0..M/2.
//            C2R inverts that packing; the imaginary parts of the self-conjugate
//            coefficients (k = 0 and k = M/2) do not reach the real result.
//            Odd M (R2C and C2R) uses a full complex FFT of length M.
// k_strided  a strided axis of a [outer][M][inner] complex array: a CTA stages a tile
//            of TW neighbouring columns (TW * 8 or 16 bytes contiguous per row, so the
//            global accesses are full 128-byte lines), transposes it into TW lines in
//            shared memory, transforms them and writes the tile back (in place).
#include <algorithm>

#include "fft_core.cuh"

namespace sgm {

template <typename T> constexpr int elems_per_cta() { return sizeof(T) == 4 ? 4096 : 2048; }

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_rows(const void* __restrict__ in, void* __restrict__ out, long nrows,
                                              int L, const __grid_constant__ FftPlan plan,
                                              const cplx<T>* __restrict__ tw_plan,
                                              const cplx<T>* __restrict__ tw_L, int lines) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = plan.L;               // FFT length
  const int ld = n;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + (long)lines * ld;
  const long row0 = (long)blockIdx.x * lines;
  const int nl = (int)min((long)lines, nrows - row0);
  const bool packed = (L % 2 == 0) && (MODE == kRowR2C || MODE == kRowC2R);
  const int h = L / 2;

  // ---- load ------------------------------------------------------------------------------
  if (MODE == kRowR2C) {
    if (packed) {
      const C* src = reinterpret_cast<const C*>(in) + row0 * h;
      for (int idx = threadIdx.x; idx < nl * h; idx += blockDim.x) A[idx] = src[idx];
    } else {
      const T* src = reinterpret_cast<const T*>(in) + row0 * L;
      for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) A[idx] = mk<C>(src[idx], (T)0);
    }
  } else if (MODE == kRowC2R) {
    const int hp = L / 2 + 1;
    const C* src = reinterpret_cast<const C*>(in) + row0 * hp;
    if (packed) {
      for (int idx = threadIdx.x; idx < nl * h; idx += blockDim.x) {
        const int line = idx / h, k = idx - line * h;
        C x = src[(long)line * hp + k];
        C y = src[(long)line * hp + (h - k)];
        if (k == 0) { x.y = 0; y.y = 0; }
        C yc = cconj(y);
        C e = cadd(x, yc);                               // 2 E_k
        C o = cmulc(csub(x, yc), __ldg(&tw_L[k]));       // 2 O_k = conj(w^k) (x - conj y)
        A[(long)line * ld + k] = mk<C>(e.x - o.y, e.y + o.x);  // 2 (E_k + i O_k)
      }
    } else {
      for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) {
        const int line = idx / L, j = idx - line * L;
        C v = (j <= L / 2) ? src[(long)line * hp + j] : cconj(src[(long)line * hp + (L - j)]);
        if (j == 0) v.y = 0;
        A[(long)line * ld + j] = v;
      }
    }
  } else {
    const C* src = reinterpret_cast<const C*>(in) + row0 * L;
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) A[idx] = src[idx];
  }
  __syncthreads();

  // ---- transform ---------------------------------------------------------------------------
  constexpr bool INV = (MODE == kRowC2R || MODE == kRowC2CInv);
  C* R = fft_lines<INV>(A, B, nl, ld, plan, tw_plan);

  // ---- store -------------------------------------------------------------------------------
  if (MODE == kRowR2C) {
    const int hp = L / 2 + 1;
    C* dst = reinterpret_cast<C*>(out) + row0 * hp;
    const T s = (T)1 / (T)L;
    for (int idx = threadIdx.x; idx < nl * hp; idx += blockDim.x) {
      const int line = idx / hp, k = idx - line * hp;
      C v;
      if (packed) {
        C z = R[(long)line * ld + (k % h)];
        C zc = cconj(R[(long)line * ld + ((h - k) % h)]);
        C e = cadd(z, zc);                               // 2 E_k
        C o = rot90<false>(cmul(__ldg(&tw_L[k]), csub(z, zc)));  // 2 w^k O_k
        v = cscale(cadd(e, o), (T)0.5 * s);
      } else {
        v = cscale(R[(long)line * ld + k], s);
      }
      dst[idx] = v;
    }
  } else if (MODE == kRowC2R) {
    if (packed) {
      C* dst = reinterpret_cast<C*>(out) + row0 * h;
      for (int idx = threadIdx.x; idx < nl * h; idx += blockDim.x) dst[idx] = R[idx];
    } else {
      T* dst = reinterpret_cast<T*>(out) + row0 * L;
      for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) dst[idx] = R[idx].x;
    }
  } else {
    C* dst = reinterpret_cast<C*>(out) + row0 * L;
    const T s = (MODE == kRowC2CFwd) ? (T)1 / (T)L : (T)1;
    for (int idx = threadIdx.x; idx < nl * L; idx += blockDim.x) dst[idx] = cscale(R[idx], s);
  }
}

template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_strided(const cplx<T>* in, cplx<T>* out, long inner, int L,
                                                 const __grid_constant__ FftPlan plan,
                                                 const cplx<T>* __restrict__ tw, int TW) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = L + 1;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + (long)TW * ld;
  const long o = blockIdx.y;
  const long t0 = (long)blockIdx.x * TW;
  const int nt = (int)min((long)TW, inner - t0);
  const C* src = in + o * L * inner + t0;
  C* dst = out + o * L * inner + t0;
  for (int idx = threadIdx.x; idx < L * TW; idx += blockDim.x) {
    const int i = idx / TW, t = idx - i * TW;
    if (t < nt) A[t * ld + i] = src[(long)i * inner + t];
  }
  __syncthreads();
  C* R = fft_lines<INV>(A, B, nt, ld, plan, tw);
  const T s = INV ? (T)1 : (T)1 / (T)L;
  for (int idx = threadIdx.x; idx < L * TW; idx += blockDim.x) {
    const int i = idx / TW, t = idx - i * TW;
    if (t < nt) dst[(long)i * inner + t] = cscale(R[t * ld + i], s);
  }
}

template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_rows(int mode, const void* in, void* out, long nrows, int L, const FftPlan& plan,
                        const cplx<T>* tw_plan, const cplx<T>* tw_L, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  const int n = plan.L;
  const int lines = max(1, elems_per_cta<T>() / n);
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)lines * n;
  const unsigned grid = (unsigned)((nrows + lines - 1) / lines);
  cudaError_t e = cudaSuccess;
  switch (mode) {
#define SGM_ROWS(M)                                                                     \
  case M:                                                                               \
    if ((e = set_smem(k_rows<T, M>, smem)) != cudaSuccess) return e;                    \
    k_rows<T, M><<<grid, 256, smem, s>>>(in, out, nrows, L, plan, tw_plan, tw_L, lines); \
    break;
    SGM_ROWS(kRowR2C)
    SGM_ROWS(kRowC2R)
    SGM_ROWS(kRowC2CFwd)
    SGM_ROWS(kRowC2CInv)
#undef SGM_ROWS
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_strided(bool inverse, const void* in, void* out, long outer, int L, long inner,
                           const FftPlan& plan, const cplx<T>* tw, cudaStream_t s) {
  if (outer <= 0 || inner <= 0) return cudaSuccess;
  // TW neighbouring columns per CTA: 128 contiguous bytes per row, fewer when the
  // staged tile would not fit in shared memory.
  const int TWmax = sizeof(T) == 4 ? 16 : 8;
  const int TW = (int)std::max(1L, std::min((long)TWmax, (long)(kSmemBudget / (2 * sizeof(cplx<T>) * (L + 1)))));
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)TW * (L + 1);
  dim3 grid((unsigned)((inner + TW - 1) / TW), (unsigned)outer);
  cudaError_t e;
  if (inverse) {
    if ((e = set_smem(k_strided<T, true>, smem)) != cudaSuccess) return e;
    k_strided<T, true><<<grid, 256, smem, s>>>((const cplx<T>*)in, (cplx<T>*)out, inner, L, plan, tw, TW);
  } else {
    if ((e = set_smem(k_strided<T, false>, smem)) != cudaSuccess) return e;
    k_strided<T, false><<<grid, 256, smem, s>>>((const cplx<T>*)in, (cplx<T>*)out, inner, L, plan, tw, TW);
  }
  return cudaGetLastError();
}

template cudaError_t launch_rows<float>(int, const void*, void*, long, int, const FftPlan&, const float2*,
                                        const float2*, cudaStream_t);
template cudaError_t launch_rows<double>(int, const void*, void*, long, int, const FftPlan&, const double2*,
                                         const double2*, cudaStream_t);
template cudaError_t launch_strided<float>(bool, const void*, void*, long, int, long, const FftPlan&,
                                           const float2*, cudaStream_t);
template cudaError_t launch_strided<double>(bool, const void*, void*, long, int, long, const FftPlan&,
                                            const double2*, cudaStream_t);

}  // namespace sgm
