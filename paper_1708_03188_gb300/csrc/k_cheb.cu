// k_cheb.cu - the Chebyshev axis (axis 0) transforms of Sec. 3.4.2 of the paper.
//
// Scalar product (the inner product S of Sec. 3.4.2, computed "with a DCT"):
//   moments  t_k = (pi/N) sum_j g_j cos(pi k (2j+1) / (2N))        (DCT-II, weights pi/N)
//   stencil  Dirichlet  S_k = t_k - t_{k+2},                         k = 0..N-3
//            Neumann    S_k = t_k - q_k t_{k+2}, q_k = (k/(k+2))^2,    k = 0..N-3
//            biharmonic S_k = t_k + beta_k t_{k+2} + gamma_k t_{k+4}, k = 0..N-5,
//            beta_k = -2(k+2)/(k+3), gamma_k = (k+1)/(k+3)          (Eq. chebbiharmonic)
//            regular    S_k = t_k
// The DCT-II of a complex column g = p + i q is one complex FFT of length N of the
// even/odd reordering v_n = g_{2n}, v_{N-1-n} = g_{2n+1}; with V = FFT(v) the two real
// DCTs are  DCT(p)_k = Re(w_k (V_k + conj V_{N-k}) / 2),  DCT(q)_k = Re(w_k (V_k - conj V_{N-k}) / (2i)),
// w_k = exp(-i pi k / (2N))  (Makhoul's reordering).
//
// Backward (Eq. fast_shen): the stencil maps Shen coefficients to Chebyshev coefficients
//   Dirichlet a_k = c_k - c_{k-2};  Neumann a_k = c_k - q_{k-2} c_{k-2};  biharmonic a_k = c_k + beta_{k-2} c_{k-2} + gamma_{k-4} c_{k-4}
// and the DCT-III u_j = sum_k a_k cos(pi k (2j+1) / (2N)) is one inverse FFT of
// V_0 = a_0, V_k = conj(w_k) (a_k - i a_{N-k}) / 2 (k >= 1), undoing the reordering.
//
// Forward for the regular basis: the mass matrix is diag(pi/2 c_k), so
//   u_hat_k = 2 t'_k / (N c_k) with t' the unweighted DCT-II.
//
// A CTA stages TW neighbouring columns (contiguous in memory) of all N rows, so the
// global reads and writes are whole 128-byte lines, and transforms them as TW lines
// in shared memory.  `real` = a real 1-D column (imaginary parts zero / dropped).
// TS is the storage type of the spectral-side array: T, or double while computing in
// FP32 (the physical-to-physical solves keep their spectral intermediate in FP64 so the
// FP64 eliminations read and write it without conversions; the conversions happen here
// on the integer pipe, convert.cuh).
#include <algorithm>

#include "convert.cuh"
#include "fft_core.cuh"

namespace sgm {

template <typename T> __device__ __forceinline__ T bih_beta(int k) { return (T)(-2 * (k + 2)) / (T)(k + 3); }
template <typename T> __device__ __forceinline__ T bih_gamma(int k) { return (T)(k + 1) / (T)(k + 3); }

__device__ __forceinline__ int nbasis(int basis, int N) {
  return basis_count(basis, N);
}

template <typename T, int MODE, typename TS>
__global__ void __launch_bounds__(256) k_cheb(const void* __restrict__ in, void* __restrict__ out, int N, long inner,
                                              int basis, int real, const __grid_constant__ FftPlan plan,
                                              const cplx<T>* __restrict__ tw, const cplx<T>* __restrict__ dctw,
                                              int TW) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = N + 1;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + (long)TW * ld;
  const long t0 = (long)blockIdx.x * TW;
  const int nt = (int)min((long)TW, inner - t0);
  const int nb = nbasis(basis, N);
  const C* src = reinterpret_cast<const C*>(in);
  const T* srcr = reinterpret_cast<const T*>(in);

  // physical side (input of the scalar product, output of the backward transform): type T
  auto load = [&](int i, int t) -> C {
    const long g = (long)i * inner + t0 + t;
    return real ? mk<C>(srcr[g], (T)0) : src[g];
  };
  auto store = [&](int i, int t, C v) {
    const long g = (long)i * inner + t0 + t;
    if (real) reinterpret_cast<T*>(out)[g] = v.x;
    else reinterpret_cast<C*>(out)[g] = v;
  };
  // spectral side: type TS
  auto load_spec = [&](int i, int t) -> C {
    return from_spec<TS, C>(reinterpret_cast<const TS*>(in), (long)i * inner + t0 + t, real);
  };
  auto store_spec = [&](int i, int t, C v) {
    to_spec<TS, C>(reinterpret_cast<TS*>(out), (long)i * inner + t0 + t, real, v);
  };

  if (MODE == kChebScalar || MODE == kChebForwardT) {
    // reordered load: g_j -> position j/2 (even j) or N-1-j/2 (odd j)
    for (int idx = threadIdx.x; idx < N * TW; idx += blockDim.x) {
      const int j = idx / TW, t = idx - j * TW;
      if (t < nt) A[t * ld + ((j & 1) ? N - 1 - (j >> 1) : (j >> 1))] = load(j, t);
    }
    __syncthreads();
    C* V = fft_lines<false>(A, B, nt, ld, plan, tw);
    C* M = (V == A) ? B : A;  // moments buffer
    const T scale = (MODE == kChebScalar) ? (T)3.14159265358979323846 / (T)N : (T)2 / (T)N;
    for (int idx = threadIdx.x; idx < N * nt; idx += blockDim.x) {
      const int t = idx / N, k = idx - t * N;
      const C v = V[t * ld + k];
      const C vr = cconj(V[t * ld + (k == 0 ? 0 : N - k)]);
      const C w = __ldg(&dctw[k]);
      const C a = cadd(v, vr), b = csub(v, vr);      // 2 A_k, 2 i B_k
      // Re(w A) = (w.x a.x - w.y a.y)/2 ; B = b / (2i) -> Re(w B) = (w.x b.y + w.y b.x)/2
      C m = mk<C>((T)0.5 * (w.x * a.x - w.y * a.y), (T)0.5 * (w.x * b.y + w.y * b.x));
      T sc = scale;
      if (MODE == kChebForwardT && k == 0) sc *= (T)0.5;
      M[t * ld + k] = cscale(m, sc);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < N * TW; idx += blockDim.x) {
      const int k = idx / TW, t = idx - k * TW;
      if (t >= nt) continue;
      const C* m = M + t * ld;
      C s = mk<C>((T)0, (T)0);
      if (k < nb) {
        if (MODE == kChebForwardT || basis == kCheb) {
          s = m[k];
        } else if (basis == kDirichlet) {
          s = csub(m[k], m[k + 2]);
        } else if (basis == kNeumann) {
          const T q = neumann_q<T>(k);
          s = mk<C>(m[k].x - q * m[k + 2].x, m[k].y - q * m[k + 2].y);
        } else {
          const T be = bih_beta<T>(k), ga = bih_gamma<T>(k);
          s = mk<C>(m[k].x + be * m[k + 2].x + ga * m[k + 4].x, m[k].y + be * m[k + 2].y + ga * m[k + 4].y);
        }
      }
      store_spec(k, t, s);
    }
  } else {  // backward
    for (int idx = threadIdx.x; idx < N * TW; idx += blockDim.x) {
      const int k = idx / TW, t = idx - k * TW;
      if (t < nt) B[t * ld + k] = (k < nb) ? load_spec(k, t) : mk<C>((T)0, (T)0);
    }
    __syncthreads();
    // stencil: Shen -> Chebyshev coefficients, into A
    for (int idx = threadIdx.x; idx < N * nt; idx += blockDim.x) {
      const int t = idx / N, k = idx - t * N;
      const C* c = B + t * ld;
      C a = c[k];
      if (basis == kDirichlet) {
        if (k >= 2) a = csub(a, c[k - 2]);
      } else if (basis == kNeumann) {
        if (k >= 2) { const T q = neumann_q<T>(k - 2); a.x -= q * c[k - 2].x; a.y -= q * c[k - 2].y; }
      } else if (basis == kBiharmonic) {
        if (k >= 2) { const T be = bih_beta<T>(k - 2); a.x += be * c[k - 2].x; a.y += be * c[k - 2].y; }
        if (k >= 4) { const T ga = bih_gamma<T>(k - 4); a.x += ga * c[k - 4].x; a.y += ga * c[k - 4].y; }
      }
      A[t * ld + k] = a;
    }
    __syncthreads();
    // V_k = conj(w_k)(a_k - i a_{N-k}) / 2, V_0 = a_0  (into B)
    for (int idx = threadIdx.x; idx < N * nt; idx += blockDim.x) {
      const int t = idx / N, k = idx - t * N;
      const C* a = A + t * ld;
      C v;
      if (k == 0) {
        v = a[0];
      } else {
        const C x = a[k], y = a[N - k];
        const C d = mk<C>(x.x + y.y, x.y - y.x);       // a_k - i a_{N-k}
        v = cscale(cmulc(d, __ldg(&dctw[k])), (T)0.5);
      }
      B[t * ld + k] = v;
    }
    __syncthreads();
    C* R = fft_lines<true>(B, A, nt, ld, plan, tw);
    for (int idx = threadIdx.x; idx < N * TW; idx += blockDim.x) {
      const int j = idx / TW, t = idx - j * TW;
      if (t < nt) store(j, t, R[t * ld + ((j & 1) ? N - 1 - (j >> 1) : (j >> 1))]);
    }
  }
}

template <typename T>
cudaError_t launch_cheb(int mode, int basis, bool real, const void* in, void* out, int N, long inner,
                        const FftPlan& plan, const cplx<T>* tw, const cplx<T>* dctw, cudaStream_t s, bool wide) {
  if (inner <= 0) return cudaSuccess;
  const int TWmax = real ? 1 : (sizeof(T) == 4 ? 16 : 8);
  const int TW = (int)std::max(1L, std::min((long)TWmax, (long)(kSmemBudget / (2 * sizeof(cplx<T>) * (N + 1)))));
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)TW * (N + 1);
  const unsigned grid = (unsigned)((inner + TW - 1) / TW);
  cudaError_t e = cudaSuccess;
  auto go = [&](auto kernel) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    kernel<<<grid, 256, smem, s>>>(in, out, N, inner, basis, real ? 1 : 0, plan, tw, dctw, TW);
    return cudaSuccess;
  };
  const bool w = wide && sizeof(T) == 4;
  switch (mode) {
    case kChebScalar: e = w ? go(k_cheb<T, kChebScalar, double>) : go(k_cheb<T, kChebScalar, T>); break;
    case kChebBackward: e = w ? go(k_cheb<T, kChebBackward, double>) : go(k_cheb<T, kChebBackward, T>); break;
    case kChebForwardT: e = go(k_cheb<T, kChebForwardT, T>); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template cudaError_t launch_cheb<float>(int, int, bool, const void*, void*, int, long, const FftPlan&,
                                        const float2*, const float2*, cudaStream_t, bool);
template cudaError_t launch_cheb<double>(int, int, bool, const void*, void*, int, long, const FftPlan&,
                                         const double2*, const double2*, cudaStream_t, bool);

}  // namespace sgm
