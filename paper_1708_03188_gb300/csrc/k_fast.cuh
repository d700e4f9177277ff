// k_fast.cuh - the rows / strided / Chebyshev transform kernels on the compile-time FFT
// engine (fft_fast.cuh).  Same arithmetic as k_fourier.cu and k_cheb.cu (whose comments give
// the formulas); only the FFT length is a template parameter.  Included by k_fast_*.cu.
#pragma once
#include <algorithm>

#include "convert.cuh"
#include "fft_fast.cuh"

namespace sgm {

template <typename T> __host__ __device__ constexpr int fast_elems() { return sizeof(T) == 4 ? 4096 : 2048; }
template <typename T> __host__ __device__ constexpr int fast_tw_cols() { return sizeof(T) == 4 ? 16 : 8; }
constexpr int kFastThreads = 256;

// Copy TOTAL elements through registers: each thread loads up to 128 bytes of its elements
// (16 complex64 or 8 pairs; element idx = threadIdx.x + q * kFastThreads) before storing them,
// so the loads of a chunk are all in flight at once (a generic global pointer may alias shared memory, so an interleaved
// load/store loop would wait for every load).  ld(idx) -> value, st(idx, value); both are only
// called for idx < TOTAL.
template <int TOTAL, typename C, typename LD, typename ST>
__device__ __forceinline__ void staged_copy(LD ld, ST st) {
  constexpr int PER = (TOTAL + kFastThreads - 1) / kFastThreads;
  constexpr int CMAX = 128 / (int)sizeof(C) > 0 ? 128 / (int)sizeof(C) : 1;
  constexpr int CH = PER < CMAX ? PER : CMAX;
#pragma unroll 1
  for (int q0 = 0; q0 < PER; q0 += CH) {
    C v[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int idx = threadIdx.x + (q0 + q) * kFastThreads;
      if (q0 + q < PER && idx < TOTAL) v[q] = ld(idx);
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int idx = threadIdx.x + (q0 + q) * kFastThreads;
      if (q0 + q < PER && idx < TOTAL) st(idx, v[q]);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// rows of the contiguous last axis; LF = FFT length (L/2 for packed R2C/C2R, else L)
template <typename T, int MODE, int LF>
__global__ void __launch_bounds__(kFastThreads) k_rows_fast(const void* __restrict__ in, void* __restrict__ out,
                                                            long nrows, int L, const cplx<T>* __restrict__ twf,
                                                            const cplx<T>* __restrict__ tw_L) {
  using C = cplx<T>;
  constexpr int LINES = fast_elems<T>() / LF > 0 ? fast_elems<T>() / LF : 1;
  constexpr int LDP = pad_ld(LF);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const long row0 = (long)blockIdx.x * LINES;
  const int nl = (int)min((long)LINES, nrows - row0);
  constexpr int H = LF;                                           // packed: L/2

  if (MODE == kRowC2R) {
    const C* src = reinterpret_cast<const C*>(in) + row0 * (H + 1);
    const int n = nl * H;
    // stage x_k and x_{H-k} as one pair per element (C2 holds both)
    struct C2 { C x, y; };
    staged_copy<LINES * H, C2>(
        [&](int idx) {
          C2 r;
          if (idx < n) {
            const int line = idx / H, k = idx - line * H;
            r.x = src[(long)line * (H + 1) + k];
            r.y = src[(long)line * (H + 1) + (H - k)];
          }
          return r;
        },
        [&](int idx, C2 v) {
          if (idx >= n) return;
          const int line = idx / H, k = idx - line * H;
          C x = v.x, y = v.y;
          if (k == 0) { x.y = 0; y.y = 0; }
          const C yc = cconj(y);
          const C e = cadd(x, yc);
          const C o = cmulc(csub(x, yc), __ldg(&tw_L[k]));
          buf[line * LDP + padi(k)] = mk<C>(e.x - o.y, e.y + o.x);
        });
  } else {
    const C* src = reinterpret_cast<const C*>(in) + row0 * LF;   // packed real rows are LF complex
    const int n = nl * LF;
    staged_copy<LINES * LF, C>([&](int idx) { return idx < n ? src[idx] : mk<C>((T)0, (T)0); },
                               [&](int idx, C v) { if (idx < n) buf[(idx / LF) * LDP + padi(idx % LF)] = v; });
  }
  __syncthreads();
  constexpr bool INV = (MODE == kRowC2R || MODE == kRowC2CInv);
  fft_fast<LF, LINES, kFastThreads, INV>(buf, nl, twf);

  if (MODE == kRowR2C) {
    C* dst = reinterpret_cast<C*>(out) + row0 * (H + 1);
    const T s = (T)0.5 / (T)L;
    for (int idx = threadIdx.x; idx < nl * (H + 1); idx += kFastThreads) {
      const int line = idx / (H + 1), k = idx - line * (H + 1);
      const C z = buf[line * LDP + padi(k == H ? 0 : k)];
      const C zc = cconj(buf[line * LDP + padi(k == 0 ? 0 : H - k)]);
      const C e = cadd(z, zc);
      const C o = rot90<false>(cmul(__ldg(&tw_L[k]), csub(z, zc)));
      dst[idx] = cscale(cadd(e, o), s);
    }
  } else {
    C* dst = reinterpret_cast<C*>(out) + row0 * LF;
    const T s = (MODE == kRowC2CFwd) ? (T)1 / (T)L : (T)1;
    for (int idx = threadIdx.x; idx < nl * LF; idx += kFastThreads) {
      const int line = idx / LF, e = idx - line * LF;
      dst[idx] = (MODE == kRowC2CFwd) ? cscale(buf[line * LDP + padi(e)], s) : buf[line * LDP + padi(e)];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// strided axis of a [outer][L][inner] complex array, TW neighbouring columns per CTA
template <typename T, bool INV, int L>
__global__ void __launch_bounds__(kFastThreads) k_strided_fast(const cplx<T>* in, cplx<T>* out, long inner,
                                                               const cplx<T>* __restrict__ twf) {
  using C = cplx<T>;
  constexpr int TW = fast_tw_cols<T>();
  constexpr int LDP = pad_ld(L);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const long o = blockIdx.y;
  const long t0 = (long)blockIdx.x * TW;
  const int nt = (int)min((long)TW, inner - t0);
  const C* src = in + o * L * inner + t0;
  C* dst = out + o * L * inner + t0;
  staged_copy<L * TW, C>(
      [&](int idx) {
        const int i = idx / TW, t = idx % TW;
        return t < nt ? src[(long)i * inner + t] : mk<C>((T)0, (T)0);
      },
      [&](int idx, C v) {
        const int i = idx / TW, t = idx % TW;
        if (t < nt) buf[t * LDP + padi(i)] = v;
      });
  __syncthreads();
  fft_fast<L, TW, kFastThreads, INV>(buf, nt, twf);
  const T s = INV ? (T)1 : (T)1 / (T)L;
  for (int idx = threadIdx.x; idx < L * TW; idx += kFastThreads) {
    const int i = idx / TW, t = idx % TW;
    if (t < nt) dst[(long)i * inner + t] = INV ? buf[t * LDP + padi(i)] : cscale(buf[t * LDP + padi(i)], s);
  }
}

// ---------------------------------------------------------------------------------------------
// Chebyshev axis (see k_cheb.cu for the DCT-via-FFT formulas and the stencils)
template <typename T> __device__ __forceinline__ T fbeta(int k) { return (T)(-2 * (k + 2)) / (T)(k + 3); }
template <typename T> __device__ __forceinline__ T fgamma(int k) { return (T)(k + 1) / (T)(k + 3); }

// Per-row tables of a Chebyshev pass held in shared memory by a persistent CTA (k_stream.cu):
// the DCT twiddles exp(-i pi k / (2N)) and the Shen stencil coefficients (c1 = beta_k for the
// biharmonic basis, q_k for the Neumann basis; c2 = gamma_k), so that the per-element work reads
// them instead of computing divisions or loading through the texture path.  A null table means:
// compute the coefficients and read the twiddles from global memory.
template <typename T> struct ChebTables {
  const cplx<T>* dctw;   // shared
  const T* c1;           // shared
  const T* c2;           // shared
};
template <typename T> __device__ __forceinline__ void fill_cheb_tables(cplx<T>* dctw_s, T* c1, T* c2, int N, int basis,
                                                                       const cplx<T>* __restrict__ dctw) {
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    dctw_s[k] = __ldg(&dctw[k]);
    c1[k] = basis == kBiharmonic ? fbeta<T>(k) : basis == kNeumann ? neumann_q<T>(k) : (T)0;
    c2[k] = basis == kBiharmonic ? fgamma<T>(k) : (T)0;
  }
}

// position of input point j in the even/odd (Makhoul) reordering of a length-N line
template <int N> __device__ __forceinline__ int cheb_reord(int j) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }

// Element (line t, position e) of a tile of TW lines: the padded layout of fft_fast
// (t * pad_ld(N) + padi(e), threads over positions first) or, with COLS, the column-tile layout of
// fft_cols (e * TW + t, threads over lines first).
template <bool COLS, int N, int TW> struct TileIdx {
  __device__ __forceinline__ static int at(int t, int e) { return COLS ? e * TW + t : t * pad_ld(N) + padi(e); }
  __device__ __forceinline__ static int line(int idx) { return COLS ? idx % TW : idx / N; }
  __device__ __forceinline__ static int pos(int idx) { return COLS ? idx / TW : idx % N; }
};

// Forward Chebyshev pass after the FFT of the reordered lines in `buf`: DCT moments in place,
// then the Shen stencil of `basis`, written to `out` at rows k, columns t0 + t (t < nt).
template <typename T, int MODE, typename TS, int N, bool COLS = false>
__device__ __forceinline__ void cheb_forward_finish(cplx<T>* buf, int nt, long t0, long inner, int basis, int real,
                                                    void* __restrict__ out, const cplx<T>* __restrict__ dctw,
                                                    const ChebTables<T>* tabs = nullptr) {
  using C = cplx<T>;
  constexpr int TW = fast_tw_cols<T>();
  using I = TileIdx<COLS, N, TW>;
  constexpr int PER = (N * TW + kFastThreads - 1) / kFastThreads;   // elements per thread
  const int nb = basis_count(basis, N);
  // moments, computed in registers and written back in place
  const T scale = (MODE == kChebScalar) ? (T)3.14159265358979323846 / (T)N : (T)2 / (T)N;
  C m[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * kFastThreads;
    const int t = I::line(idx), k = I::pos(idx);
    if (t < nt) {
      const C v = buf[I::at(t, k)];
      const C vr = cconj(buf[I::at(t, k == 0 ? 0 : N - k)]);
      const C w = tabs ? tabs->dctw[k] : __ldg(&dctw[k]);
      const C a = cadd(v, vr), b = csub(v, vr);
      T sc = scale;
      if (MODE == kChebForwardT && k == 0) sc *= (T)0.5;
      m[q] = mk<C>((T)0.5 * sc * (w.x * a.x - w.y * a.y), (T)0.5 * sc * (w.x * b.y + w.y * b.x));
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = threadIdx.x + q * kFastThreads;
    const int t = I::line(idx), k = I::pos(idx);
    if (t < nt) buf[I::at(t, k)] = m[q];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * TW; idx += kFastThreads) {
    const int k = idx / TW, t = idx % TW;
    if (t >= nt) continue;
    C s = mk<C>((T)0, (T)0);
    if (k < nb) {
      if (MODE == kChebForwardT || basis == kCheb) {
        s = buf[I::at(t, k)];
      } else if (basis == kDirichlet) {
        s = csub(buf[I::at(t, k)], buf[I::at(t, k + 2)]);
      } else if (basis == kNeumann) {
        const T q = tabs ? tabs->c1[k] : neumann_q<T>(k);
        const C a0 = buf[I::at(t, k)], a2 = buf[I::at(t, k + 2)];
        s = mk<C>(a0.x - q * a2.x, a0.y - q * a2.y);
      } else {
        const T be = tabs ? tabs->c1[k] : fbeta<T>(k), ga = tabs ? tabs->c2[k] : fgamma<T>(k);
        const C a0 = buf[I::at(t, k)], a2 = buf[I::at(t, k + 2)], a4 = buf[I::at(t, k + 4)];
        s = mk<C>(a0.x + be * a2.x + ga * a4.x, a0.y + be * a2.y + ga * a4.y);
      }
    }
    const long g = (long)k * inner + t0 + t;
    if (MODE == kChebForwardT) {
      if (real) reinterpret_cast<T*>(out)[g] = s.x; else reinterpret_cast<C*>(out)[g] = s;
    } else {
      to_spec<TS, C>(reinterpret_cast<TS*>(out), g, real, s);
    }
  }
}

// Backward Chebyshev pass before the inverse FFT: `buf` holds the coefficient rows k < nb of
// each line (zero past them); applies the Shen stencil (Eq. fast_shen) and the DCT-III
// pre-twiddle in place.  Ends with __syncthreads().
template <typename T, int N, bool COLS = false>
__device__ __forceinline__ void cheb_backward_prepare(cplx<T>* buf, int nt, int basis, const cplx<T>* __restrict__ dctw) {
  using C = cplx<T>;
  constexpr int TW = fast_tw_cols<T>();
  using I = TileIdx<COLS, N, TW>;
  constexpr int HALF = N / 2;
  constexpr int PH = (HALF * TW + kFastThreads - 1) / kFastThreads;
  // Shen stencil in place, in two halves of the rows: the upper half (k >= N/2) first, whose reads
  // (rows k, k - 2, k - 4) all still hold coefficients, then the lower half, which reads only rows
  // below N/2, untouched by the first half's writes.  Half the rows per round halves the values a
  // thread holds across the synchronisation.
#pragma unroll
  for (int h = 1; h >= 0; --h) {
    C a[PH];
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      const int idx = threadIdx.x + q * kFastThreads;
      const int t = COLS ? idx % TW : idx / HALF, k = h * HALF + (COLS ? idx / TW : idx % HALF);
      if (idx < HALF * TW && t < nt) {
        C v = buf[I::at(t, k)];
        if (basis == kDirichlet) {
          if (k >= 2) v = csub(v, buf[I::at(t, k - 2)]);
        } else if (basis == kNeumann) {
          if (k >= 2) { const T q2 = neumann_q<T>(k - 2); const C u = buf[I::at(t, k - 2)]; v.x -= q2 * u.x; v.y -= q2 * u.y; }
        } else if (basis == kBiharmonic) {
          if (k >= 2) { const T be = fbeta<T>(k - 2); const C u = buf[I::at(t, k - 2)]; v.x += be * u.x; v.y += be * u.y; }
          if (k >= 4) { const T ga = fgamma<T>(k - 4); const C u = buf[I::at(t, k - 4)]; v.x += ga * u.x; v.y += ga * u.y; }
        }
        a[q] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PH; ++q) {
      const int idx = threadIdx.x + q * kFastThreads;
      const int t = COLS ? idx % TW : idx / HALF, k = h * HALF + (COLS ? idx / TW : idx % HALF);
      if (idx < HALF * TW && t < nt) buf[I::at(t, k)] = a[q];
    }
    __syncthreads();
  }
  // DCT-III pre-twiddle: rows k and N - k of a line are formed from the same two values, so one
  // thread reads both and writes both (row 0 is unchanged; row N/2 pairs with itself).
  for (int idx = threadIdx.x; idx < HALF * TW; idx += kFastThreads) {
    const int t = COLS ? idx % TW : idx / HALF, k = 1 + (COLS ? idx / TW : idx % HALF);
    if (t >= nt) continue;
    const C x = buf[I::at(t, k)], y = buf[I::at(t, N - k)];
    const C d = mk<C>(x.x + y.y, x.y - y.x);
    buf[I::at(t, k)] = cscale(cmulc(d, __ldg(&dctw[k])), (T)0.5);
    if (k < HALF) {
      const C e = mk<C>(y.x + x.y, y.y - x.x);
      buf[I::at(t, N - k)] = cscale(cmulc(e, __ldg(&dctw[N - k])), (T)0.5);
    }
  }
  __syncthreads();
}

template <typename T, int MODE, typename TS, int N>
__global__ void __launch_bounds__(kFastThreads) k_cheb_fast(const void* __restrict__ in, void* __restrict__ out,
                                                            long inner, int basis, int real,
                                                            const cplx<T>* __restrict__ twf,
                                                            const cplx<T>* __restrict__ dctw) {
  using C = cplx<T>;
  constexpr int TW = fast_tw_cols<T>();
  constexpr int LDP = pad_ld(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const long t0 = (long)blockIdx.x * TW;
  const int nt = (int)min((long)TW, inner - t0);
  const int nb = basis_count(basis, N);

  if (MODE == kChebScalar || MODE == kChebForwardT) {
    staged_copy<N * TW, C>(
        [&](int idx) {
          const int j = idx / TW, t = idx % TW;
          if (t >= nt) return mk<C>((T)0, (T)0);
          const long g = (long)j * inner + t0 + t;
          return real ? mk<C>(reinterpret_cast<const T*>(in)[g], (T)0) : reinterpret_cast<const C*>(in)[g];
        },
        [&](int idx, C v) {
          const int j = idx / TW, t = idx % TW;
          if (t < nt) buf[t * LDP + padi(cheb_reord<N>(j))] = v;
        });
    __syncthreads();
    fft_fast<N, TW, kFastThreads, false>(buf, nt, twf);
    cheb_forward_finish<T, MODE, TS, N>(buf, nt, t0, inner, basis, real, out, dctw);
  } else {  // backward
    staged_copy<N * TW, C>(
        [&](int idx) {
          const int k = idx / TW, t = idx % TW;
          return (t < nt && k < nb) ? from_spec<TS, C>(reinterpret_cast<const TS*>(in), (long)k * inner + t0 + t, real)
                                    : mk<C>((T)0, (T)0);
        },
        [&](int idx, C v) {
          const int k = idx / TW, t = idx % TW;
          if (t < nt) buf[t * LDP + padi(k)] = v;
        });
    __syncthreads();
    cheb_backward_prepare<T, N>(buf, nt, basis, dctw);
    fft_fast<N, TW, kFastThreads, true>(buf, nt, twf);
    for (int idx = threadIdx.x; idx < N * TW; idx += kFastThreads) {
      const int j = idx / TW, t = idx % TW;
      if (t < nt) {
        const C v = buf[t * LDP + padi(cheb_reord<N>(j))];
        const long g = (long)j * inner + t0 + t;
        if (real) reinterpret_cast<T*>(out)[g] = v.x; else reinterpret_cast<C*>(out)[g] = v;
      }
    }
  }
}

template <typename K> inline cudaError_t fast_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

}  // namespace sgm
