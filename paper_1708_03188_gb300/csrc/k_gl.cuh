// k_gl.cuh - complex Ginzburg-Landau right-hand side with the 3/2-rule padded nonlinear term
// (Sec. 6 of the paper) and the RK4 stage updates, on an M x M doubly periodic grid.
//
// Equation (general form; the paper's is beta = 0, gamma = 1.5):
//     u_t = u + (1 + i beta) lap(u) - (1 + i gamma) |u|^2 u,
// in Fourier space  du_hat/dt = L(k) u_hat - N(u_hat),  L(k) = 1 - (1 + i beta) |k|^2 with
// k = 2 pi l / length on each axis.  N(u_hat) is the padded product of Sec. 6: the
// coefficients are copied to an Mp x Mp array (Mp = 3M/2) at the same wavenumbers, zero
// elsewhere, transformed back without scaling, multiplied pointwise by (1 + i gamma)|u|^2,
// transformed forward with 1/Mp per axis and truncated to the original wavenumber set.
//
// Three kernels per right-hand side, all on the compile-time FFT engine of length Mp:
//   K1 k_gl_rows_pad   each of the M spectral rows: zero-pad to Mp, inverse FFT along the
//                      row -> P (M x Mp); the padded rows are zero and never stored.
//   K2 k_gl_cols       each column of P (TW columns per CTA): place the M values at their
//                      padded positions, inverse FFT along the column, pointwise nonlinear
//                      product, forward FFT, keep the M original positions (x 1/Mp), in place.
//   K3 k_gl_rows_out   each row of P: forward FFT (x 1/Mp), truncate to M, then either write
//                      the right-hand side or apply one RK4 stage update (explicit RK4 of the
//                      paper's time loop, or integrating-factor RK4) to the stage input V,
//                      the accumulator A and the state S.  Within a run of stages K3 also does
//                      the next stage's K1 on the rows it holds (PAD_NEXT): the rows of the new
//                      stage input (or, after the last stage, of the new state) are already in
//                      its shared memory, so it zero-pads them, transforms them back and writes
//                      them to P, and a stage costs two launches instead of three.
// Explicit RK4 (a = 1/6, 1/3, 1/3, 1/6; b = 1/2, 1/2, 1), stage s with input V (V = S at s = 0):
//     d = L V - N(V);  s < 3: V <- S + b_s dt d, A <- (s ? A : S) + a_s dt d;  s = 3: S <- A + a_3 dt d.
// Integrating-factor RK4 (classical RK4 on exp(-L t) u_hat, E = exp(L dt / 2)), n = -N(V):
//     s = 0: V <- E (S + dt/2 n),  A <- E^2 S + dt/6 E^2 n
//     s = 1: V <- E S + dt/2 n,    A <- A + dt/3 E n
//     s = 2: V <- E^2 S + dt E n,  A <- A + dt/3 E n
//     s = 3: S <- A + dt/6 n
#pragma once
#include "k_fast.cuh"

namespace sgm {

enum GlMode { kGlRhs = 0, kGlRk4 = 1, kGlIfRk4 = 2 };

struct GlParams {
  double beta, gamma, dt, kscale;   // kscale = 2 pi / domain length
  int stage;
};

// padded position of original index j of a length-M C2C axis, and the inverse map
template <int M, int MP> __device__ __forceinline__ int gl_padpos(int j) { return j < (M + 1) / 2 ? j : j - M + MP; }
template <int M, int MP> __device__ __forceinline__ int gl_origidx(int q) {
  return q < (M + 1) / 2 ? q : (q >= MP - M / 2 ? q - MP + M : -1);
}
template <int M> __device__ __forceinline__ int gl_wavenumber(int j) { return j < (M + 1) / 2 ? j : j - M; }

// Lines per CTA of the row passes and columns per CTA of the column pass: as many as the
// shared-memory budget allows, reduced until the grid has at least 256 CTAs (about two per SM),
// so that small grids do not leave SMs idle.
template <typename T, int M, int MP> __host__ __device__ constexpr int gl_lines() {
  int l = fast_elems<T>() / MP > 0 ? fast_elems<T>() / MP : 1;
  while (l > 1 && (M + l - 1) / l < 256) --l;
  return l;
}
template <typename T, int MP> __host__ __device__ constexpr int gl_tw() {
  return MP / 4 >= 256 ? 4 : (MP / 2 >= 256 ? 2 : 1);
}

template <typename T, int M, int MP>
__global__ void __launch_bounds__(kFastThreads) k_gl_rows_pad(const cplx<T>* __restrict__ U, cplx<T>* __restrict__ P,
                                                              const cplx<T>* __restrict__ twf) {
  using C = cplx<T>;
  constexpr int LINES = gl_lines<T, M, MP>();
  constexpr int LDP = pad_ld(MP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int r0 = blockIdx.x * LINES;
  const int nl = min(LINES, M - r0);
  staged_copy<LINES * MP, C>(
      [&](int idx) {
        const int line = idx / MP, q = idx - line * MP;
        const int j = gl_origidx<M, MP>(q);
        return (idx < nl * MP && j >= 0) ? U[(long)(r0 + line) * M + j] : mk<C>((T)0, (T)0);
      },
      [&](int idx, C v) { if (idx < nl * MP) buf[(idx / MP) * LDP + padi(idx % MP)] = v; });
  __syncthreads();
  fft_fast<MP, LINES, kFastThreads, true>(buf, nl, twf);
  for (int idx = threadIdx.x; idx < nl * MP; idx += kFastThreads) {
    const int line = idx / MP, q = idx - line * MP;
    P[(long)(r0 + line) * MP + q] = buf[line * LDP + padi(q)];
  }
}

template <typename T, int M, int MP>
__global__ void __launch_bounds__(kFastThreads) k_gl_cols(cplx<T>* __restrict__ P, const cplx<T>* __restrict__ twf,
                                                          double gamma) {
  using C = cplx<T>;
  constexpr int TW = gl_tw<T, MP>();
  constexpr int LDP = pad_ld(MP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int c0 = blockIdx.x * TW;
  const int nt = min(TW, MP - c0);
  staged_copy<MP * TW, C>(
      [&](int idx) {
        const int q = idx / TW, t = idx % TW;
        const int j = gl_origidx<M, MP>(q);
        return (t < nt && j >= 0) ? P[(long)j * MP + c0 + t] : mk<C>((T)0, (T)0);
      },
      [&](int idx, C v) {
        const int q = idx / TW, t = idx % TW;
        if (t < nt) buf[t * LDP + padi(q)] = v;
      });
  __syncthreads();
  fft_fast<MP, TW, kFastThreads, true>(buf, nt, twf);
  const T g = (T)gamma;
  for (int idx = threadIdx.x; idx < MP * TW; idx += kFastThreads) {
    const int t = idx / MP, q = idx - t * MP;
    if (t < nt) {
      const C u = buf[t * LDP + padi(q)];
      const T s2 = u.x * u.x + u.y * u.y;
      buf[t * LDP + padi(q)] = mk<C>(s2 * (u.x - g * u.y), s2 * (u.y + g * u.x));   // (1 + i gamma)|u|^2 u
    }
  }
  __syncthreads();
  fft_fast<MP, TW, kFastThreads, false>(buf, nt, twf);
  const T s = (T)1 / (T)MP;
  for (int idx = threadIdx.x; idx < M * TW; idx += kFastThreads) {
    const int j = idx / TW, t = idx % TW;
    if (t < nt) P[(long)j * MP + c0 + t] = cscale(buf[t * LDP + padi(gl_padpos<M, MP>(j))], s);
  }
}

template <typename T, int M, int MP, int MODE, bool PAD_NEXT>
__global__ void __launch_bounds__(kFastThreads) k_gl_rows_out(cplx<T>* __restrict__ P, const cplx<T>* Vin,
                                                              cplx<T>* Vout, cplx<T>* A, cplx<T>* S,
                                                              const cplx<T>* __restrict__ E, cplx<T>* out,
                                                              const __grid_constant__ GlParams prm,
                                                              const cplx<T>* __restrict__ twf) {
  using C = cplx<T>;
  constexpr int LINES = gl_lines<T, M, MP>();
  constexpr int LDP = pad_ld(MP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int r0 = blockIdx.x * LINES;
  const int nl = min(LINES, M - r0);
  staged_copy<LINES * MP, C>(
      [&](int idx) { return idx < nl * MP ? P[(long)r0 * MP + idx] : mk<C>((T)0, (T)0); },
      [&](int idx, C v) { if (idx < nl * MP) buf[(idx / MP) * LDP + padi(idx % MP)] = v; });
  __syncthreads();
  fft_fast<MP, LINES, kFastThreads, false>(buf, nl, twf);
  const T inv = (T)1 / (T)MP;
  const T beta = (T)prm.beta, dt = (T)prm.dt, ks = (T)prm.kscale;
  for (int idx = threadIdx.x; idx < nl * M; idx += kFastThreads) {
    const int line = idx / M, j = idx - line * M;
    const int r = r0 + line;
    const long g = (long)r * M + j;
    C* slot = &buf[line * LDP + padi(gl_padpos<M, MP>(j))];   // read and rewritten by this thread only
    const C nl_ = cscale(*slot, inv);                          // N(V) at (r, j)
    C nv = mk<C>((T)0, (T)0);                                  // next stage input (or new state) at (r, j)
    if (MODE == kGlIfRk4) {
      const C n = mk<C>(-nl_.x, -nl_.y);
      const C e = E[g];
      const C s = S[g];
      switch (prm.stage) {
        case 0: {
          const C e2 = cmul(e, e);
          nv = cmul(e, mk<C>(s.x + (T)0.5 * dt * n.x, s.y + (T)0.5 * dt * n.y));
          Vout[g] = nv;
          const C t = cadd(s, cscale(n, dt / (T)6));
          A[g] = cmul(e2, t);
          break;
        }
        case 1: {
          const C es = cmul(e, s);
          nv = mk<C>(es.x + (T)0.5 * dt * n.x, es.y + (T)0.5 * dt * n.y);
          Vout[g] = nv;
          const C en = cmul(e, n);
          const C a = A[g];
          A[g] = mk<C>(a.x + dt / (T)3 * en.x, a.y + dt / (T)3 * en.y);
          break;
        }
        case 2: {
          const C e2 = cmul(e, e);
          const C en = cmul(e, n);
          const C e2s = cmul(e2, s);
          nv = mk<C>(e2s.x + dt * en.x, e2s.y + dt * en.y);
          Vout[g] = nv;
          const C a = A[g];
          A[g] = mk<C>(a.x + dt / (T)3 * en.x, a.y + dt / (T)3 * en.y);
          break;
        }
        default: {
          const C a = A[g];
          nv = mk<C>(a.x + dt / (T)6 * n.x, a.y + dt / (T)6 * n.y);
          S[g] = nv;
          break;
        }
      }
    } else {
      const T kx = ks * (T)gl_wavenumber<M>(r), ky = ks * (T)gl_wavenumber<M>(j);
      const T k2 = kx * kx + ky * ky;
      const C v = Vin[g];
      // L v = (1 - k2) v - i beta k2 v
      const C d = mk<C>((1 - k2) * v.x + beta * k2 * v.y - nl_.x, (1 - k2) * v.y - beta * k2 * v.x - nl_.y);
      if (MODE == kGlRhs) {
        out[g] = d;
      } else {
        const int st = prm.stage;
        const T a_s = (st == 0 || st == 3) ? (T)1 / (T)6 : (T)1 / (T)3;
        const T b_s = (st == 2) ? (T)1 : (T)0.5;
        if (st < 3) {
          const C s = S[g];
          const C base = (st == 0) ? s : A[g];
          A[g] = mk<C>(base.x + a_s * dt * d.x, base.y + a_s * dt * d.y);
          nv = mk<C>(s.x + b_s * dt * d.x, s.y + b_s * dt * d.y);
          Vout[g] = nv;
        } else {
          const C a = A[g];
          nv = mk<C>(a.x + a_s * dt * d.x, a.y + a_s * dt * d.y);
          S[g] = nv;
        }
      }
    }
    if constexpr (PAD_NEXT) *slot = nv;
  }
  if constexpr (PAD_NEXT) {
    // the next stage's K1 on these rows: the padded positions that hold no original wavenumber
    // (read by no thread above) become zero, then the rows are transformed back into P
    constexpr int NZ = MP - M;
    for (int idx = threadIdx.x; idx < nl * NZ; idx += kFastThreads) {
      const int line = idx / NZ, q = (M + 1) / 2 + (idx - line * NZ);
      buf[line * LDP + padi(q)] = mk<C>((T)0, (T)0);
    }
    __syncthreads();
    fft_fast<MP, LINES, kFastThreads, true>(buf, nl, twf);
    for (int idx = threadIdx.x; idx < nl * MP; idx += kFastThreads) {
      const int line = idx / MP, q = idx - line * MP;
      P[(long)(r0 + line) * MP + q] = buf[line * LDP + padi(q)];
    }
  }
}

// ---- launch of one right-hand side evaluation + stage update --------------------------------
// pad_first: run K1 on Vin (otherwise P already holds the padded, back-transformed rows of Vin,
// written by the previous launch with pad_next); pad_next: K3 also prepares P for the next stage
// from the stage's result (the new V, or S after stage 3).
template <typename T, int M, int MP, int MODE>
cudaError_t gl_rows_out(bool pad_next, unsigned grid, size_t smem, cplx<T>* P, const cplx<T>* Vin,
                        cplx<T>* Vout, cplx<T>* A, cplx<T>* S, const cplx<T>* E, cplx<T>* out, const GlParams& prm,
                        const cplx<T>* twf, cudaStream_t st) {
  cudaError_t e;
  if (pad_next) {
    if ((e = fast_smem(k_gl_rows_out<T, M, MP, MODE, true>, smem)) != cudaSuccess) return e;
    k_gl_rows_out<T, M, MP, MODE, true><<<grid, kFastThreads, smem, st>>>(P, Vin, Vout, A, S, E, out, prm, twf);
  } else {
    if ((e = fast_smem(k_gl_rows_out<T, M, MP, MODE, false>, smem)) != cudaSuccess) return e;
    k_gl_rows_out<T, M, MP, MODE, false><<<grid, kFastThreads, smem, st>>>(P, Vin, Vout, A, S, E, out, prm, twf);
  }
  return cudaSuccess;
}

template <typename T, int M, int MP>
cudaError_t gl_launch_sized(int mode, bool pad_first, bool pad_next, const cplx<T>* Vin, cplx<T>* Vout, cplx<T>* A,
                            cplx<T>* S, const cplx<T>* E, cplx<T>* out, cplx<T>* P, const GlParams& prm,
                            const cplx<T>* twf, cudaStream_t st) {
  constexpr int LINES = gl_lines<T, M, MP>();
  constexpr int TW = gl_tw<T, MP>();
  const size_t smem_rows = sizeof(cplx<T>) * LINES * pad_ld(MP);
  const size_t smem_cols = sizeof(cplx<T>) * TW * pad_ld(MP);
  cudaError_t e;
  if ((e = fast_smem(k_gl_rows_pad<T, M, MP>, smem_rows)) != cudaSuccess) return e;
  if ((e = fast_smem(k_gl_cols<T, M, MP>, smem_cols)) != cudaSuccess) return e;
  const unsigned grows = (M + LINES - 1) / LINES;
  if (pad_first) k_gl_rows_pad<T, M, MP><<<grows, kFastThreads, smem_rows, st>>>(Vin, P, twf);
  k_gl_cols<T, M, MP><<<(MP + TW - 1) / TW, kFastThreads, smem_cols, st>>>(P, twf, prm.gamma);
  switch (mode) {
    case kGlRhs:
      e = gl_rows_out<T, M, MP, kGlRhs>(false, grows, smem_rows, P, Vin, Vout, A, S, E, out, prm, twf, st);
      break;
    case kGlRk4:
      e = gl_rows_out<T, M, MP, kGlRk4>(pad_next, grows, smem_rows, P, Vin, Vout, A, S, E, out, prm, twf, st);
      break;
    default:
      e = gl_rows_out<T, M, MP, kGlIfRk4>(pad_next, grows, smem_rows, P, Vin, Vout, A, S, E, out, prm, twf, st);
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T>
cudaError_t gl_launch(int M, int mode, bool pad_first, bool pad_next, const cplx<T>* Vin, cplx<T>* Vout, cplx<T>* A,
                      cplx<T>* S, const cplx<T>* E, cplx<T>* out, cplx<T>* P, const GlParams& prm,
                      const cplx<T>* twf, cudaStream_t st) {
  switch (M) {
#define SGM_GL(m)                                                                                                \
  case m:                                                                                                        \
    return gl_launch_sized<T, m, 3 * m / 2>(mode, pad_first, pad_next, Vin, Vout, A, S, E, out, P, prm, twf, st);
    SGM_GL(32) SGM_GL(64) SGM_GL(128) SGM_GL(256) SGM_GL(512) SGM_GL(1024)
#undef SGM_GL
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sgm
