// fft_core.cuh - batched mixed-radix Stockham FFT on lines held in shared memory.
//
// A CTA holds `nlines` complex lines of length L (line b starts at b * ld) in buffer
// X and transforms all of them with the passes of an FftPlan, ping-ponging between X
// and a second buffer Y of the same layout.  Pass p with radix R and Ns = product of
// the earlier radices reads X[j + r L/R] (r < R), applies the twiddles
// w^(k r), w = exp(-+ 2 pi i / (Ns R)), k = j mod Ns, takes an R-point DFT and writes
// Y[(j/Ns) Ns R + k + s Ns] (s < R): the self-sorting (Stockham) ordering, so the
// result is in natural order without a bit-reversal step.  Radices 2, 3, 4, 5, 8
// have straight-line butterflies; any other factor uses an O(R) sum per output.
// Forward = exp(-i ...) with no scaling; inverse = exp(+i ...), no scaling.
#pragma once
#include "common.cuh"

namespace sgm {

template <typename C> __device__ __forceinline__ C twiddle(const C* __restrict__ tw, int idx, bool inv) {
  C w = __ldg(&tw[idx]);
  if (inv) w.y = -w.y;
  return w;
}

template <int R, bool INV, typename C> __device__ __forceinline__ void butterfly(C* v) {
  using T = decltype(C::x);
  if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else if constexpr (R == 8) {
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    butterfly<4, INV>(e);
    butterfly<4, INV>(o);
    const T h = (T)0.70710678118654752440;
    // o[s] *= W8^s
    o[1] = INV ? mk<C>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
               : mk<C>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    o[2] = rot90<INV>(o[2]);
    o[3] = INV ? mk<C>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
               : mk<C>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      v[s] = cadd(e[s], o[s]);
      v[s + 4] = csub(e[s], o[s]);
    }
  } else if constexpr (R == 3) {
    const T c = (T)-0.5, sn = (T)0.86602540378443864676;
    C t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m = mk<C>(v[0].x + c * t.x, v[0].y + c * t.y);
    C r = rot90<INV>(cscale(d, sn));  // -i sn d (forward)
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  } else if constexpr (R == 5) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    C m1 = mk<C>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
    C m2 = mk<C>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
    C r1 = rot90<INV>(mk<C>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
    C r2 = rot90<INV>(mk<C>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(m1, r1);
    v[4] = csub(m1, r1);
    v[2] = cadd(m2, r2);
    v[3] = csub(m2, r2);
  }
}

// One fixed-radix Stockham pass over all lines.
template <int R, bool INV, typename C>
__device__ __forceinline__ void pass_fixed(const C* X, C* Y, int L, int Ns, int nlines, int ld,
                                           const C* __restrict__ tw) {
  const int Lr = L / R;
  const int total = nlines * Lr;
  const int tws = L / (Ns * R);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = b / Lr, j = b - line * Lr;
    const C* x = X + (long)line * ld;
    C* y = Y + (long)line * ld;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[j + r * Lr];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle(tw, k * r * tws, INV));
    }
    butterfly<R, INV>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int s = 0; s < R; ++s) y[base + s * Ns] = v[s];
  }
}

// Generic-radix pass: every output is an O(R) sum over the R inputs of its butterfly.
template <bool INV, typename C>
__device__ __forceinline__ void pass_generic(const C* X, C* Y, int L, int R, int Ns, int nlines, int ld,
                                             const C* __restrict__ tw) {
  const int Lr = L / R;
  const int total = nlines * L;
  const int tws = L / (Ns * R);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = b / L, rem = b - line * L;
    const int j = rem / R, s = rem - j * R;
    const C* x = X + (long)line * ld;
    const int k = j % Ns;
    // exponent of input r: r (k + s Ns) / (Ns R) turns = r (k + s Ns) tws / L
    const int step = ((k + s * Ns) * tws) % L;
    int idx = 0;
    C acc = mk<C>(0, 0);
    for (int r = 0; r < R; ++r) {
      acc = cadd(acc, cmul(x[j + r * Lr], twiddle(tw, idx, INV)));
      idx += step;
      if (idx >= L) idx -= L;
    }
    Y[(long)line * ld + (j - k) * R + k + s * Ns] = acc;
  }
}

// Transform all lines; data starts in A, B is scratch.  Returns the buffer holding the
// result.  Ends with __syncthreads().
template <bool INV, typename C>
__device__ C* fft_lines(C* A, C* B, int nlines, int ld, const FftPlan& p, const C* __restrict__ tw) {
  int Ns = 1;
  for (int ip = 0; ip < p.npass; ++ip) {
    const int R = p.radix[ip];
    switch (R) {
      case 2: pass_fixed<2, INV>(A, B, p.L, Ns, nlines, ld, tw); break;
      case 3: pass_fixed<3, INV>(A, B, p.L, Ns, nlines, ld, tw); break;
      case 4: pass_fixed<4, INV>(A, B, p.L, Ns, nlines, ld, tw); break;
      case 5: pass_fixed<5, INV>(A, B, p.L, Ns, nlines, ld, tw); break;
      case 8: pass_fixed<8, INV>(A, B, p.L, Ns, nlines, ld, tw); break;
      default: pass_generic<INV>(A, B, p.L, R, Ns, nlines, ld, tw); break;
    }
    __syncthreads();
    C* t = A; A = B; B = t;
    Ns *= R;
  }
  return A;
}

// Bluestein (chirp-z) DFT of one line of length N via a circular convolution of length L, a
// length with a fast plan (L >= 2N - 1).  With the chirp c_n = exp(-i pi n^2 / N), the identity
// j k = (j^2 + k^2 - (k - j)^2) / 2 turns the forward DFT into
//     X_k = c_k sum_j (x_j c_j) conj(c_{k-j}),
// a convolution of a_j = x_j c_j with b_n = conj(c_|n|); the inverse DFT conjugates every chirp.
// chirp[n] (n < N) holds c_n; bhat[m] (m < L) holds FFT_L(b) / L with b circularly wrapped
// (b_{L-n} = b_n); for the inverse, FFT_L(conj b)_m = conj(bhat[(L - m) mod L]).
// The line's N values are in A; A and B hold >= L elements.  Returns the buffer holding the N
// results.  Ends with __syncthreads().
template <bool INV, typename C>
__device__ C* bluestein(C* A, C* B, int N, int L, const FftPlan& pL, const C* __restrict__ twL,
                        const C* __restrict__ chirp, const C* __restrict__ bhat) {
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    C v = mk<C>(0, 0);
    if (j < N) v = cmul(A[j], twiddle(chirp, j, INV));
    A[j] = v;
  }
  __syncthreads();
  C* Y = fft_lines<false>(A, B, 1, L, pL, twL);
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    C h;
    if (INV) {
      h = __ldg(&bhat[m == 0 ? 0 : L - m]);
      h.y = -h.y;
    } else {
      h = __ldg(&bhat[m]);
    }
    Y[m] = cmul(Y[m], h);
  }
  __syncthreads();
  C* R = fft_lines<true>(Y, Y == A ? B : A, 1, L, pL, twL);
  for (int k = threadIdx.x; k < N; k += blockDim.x) R[k] = cmul(R[k], twiddle(chirp, k, INV));
  __syncthreads();
  return R;
}

}  // namespace sgm
