// k_batch.cu - batched independent 1-D Shen-Dirichlet Helmholtz problems
//     u_p'' - alpha_p u_p = f_p  on [-1, 1], u_p(+-1) = 0,   p = 0..P-1,
// each with its own number of Chebyshev-Gauss points N_p (any 4 <= N_p <= 4096), transform +
// solve + transform (the weak form of Sec. 3.4.2 with a = 1, b = -alpha_p, kappa = 0).
//
// Work decomposition for GB300, where an FP64 warp-instruction occupies its sub-partition's
// FP64 pipe for ~64 cycles whatever the number of active lanes:
//   K_A  one CTA per problem: DCT-II of the real samples via one complex FFT (runtime-radix
//        engine; a size with a prime factor above 32 runs its DFT as Bluestein's chirp-z
//        convolution of a power-of-two length instead of an O(N p) generic-radix pass),
//        Dirichlet stencil S_k = t_k - t_{k+2}; S_k is written in FP64 into a
//        warp-interleaved layout [warp][row][lane] (problems sorted by N, 32 per warp).
//   K_B  two threads per (problem, parity), one per half of the rows: the two-sided FP64
//        elimination of k_solve.cu's Dirichlet kernels with kappa = 0, lanes = 32 problems of
//        similar size, so every FP64 instruction serves 32 problems and every load/store of a
//        row is one 256-byte access.
//   K_C  one CTA per problem: stencil a_k = u_k - u_{k-2} and DCT-III back to the points.
#include <algorithm>

#include "convert.cuh"
#include "fft_core.cuh"

namespace sgm {

struct BatchProblem {
  int N;          // Chebyshev points
  int slot;       // position in the size-sorted order: warp = slot / 32, lane = slot % 32
  long offset;    // first element of f_p / u_p in the caller's arrays
  double alpha;
  int tw_off;     // exp(-2 pi i k / N), k < N (or / L, k < L with Bluestein), in the twiddle pool
  int dct_off;    // exp(-i pi k / (2N)), k < N, in the twiddle pool
  int plan;       // index into the plan table (of length N, or of L with Bluestein)
  int L;          // 0: direct FFT of length N; else Bluestein convolution length
  int chirp_off;  // Bluestein: exp(-i pi n^2 / N), n < N, in the twiddle pool
  int bhat_off;   // Bluestein: FFT_L of the wrapped conjugate chirp, / L, in the twiddle pool
};

// interleaved FP64 arrays: element (row k, slot s) at wbase[s / 32] + k * 32 + s % 32
__device__ __forceinline__ long ilv(const long* wbase, int slot, int k) {
  return wbase[slot >> 5] + (long)k * 32 + (slot & 31);
}

template <typename T>
__global__ void __launch_bounds__(256) k_batch_dct(const T* __restrict__ f, const BatchProblem* __restrict__ probs,
                                                   const int* __restrict__ by_slot, const FftPlan* __restrict__ plans,
                                                   const cplx<T>* __restrict__ pool, const long* __restrict__ wbase,
                                                   double* __restrict__ S, int ldb) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchProblem pr = probs[by_slot[blockIdx.x]];   // largest problems first
  const int N = pr.N;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + ldb;
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    A[(j & 1) ? N - 1 - (j >> 1) : (j >> 1)] = mk<C>(f[pr.offset + j], (T)0);
  __syncthreads();
  const FftPlan plan = plans[pr.plan];
  C* V = pr.L ? bluestein<false>(A, B, N, pr.L, plan, pool + pr.tw_off, pool + pr.chirp_off, pool + pr.bhat_off)
              : fft_lines<false>(A, B, 1, ldb, plan, pool + pr.tw_off);
  C* M = (V == A) ? B : A;
  const C* dctw = pool + pr.dct_off;
  const T scale = (T)3.14159265358979323846 / (T)N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const C v = V[k], vr = cconj(V[k == 0 ? 0 : N - k]);
    const C w = __ldg(&dctw[k]);
    const C a = cadd(v, vr);
    M[k] = mk<C>((T)0.5 * scale * (w.x * a.x - w.y * a.y), (T)0);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    S[ilv(wbase, pr.slot, k)] = k < N - 2 ? widen<T>(M[k].x - M[k + 2].x) : 0.0;
}

__device__ __forceinline__ double rcp64b(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// K_B.  U (interleaved) receives the Shen coefficients.  coef[k] = (-2 pi (k+1)(k+2),
// -4 pi (k+1)) (the diagonal and the constant upper entries of the Dirichlet stiffness rows) and
// mass[k] = B_kk (3 pi / 2 for k = 0, else pi) come from host tables: the row coefficients cost
// loads instead of FP64 instructions on the critical path.
// A CTA of four warps owns one slot warp (32 problems); warp (p, side) takes parity p, side 0
// rows 0 .. h-1 top-down (mu = ell / d'_{i-1}, d'_i = d_i - mu (g'_{i-1} + ell), g'_i = g_i -
// mu g'_{i-1}, f'_i = f_i - mu f'_{i-1}), side 1 rows
// n-1 .. h bottom-up with u_i = a_i + b_i u_{i-1}, T_i = A_i + B_i u_{i-1} (the recurrences of
// k_solve_dirichlet2 in k_solve.cu), h = ceil(n / 2) per problem; the halves meet through
// shared memory at row h-1.  Rows keep their own scratch slot, so both sides share the
// parity's scratch region.  The serial chain of the largest problems is halved.
__global__ void __launch_bounds__(128) k_batch_solve2(const BatchProblem* __restrict__ probs, const int* __restrict__ by_slot,
                                                      const long* __restrict__ wbase, const double* __restrict__ S,
                                                      double* __restrict__ U, double* __restrict__ scratch,
                                                      const long* __restrict__ sbase, int nslots,
                                                      const double2* __restrict__ coef, const double* __restrict__ mass) {
  __shared__ double xch[2][32][5];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = warp & 1, side = warp >> 1;
  const int wslot = blockIdx.x;
  const int slot = wslot * 32 + lane;
  const bool valid = slot < nslots;
  const BatchProblem pr = probs[by_slot[valid ? slot : wslot * 32]];
  const int N = pr.N, nb = N - 2;
  const double pi = 3.141592653589793;
  const double aB = -pr.alpha;       // a = 1, b = -alpha, kappa = 0
  const double ell = -aB * 0.5 * pi;
  const int n = valid ? (nb - p + 1) / 2 : 0, h = (n + 1) / 2;
  const long rbase = wbase[wslot] + lane;
  double* s0 = scratch + sbase[wslot] * 2 + (long)p * (sbase[wslot + 1] - sbase[wslot]) + lane;   // slot of row 0
  double* x = xch[p][lane];
  double dl = 1.0, gl = 0.0, fl = 0.0;
  // the operands of a row (right-hand side, stiffness and mass coefficients) come through a ring
  // of DM rows of loads issued ahead: a row's FP64 work is shorter than the load latency
  constexpr int DM = 4;
  double fb[DM], mb[DM];
  double2 cb[DM];
  auto load_row = [&](int d, int i) {
    const int k = p + 2 * i;
    fb[d] = S[rbase + (long)k * 32];
    cb[d] = __ldg(&coef[k]);
    mb[d] = __ldg(&mass[k]);
  };
  if (side == 0) {
    double pr_ = 0.0, pg = 0.0, pge = 0.0, pf = 0.0;
#pragma unroll
    for (int d = 0; d < DM; ++d)
      if (d < h) load_row(d, d);
    for (int i0 = 0; i0 < h; i0 += DM) {
#pragma unroll
      for (int d = 0; d < DM; ++d) {
        const int i = i0 + d;
        if (i < h) {
          double f = fb[d];
          const double2 c = cb[d];
          const double mk2 = mb[d];
          if (i + DM < h) load_row(d, i + DM);
          double dd = fma(aB, mk2, c.x);
          double g = c.y;
          if (i > 0) {
            const double mu = ell * pr_;
            dd = fma(-mu, pge, dd);
            g = fma(-mu, pg, g);
            f = fma(-mu, pf, f);
          }
          const double r = rcp64b(dd);
          double* s = s0 + (long)i * 96;
          s[0] = r;
          s[32] = g;
          s[64] = f;
          pr_ = r; pg = g; pge = g + ell; pf = f;
          dl = dd; gl = g; fl = f;
        }
      }
    }
  } else {
    double bn = 0.0, Bn = 0.0, an = 0.0, An = 0.0;
    // ring slot d of pass j0 holds row n - 1 - (j0 + d)
#pragma unroll
    for (int d = 0; d < DM; ++d)
      if (n - 1 - d >= h) load_row(d, n - 1 - d);
    for (int j0 = 0; j0 < n - h; j0 += DM) {
#pragma unroll
      for (int d = 0; d < DM; ++d) {
        const int i = n - 1 - (j0 + d);
        if (i >= h) {
          const double f = fb[d];
          const double2 c = cb[d];
          const double mk2 = mb[d];
          if (i - DM >= h) load_row(d, i - DM);
          const double dd = fma(aB, mk2, c.x), g = c.y;
          const double R = rcp64b(fma(g, Bn, fma(ell, bn, dd)));
          const double bi = -ell * R, onep = 1.0 + Bn;
          const double ai = fma(-g, An, fma(-ell, an, f)) * R;
          double* s = s0 + (long)i * 96;
          s[0] = bi;
          s[32] = ai;
          An = fma(onep, ai, An);
          Bn = onep * bi;
          an = ai;
          bn = bi;
        }
      }
    }
    x[0] = an;
    x[1] = An;
    x[2] = bn;
    x[3] = Bn;
  }
  __syncthreads();
  // side 0 forms u_{h-1}; after one synchronisation side 0 back-substitutes rows h-2 .. 0 while
  // side 1 forward-substitutes rows h .. n-1, each through a ring of scratch loads issued ahead
  double un = 0.0, Ts = 0.0;
  if (side == 0 && h > 0) {
    const double ah = x[0], Ah = x[1], bh = x[2], Bh = x[3];
    const double u = fma(-gl, Ah, fma(-ell, ah, fl)) * rcp64b(fma(gl, Bh, fma(ell, bh, dl)));
    x[4] = u;
    U[rbase + (long)(p + 2 * (h - 1)) * 32] = u;
    un = u;
    Ts = fma(Bh, u, Ah);   // T_h
  }
  __syncthreads();
  if (side == 0) {
    // ring slot d of pass j0 holds (r, g, f) of row h - 2 - (j0 + d)
    constexpr int D0 = 4;
    double rb[D0], gb[D0], fb[D0];
#pragma unroll
    for (int d = 0; d < D0; ++d)
      if (h - 2 - d >= 0) {
        const double* s = s0 + (long)(h - 2 - d) * 96;
        rb[d] = s[0];
        gb[d] = s[32];
        fb[d] = s[64];
      }
    for (int j0 = 0; j0 < h - 1; j0 += D0) {
#pragma unroll
      for (int d = 0; d < D0; ++d) {
        const int i = h - 2 - (j0 + d);
        if (i >= 0) {
          const double r = rb[d], g = gb[d], f = fb[d];
          if (i - D0 >= 0) {
            const double* s = s0 + (long)(i - D0) * 96;
            rb[d] = s[0];
            gb[d] = s[32];
            fb[d] = s[64];
          }
          Ts += un;
          const double uu = fma(-g, Ts, fma(-ell, un, f)) * r;
          U[rbase + (long)(p + 2 * i) * 32] = uu;
          un = uu;
        }
      }
    }
  } else if (n > h) {
    // ring slot d of pass i0 holds (b_i, a_i) of row i0 + d
    constexpr int D1 = 8;
    double up = h > 0 ? x[4] : 0.0;
    double bb[D1], ab[D1];
#pragma unroll
    for (int d = 0; d < D1; ++d)
      if (h + d < n) {
        const double* s = s0 + (long)(h + d) * 96;
        bb[d] = s[0];
        ab[d] = s[32];
      }
    for (int i0 = h; i0 < n; i0 += D1) {
#pragma unroll
      for (int d = 0; d < D1; ++d) {
        const int i = i0 + d;
        if (i < n) {
          const double bi = bb[d], ai = ab[d];
          if (i + D1 < n) {
            const double* s = s0 + (long)(i + D1) * 96;
            bb[d] = s[0];
            ab[d] = s[32];
          }
          const double uu = fma(bi, up, ai);
          U[rbase + (long)(p + 2 * i) * 32] = uu;
          up = uu;
        }
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_batch_idct(T* __restrict__ u, const BatchProblem* __restrict__ probs,
                                                    const int* __restrict__ by_slot, const FftPlan* __restrict__ plans,
                                                    const cplx<T>* __restrict__ pool, const long* __restrict__ wbase,
                                                    const double* __restrict__ U, int ldb) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchProblem pr = probs[by_slot[blockIdx.x]];   // largest problems first
  const int N = pr.N, nb = N - 2;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + ldb;
  for (int k = threadIdx.x; k < N; k += blockDim.x)
    B[k] = mk<C>(k < nb ? narrow<T>(U[ilv(wbase, pr.slot, k)]) : (T)0, (T)0);
  __syncthreads();
  for (int k = threadIdx.x; k < N; k += blockDim.x) A[k] = k >= 2 ? csub(B[k], B[k - 2]) : B[k];
  __syncthreads();
  const C* dctw = pool + pr.dct_off;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    C v;
    if (k == 0) {
      v = A[0];
    } else {
      const C x = A[k], y = A[N - k];
      v = cscale(cmulc(mk<C>(x.x + y.y, x.y - y.x), __ldg(&dctw[k])), (T)0.5);
    }
    B[k] = v;
  }
  __syncthreads();
  const FftPlan plan = plans[pr.plan];
  C* R = pr.L ? bluestein<true>(B, A, N, pr.L, plan, pool + pr.tw_off, pool + pr.chirp_off, pool + pr.bhat_off)
              : fft_lines<true>(B, A, 1, ldb, plan, pool + pr.tw_off);
  for (int j = threadIdx.x; j < N; j += blockDim.x) u[pr.offset + j] = R[(j & 1) ? N - 1 - (j >> 1) : (j >> 1)].x;
}

template <typename T>
cudaError_t launch_batch(const void* f, void* u, int nprob, int nslots, int ldb, const void* probs,
                         const int* by_slot, const void* plans, const void* pool, const long* wbase, double* S,
                         double* U, double* scratch, const long* sbase, const void* coef, const double* mass,
                         cudaStream_t s) {
  if (nprob <= 0) return cudaSuccess;
  const size_t smem = 2 * sizeof(cplx<T>) * (size_t)ldb;
  cudaError_t e;
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_batch_dct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_batch_idct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  }
  const BatchProblem* P = (const BatchProblem*)probs;
  k_batch_dct<T><<<nprob, 256, smem, s>>>((const T*)f, P, by_slot, (const FftPlan*)plans, (const cplx<T>*)pool, wbase, S,
                                          ldb);
  k_batch_solve2<<<(nslots + 31) / 32, 128, 0, s>>>(P, by_slot, wbase, S, U, scratch, sbase, nslots,
                                                    (const double2*)coef, mass);
  k_batch_idct<T><<<nprob, 256, smem, s>>>((T*)u, P, by_slot, (const FftPlan*)plans, (const cplx<T>*)pool, wbase, U,
                                           ldb);
  return cudaGetLastError();
}

template cudaError_t launch_batch<float>(const void*, void*, int, int, int, const void*, const int*, const void*,
                                         const void*, const long*, double*, double*, double*, const long*, const void*,
                                         const double*, cudaStream_t);
template cudaError_t launch_batch<double>(const void*, void*, int, int, int, const void*, const int*, const void*,
                                          const void*, const long*, double*, double*, double*, const long*, const void*,
                                          const double*, cudaStream_t);

size_t batch_problem_bytes() { return sizeof(BatchProblem); }

}  // namespace sgm
