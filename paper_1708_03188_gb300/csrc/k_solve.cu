// k_solve.cu - per-wavenumber FP64 solves along the Chebyshev axis.
//
// For every Fourier column (squared wavenumber kappa2, Eq. laplace of the paper) and each
// parity of the Chebyshev index (the Galerkin matrices couple only equal parities), one
// thread solves its system by Gaussian elimination without pivoting, top-down, in FP64:
//
// Shen-Dirichlet, a lap(u) + b u = f (Sec. 3.4.2, Sec. 4):  M = a A + aB B, aB = b - a kappa2.
//   Within a parity, with i the position (k = 2i + p):
//     B: diagonal B0_k = pi/2 (c_k + 1), off-diagonals -pi/2;
//     A: upper triangular, diagonal -2 pi (k+1)(k+2), every entry right of it -4 pi (k+1).
//   Row i: ell u_{i-1} + d_i u_i + (g_i + ell) u_{i+1} + g_i sum_{j>=i+2} u_j,  ell = -aB pi/2,
//   g_i = -4 pi a (k+1).  Eliminating the sub-diagonal keeps that shape: the reduced row has
//   pivot d'_i, super-diagonal g'_i + ell and tail coefficient g'_i with
//     mu = ell / d'_{i-1},  d'_i = d_i - mu (g'_{i-1} + ell),  g'_i = g_i - mu g'_{i-1},
//     f'_i = f_i - mu f'_{i-1};
//   back substitution  u_i = (f'_i - ell u_{i+1} - g'_i sum_{j>=i+1} u_j) / d'_i.
//
// Shen-biharmonic, a lap^2 u + b lap u + c u = f (Sec. 4):
//   M = a S + aA A + aB B, aA = b - 2 a kappa2, aB = a kappa2^2 - b kappa2 + c.
//   Within a parity: B pentadiagonal, A tridiagonal, S upper triangular whose entries two or
//   more positions right of the diagonal are the rank-2 product G0_m F0_l + G1_m F1_l
//   (the T_l'''' coefficient polynomial in the row degree, with the boundary conditions
//   of phi_m removing its two lowest powers).  Rows are kept as [pivot, two
//   super-diagonals, two tail coefficients on the rank-2 weights F0, F1 from 3 positions
//   right]; each row eliminates its two sub-diagonal entries against the two reduced rows
//   above it.
//
// The per-row reduced quantities are written to a global FP64 scratch laid out
// [row][value][thread] (a warp's 32 threads touch 256 contiguous bytes) and read back by
// the back substitution.  Warps own 32 neighbouring columns of one parity, so every load
// and store of a row is coalesced.  Reciprocals: an FP32 seed refined by two
// Newton-Raphson steps in FP64 (r <- r + r (1 - x r)), each squaring the relative error.
#include <algorithm>

#include "common.cuh"

namespace sgm {

__device__ __forceinline__ double rcp64(double x) {
  const float xf = (float)x;
  const float ax = fabsf(xf);
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

template <typename T> __device__ __forceinline__ double2 ld2(const void* p, long i, bool real) {
  if (real) return make_double2((double)reinterpret_cast<const T*>(p)[i], 0.0);
  const cplx<T> v = reinterpret_cast<const cplx<T>*>(p)[i];
  return make_double2((double)v.x, (double)v.y);
}
template <typename T> __device__ __forceinline__ void st2(void* p, long i, bool real, double2 v) {
  if (real) { reinterpret_cast<T*>(p)[i] = (T)v.x; return; }
  cplx<T> w; w.x = (T)v.x; w.y = (T)v.y;
  reinterpret_cast<cplx<T>*>(p)[i] = w;
}

// table indices
enum { TD_B0 = 0, TD_A0 = 1, TD_G = 2, TD_COUNT = 3 };
enum { TB_B0 = 0, TB_B2, TB_B4, TB_ALO, TB_A0, TB_AUP, TB_S0, TB_S1, TB_S2, TB_G0, TB_G1, TB_F0, TB_F1, TB_COUNT };

template <typename T>
__global__ void __launch_bounds__(128) k_solve_dirichlet(const void* __restrict__ in, void* __restrict__ out, int N,
                                                         long ncols, int real, double a, double b,
                                                         const __grid_constant__ Wavenumbers wn,
                                                         const double* __restrict__ tab, int ts,
                                                         double* __restrict__ scratch) {
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwarps_total = nth / 32;
  const long ncb = (ncols + 31) / 32;
  const int nb = N - 2;
  const double* B0 = tab + TD_B0 * ts;
  const double* A0 = tab + TD_A0 * ts;
  const double* G = tab + TD_G * ts;
  for (long w = gt / 32; w < 2 * ncb; w += nwarps_total) {
    const int p = (int)(w & 1);
    const long c = (w >> 1) * 32 + lane;
    if (c >= ncols) continue;
    const double k2 = kappa2_of(wn, c);
    const double aB = b - a * k2;
    const double ell = -aB * 1.5707963267948966;
    const int n = (nb - p + 1) / 2;
    double pr = 0.0, pg = 0.0;
    double2 pf = make_double2(0.0, 0.0);
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double2 f = ld2<T>(in, (long)k * ncols + c, real);
      double d = fma(a, __ldg(&A0[k]), aB * __ldg(&B0[k]));
      double g = a * __ldg(&G[k]);
      if (i > 0) {
        const double mu = ell * pr;
        d = fma(-mu, pg + ell, d);
        g = fma(-mu, pg, g);
        f.x = fma(-mu, pf.x, f.x);
        f.y = fma(-mu, pf.y, f.y);
      }
      const double r = rcp64(d);
      double* s = scratch + (long)i * 4 * nth + gt;
      s[0] = r;
      s[nth] = g;
      s[2 * nth] = f.x;
      s[3 * nth] = f.y;
      pr = r; pg = g; pf = f;
    }
    double2 un = make_double2(0.0, 0.0), Ts = make_double2(0.0, 0.0);
    for (int i = n - 1; i >= 0; --i) {
      const int k = p + 2 * i;
      const double* s = scratch + (long)i * 4 * nth + gt;
      const double r = s[0], g = s[nth];
      Ts.x += un.x; Ts.y += un.y;
      double2 u;
      u.x = (s[2 * nth] - ell * un.x - g * Ts.x) * r;
      u.y = (s[3 * nth] - ell * un.y - g * Ts.y) * r;
      st2<T>(out, (long)k * ncols + c, real, u);
      un = u;
    }
    for (int k = nb + p; k < N; k += 2) st2<T>(out, (long)k * ncols + c, real, make_double2(0.0, 0.0));
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_solve_biharmonic(const void* __restrict__ in, void* __restrict__ out,
                                                          int N, long ncols, int real, double a, double b,
                                                          double cc, const __grid_constant__ Wavenumbers wn,
                                                          const double* __restrict__ tab, int ts,
                                                          double* __restrict__ scratch) {
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwarps_total = nth / 32;
  const long ncb = (ncols + 31) / 32;
  const int nb = N - 4;
  auto tb = [&](int t, int k) -> double { return __ldg(&tab[t * ts + k]); };
  for (long w = gt / 32; w < 2 * ncb; w += nwarps_total) {
    const int p = (int)(w & 1);
    const long c = (w >> 1) * 32 + lane;
    if (c >= ncols) continue;
    const double k2 = kappa2_of(wn, c);
    const double aA = b - 2.0 * a * k2;
    const double aB = fma(a * k2, k2, fma(-b, k2, cc));
    const int n = (nb - p + 1) / 2;
    // reduced rows i-1 (suffix 1) and i-2 (suffix 2)
    double r1 = 0, U11 = 0, U21 = 0, g01 = 0, g11 = 0;
    double r2 = 0, U12 = 0, U22 = 0, g02 = 0, g12 = 0;
    double2 f1 = make_double2(0, 0), f2 = make_double2(0, 0);
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double2 f = ld2<T>(in, (long)k * ncols + c, real);
      double D = fma(a, tb(TB_S0, k), fma(aA, tb(TB_A0, k), aB * tb(TB_B0, k)));
      double u1 = fma(a, tb(TB_S1, k), fma(aA, tb(TB_AUP, k), aB * tb(TB_B2, k)));
      double u2 = fma(a, tb(TB_S2, k), aB * tb(TB_B4, k));
      double h0 = a * tb(TB_G0, k), h1 = a * tb(TB_G1, k);
      const double F0a = tb(TB_F0, k + 2), F1a = tb(TB_F1, k + 2);
      const double F0b = tb(TB_F0, k + 4), F1b = tb(TB_F1, k + 4);
      if (i >= 2) {
        double L1 = fma(aA, tb(TB_ALO, k), aB * tb(TB_B2, k - 2));
        const double mu = aB * tb(TB_B4, k - 4) * r2;
        L1 = fma(-mu, U12, L1);
        D = fma(-mu, U22, D);
        u1 = fma(-mu, fma(g02, F0a, g12 * F1a), u1);
        u2 = fma(-mu, fma(g02, F0b, g12 * F1b), u2);
        h0 = fma(-mu, g02, h0);
        h1 = fma(-mu, g12, h1);
        f.x = fma(-mu, f2.x, f.x);
        f.y = fma(-mu, f2.y, f.y);
        const double mu1 = L1 * r1;
        D = fma(-mu1, U11, D);
        u1 = fma(-mu1, U21, u1);
        u2 = fma(-mu1, fma(g01, F0b, g11 * F1b), u2);
        h0 = fma(-mu1, g01, h0);
        h1 = fma(-mu1, g11, h1);
        f.x = fma(-mu1, f1.x, f.x);
        f.y = fma(-mu1, f1.y, f.y);
      } else if (i == 1) {
        const double L1 = fma(aA, tb(TB_ALO, k), aB * tb(TB_B2, k - 2));
        const double mu1 = L1 * r1;
        D = fma(-mu1, U11, D);
        u1 = fma(-mu1, U21, u1);
        u2 = fma(-mu1, fma(g01, F0b, g11 * F1b), u2);
        h0 = fma(-mu1, g01, h0);
        h1 = fma(-mu1, g11, h1);
        f.x = fma(-mu1, f1.x, f.x);
        f.y = fma(-mu1, f1.y, f.y);
      }
      const double r = rcp64(D);
      double* s = scratch + (long)i * 7 * nth + gt;
      s[0] = r; s[nth] = u1; s[2 * nth] = u2; s[3 * nth] = h0; s[4 * nth] = h1;
      s[5 * nth] = f.x; s[6 * nth] = f.y;
      r2 = r1; U12 = U11; U22 = U21; g02 = g01; g12 = g11; f2 = f1;
      r1 = r; U11 = u1; U21 = u2; g01 = h0; g11 = h1; f1 = f;
    }
    double2 ua = make_double2(0, 0), ub = make_double2(0, 0), uc = make_double2(0, 0);  // u_{i+1}, u_{i+2}, u_{i+3}
    double2 T0 = make_double2(0, 0), T1 = make_double2(0, 0);
    for (int i = n - 1; i >= 0; --i) {
      const int k = p + 2 * i;
      if (i + 3 < n) {
        const double F0 = tb(TB_F0, k + 6), F1 = tb(TB_F1, k + 6);
        T0.x = fma(F0, uc.x, T0.x); T0.y = fma(F0, uc.y, T0.y);
        T1.x = fma(F1, uc.x, T1.x); T1.y = fma(F1, uc.y, T1.y);
      }
      const double* s = scratch + (long)i * 7 * nth + gt;
      const double r = s[0], u1 = s[nth], u2 = s[2 * nth], h0 = s[3 * nth], h1 = s[4 * nth];
      double2 u;
      u.x = (s[5 * nth] - u1 * ua.x - u2 * ub.x - h0 * T0.x - h1 * T1.x) * r;
      u.y = (s[6 * nth] - u1 * ua.y - u2 * ub.y - h0 * T0.y - h1 * T1.y) * r;
      st2<T>(out, (long)k * ncols + c, real, u);
      uc = ub; ub = ua; ua = u;
    }
    for (int k = nb + p; k < N; k += 2) st2<T>(out, (long)k * ncols + c, real, make_double2(0.0, 0.0));
  }
}

template <typename T>
cudaError_t launch_solve(int basis, bool real, double a, double b, double c, const void* in, void* out, int N,
                         long ncols, const Wavenumbers& wn, const double* tab, double* scratch,
                         long scratch_threads, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const long warps_needed = 2 * ((ncols + 31) / 32);
  long threads = std::min(scratch_threads, warps_needed * 32);
  threads = std::max(128L, (threads / 128) * 128);
  const unsigned grid = (unsigned)(threads / 128);
  const int ts = N + 8;
  if (basis == kDirichlet)
    k_solve_dirichlet<T><<<grid, 128, 0, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, wn, tab, ts, scratch);
  else
    k_solve_biharmonic<T><<<grid, 128, 0, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, c, wn, tab, ts, scratch);
  return cudaGetLastError();
}

template cudaError_t launch_solve<float>(int, bool, double, double, double, const void*, void*, int, long,
                                         const Wavenumbers&, const double*, double*, long, cudaStream_t);
template cudaError_t launch_solve<double>(int, bool, double, double, double, const void*, void*, int, long,
                                          const Wavenumbers&, const double*, double*, long, cudaStream_t);

}  // namespace sgm
