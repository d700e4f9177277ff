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
// Work decomposition of the self-contained kernels below (the factored solves of 3-D spaces, further
// down, take one column per thread).  On a 3-D space the columns with Fourier indices (l1, l2) and
// (-l1, l2) have the same kappa2 and hence the same matrix, so one thread eliminates the
// pair (NC = 2): the FP64 factorisation (pivots, reciprocals, tail coefficients) is shared
// and only the right-hand-side recurrences are done per column.  Columns l1 = 0 and
// l1 = -M1/2 have no partner and are solved as a pair of identical columns.  When both
// Fourier axes have the same length and domain, (l1, l2) and (l2, l1) share kappa2 too and
// one thread eliminates the four columns (+-a, b), (+-b, a) (NC = 4): fewer FP64 operations
// per column and about one warp per SM sub-partition on the 256^3 box (the space uses it for the
// biharmonic elimination, whose factorisation dominates; the Dirichlet one keeps pairs and twice
// the warps).  1-D and 2-D spaces use the two-sided kernel k_solve_dirichlet2.  Warps own 32
// consecutive work items of one parity, so every load and store of a row is coalesced.
// The per-row reduced quantities go to a global FP64 scratch laid out [row][value][thread]
// (a warp touches 256 contiguous bytes) and are read back by the back substitution.
// Coefficient tables are pre-multiplied by the call's scalars into shared memory.
// Each sweep loads the next row's operands one row ahead, so the global-memory latency
// overlaps the FP64 work of the current row.
// Reciprocals: the PTX approximate FP64 reciprocal refined by one step of a third-order iteration
// (r <- r + r (e + e^2), e = 1 - x r), which cubes the relative error.  FP32 data is
// widened and narrowed on the integer pipe (convert.cuh).
#include <algorithm>

#include "common.cuh"
#include "convert.cuh"

namespace sgm {

__device__ __forceinline__ double rcp64(double x) {
  // seed: PTX rcp.approx.ftz.f64 (relative error below 2^-22 for normal x); one step of the
  // third-order (Householder's order-2, or Chebyshev's) iteration for 1/x, r (1 + e + e^2) with
  // e = 1 - x r: since 1/x = r / (1 - e) = r (1 + e + e^2 + ...), the truncation leaves a relative
  // error e^3, the cube of the seed's (< 2^-66).
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

template <typename T> __device__ __forceinline__ double2 ld2(const void* p, long i, bool real) {
  if (real) return make_double2(widen<T>(reinterpret_cast<const T*>(p)[i]), 0.0);
  const cplx<T> v = reinterpret_cast<const cplx<T>*>(p)[i];
  return make_double2(widen<T>(v.x), widen<T>(v.y));
}
// The element as stored (real arrays: imaginary part zero), for loads issued ahead of their use:
// widening at the load would make the warp wait for the load right there.
template <typename T> __device__ __forceinline__ cplx<T> ldraw(const void* p, long i, bool real) {
  if (real) {
    cplx<T> v;
    v.x = reinterpret_cast<const T*>(p)[i];
    v.y = T(0);
    return v;
  }
  return reinterpret_cast<const cplx<T>*>(p)[i];
}
template <typename T> __device__ __forceinline__ double2 widen2(const cplx<T>& v) {
  return make_double2(widen<T>(v.x), widen<T>(v.y));
}
template <typename T> __device__ __forceinline__ void st2(void* p, long i, bool real, double2 v) {
  if (real) { reinterpret_cast<T*>(p)[i] = narrow<T>(v.x); return; }
  cplx<T> w; w.x = narrow<T>(v.x); w.y = narrow<T>(v.y);
  reinterpret_cast<cplx<T>*>(p)[i] = w;
}

// Column mapping: work item -> the NC columns that share one matrix (kappa2).
//   NC = 1: item = column.
//   NC = 2 (3-D): axis 1 has M1 = pair_m1 entries; group g = item / n2 picks i1 = g for
//           g <= (M1-1)/2 paired with M1 - g, and i1 = M1/2 (even M1) alone (then c1 = c2).
//   NC = 4 (3-D, equal lengths and domains on axes 1 and 2): item -> (a, b) = groups[item],
//           0 <= a <= b <= M/2, columns (+a, b), (-a, b), (+b, a), (-b, a) in (axis-1 index,
//           axis-2 index); coinciding columns (a = 0, a = b, a or b = M/2) are solved twice.
struct ColumnMap {
  long nitems;
  int pair_m1;
  int n2;
  const int2* groups;
};

template <int NC> __device__ __forceinline__ void map_columns(const ColumnMap& m, long w, long* c) {
  if constexpr (NC == 1) {
    c[0] = w;
  } else if constexpr (NC == 2) {
    const long g = w / m.n2;
    const long i2 = w - g * m.n2;
    const int npairs = (m.pair_m1 - 1) / 2;
    long i1, j1;
    if (g == 0) { i1 = j1 = 0; }
    else if (g <= npairs) { i1 = g; j1 = m.pair_m1 - g; }
    else { i1 = j1 = m.pair_m1 / 2; }
    c[0] = i1 * m.n2 + i2;
    c[1] = j1 * m.n2 + i2;
  } else {
    const int2 ab = m.groups[w];
    const int M = m.pair_m1;
    c[0] = (long)ab.x * m.n2 + ab.y;
    c[1] = (long)((M - ab.x) % M) * m.n2 + ab.y;
    c[2] = (long)ab.y * m.n2 + ab.x;
    c[3] = (long)((M - ab.y) % M) * m.n2 + ab.x;
  }
}

// table indices (layout written by space.cu)
enum { TD_B0 = 0, TD_A0 = 1, TD_G = 2, TD_COUNT = 3 };
enum { TB_B0 = 0, TB_B2, TB_B4, TB_ALO, TB_A0, TB_AUP, TB_S0, TB_S1, TB_S2, TB_G0, TB_G1, TB_F0, TB_F1, TB_COUNT };

template <typename T, int NC, typename TO = T>
__global__ void __launch_bounds__(128) k_solve_dirichlet(const void* __restrict__ in, void* __restrict__ out, int N,
                                                         long ncols, int real, double a, double b,
                                                         const __grid_constant__ Wavenumbers wn,
                                                         const __grid_constant__ ColumnMap cm,
                                                         const double* __restrict__ tab, int ts,
                                                         double* __restrict__ scratch) {
  extern __shared__ double sh[];
  double* aA0 = sh;        // a * A0_k
  double* aG = sh + ts;    // a * G_k
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    aA0[k] = a * tab[TD_A0 * ts + k];
    aG[k] = a * tab[TD_G * ts + k];
  }
  __syncthreads();
  constexpr int NV = 2 + 2 * NC;
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const int nb = N - 2;
  const double half_pi = 1.5707963267948966;
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const double k2 = kappa2_of(wn, cc[0]);
    const double aB = b - a * k2;
    const double ell = -aB * half_pi;
    const double aBpi = aB * 3.141592653589793;   // aB * B0_k for k > 0
    const int n = (nb - p + 1) / 2;
    double pr = 0.0, pge = 0.0, pg = 0.0;
    double2 pf[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) pf[q] = make_double2(0.0, 0.0);
    // element offsets of row p of each column, and the stride of two rows
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    const long rstep = 2 * ncols;
    cplx<T> fn[NC];   // right-hand side of the next row, loaded one row ahead (widened when used)
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if (n > 0) fn[q] = ldraw<T>(in, off[q], real);
    double* s = scratch + gt;
    const long sstep = (long)NV * nth;
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double2 f[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        f[q] = widen2<T>(fn[q]);
        if (i + 1 < n) fn[q] = ldraw<T>(in, off[q] + (long)(i + 1) * rstep, real);
      }
      double d = aA0[k] + (k == 0 ? aB * 4.71238898038469 : aBpi);
      double g = aG[k];
      if (i > 0) {
        const double mu = ell * pr;
        d = fma(-mu, pge, d);
        g = fma(-mu, pg, g);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          f[q].x = fma(-mu, pf[q].x, f[q].x);
          f[q].y = fma(-mu, pf[q].y, f[q].y);
        }
      }
      const double r = rcp64(d);
      s[0] = r;
      s[nth] = g;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        s[(2 + 2 * q) * nth] = f[q].x;
        s[(3 + 2 * q) * nth] = f[q].y;
        pf[q] = f[q];
      }
      s += sstep;
      pr = r; pg = g; pge = g + ell;
    }
    double2 un[NC], Ts[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { un[q] = make_double2(0.0, 0.0); Ts[q] = make_double2(0.0, 0.0); }
    double vn[NV];   // reduced row i, loaded one row ahead
    s -= sstep;      // row n-1
    if (n > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) vn[v] = s[v * nth];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] = vn[j];
      if (i > 0) {
        s -= sstep;
#pragma unroll
        for (int j = 0; j < NV; ++j) vn[j] = s[j * nth];
      }
      const double r = v[0], g = v[1];
      // row i + 1 is stored one iteration late (see k_solve_biharmonic)
      if (i + 1 < n) {
#pragma unroll
        for (int q = 0; q < NC; ++q) st2<TO>(out, off[q] + (long)(i + 1) * rstep, real, un[q]);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        Ts[q].x += un[q].x;
        Ts[q].y += un[q].y;
        double2 u;
        u.x = fma(-g, Ts[q].x, fma(-ell, un[q].x, v[2 + 2 * q])) * r;
        u.y = fma(-g, Ts[q].y, fma(-ell, un[q].y, v[3 + 2 * q])) * r;
        un[q] = u;
      }
    }
    if (n > 0) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, off[q], real, un[q]);
    }
    for (int k = nb + p; k < N; k += 2) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], real, make_double2(0.0, 0.0));
    }
  }
}

// Shen-Neumann, a lap(u) + b u = f (phi_k = T_k - q_k T_{k+2}, q_k = (k/(k+2))^2):
// M = a A + aB B, aB = b - a kappa2.  Within a parity, with i the position (k = p + 2i):
//   B: diagonal pi/2 (c_k + q_k^2), off-diagonals B_{k,k+2} = B_{k+2,k} = -pi/2 q_k;
//   A: upper triangular, diagonal -2 pi k^2 (k+1)/(k+2), and A_{kj} = G_k F_j to the right of it
//      with G_k = -4 pi (k+1)/(k+2)^2 and F_j = j^2 (a rank-one tail weighted by the trial index).
//   Row i: l_i u_{i-1} + d_i u_i + e_i u_{i+1} + a G_k sum_{j >= i+2} F_j u_j,
//   l_i = aB B_{k-2,k},  d_i = a A_kk + aB B_kk,  e_i = a G_k F_{k+2} + aB B_{k,k+2}.
// Top-down elimination keeps that shape: mu = l_i / D_{i-1},  D_i = d_i - mu E_{i-1},
// E_i = e_i - mu G'_{i-1} F_{k+2},  G'_i = a G_k - mu G'_{i-1},  f'_i = f_i - mu f'_{i-1};
// back substitution u_i = (f'_i - E_i u_{i+1} - G'_i sum_{j >= i+2} F_j u_j) / D_i.
// When aB = 0 (no zeroth-order term in this Fourier column) the constant phi_0 is in the null
// space: the even parity then sets u_0 = 0 and drops the equation of phi_0, starting the
// elimination at row 1.  Table layout (space.cu): TN_B0, TN_BUP (= B_{k,k+2}), TN_A0, TN_G.
enum { TN_B0 = 0, TN_BUP = 1, TN_A0 = 2, TN_G = 3, TN_COUNT = 4 };

template <typename T, int NC, typename TO = T>
__global__ void __launch_bounds__(128) k_solve_neumann(const void* __restrict__ in, void* __restrict__ out, int N,
                                                       long ncols, int real, double a, double b,
                                                       const __grid_constant__ Wavenumbers wn,
                                                       const __grid_constant__ ColumnMap cm,
                                                       const double* __restrict__ tab, int ts,
                                                       double* __restrict__ scratch) {
  extern __shared__ double sh[];
  double* tB0 = sh;
  double* tBU = sh + ts;
  double* aA0 = sh + 2 * ts;   // a * A_kk
  double* aG = sh + 3 * ts;    // a * G_k
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    tB0[k] = tab[TN_B0 * ts + k];
    tBU[k] = tab[TN_BUP * ts + k];
    aA0[k] = a * tab[TN_A0 * ts + k];
    aG[k] = a * tab[TN_G * ts + k];
  }
  __syncthreads();
  constexpr int NV = 3 + 2 * NC;
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const int nb = N - 2;
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const double k2 = kappa2_of(wn, cc[0]);
    const double aB = b - a * k2;
    const int n = (nb - p + 1) / 2;
    const int i0 = (p == 0 && aB == 0.0) ? 1 : 0;   // u_0 = 0 for the singular even parity
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    const long rstep = 2 * ncols;
    double pr = 0.0, pE = 0.0, pG = 0.0;
    double2 pf[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) pf[q] = make_double2(0.0, 0.0);
    double* s = scratch + gt + (long)i0 * NV * nth;
    const long sstep = (long)NV * nth;
    for (int i = i0; i < n; ++i) {
      const int k = p + 2 * i;
      double2 f[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) f[q] = ld2<T>(in, off[q] + (long)i * rstep, real);
      const double fk2 = (double)(k + 2) * (double)(k + 2);
      double d = fma(aB, tB0[k], aA0[k]);
      double e = fma(aB, tBU[k], aG[k] * fk2);
      double g = aG[k];
      if (i > i0) {
        const double mu = aB * tBU[k - 2] * pr;
        d = fma(-mu, pE, d);
        e = fma(-mu * pG, fk2, e);
        g = fma(-mu, pG, g);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          f[q].x = fma(-mu, pf[q].x, f[q].x);
          f[q].y = fma(-mu, pf[q].y, f[q].y);
        }
      }
      const double r = rcp64(d);
      s[0] = r;
      s[nth] = e;
      s[2 * nth] = g;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        s[(3 + 2 * q) * nth] = f[q].x;
        s[(4 + 2 * q) * nth] = f[q].y;
        pf[q] = f[q];
      }
      s += sstep;
      pr = r; pE = e; pG = g;
    }
    double2 un[NC], Ts[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { un[q] = make_double2(0.0, 0.0); Ts[q] = make_double2(0.0, 0.0); }
    for (int i = n - 1; i >= i0; --i) {
      const int k = p + 2 * i;
      s -= sstep;
      const double r = s[0], e = s[nth], g = s[2 * nth];
      const double fk2 = (double)(k + 2) * (double)(k + 2);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        double2 u;
        u.x = fma(-g, Ts[q].x, fma(-e, un[q].x, s[(3 + 2 * q) * nth])) * r;
        u.y = fma(-g, Ts[q].y, fma(-e, un[q].y, s[(4 + 2 * q) * nth])) * r;
        st2<TO>(out, off[q] + (long)i * rstep, real, u);
        // the tail seen by row i - 1 starts at row i + 1, the trial index k + 2
        Ts[q].x = fma(fk2, un[q].x, Ts[q].x);
        Ts[q].y = fma(fk2, un[q].y, Ts[q].y);
        un[q] = u;
      }
    }
    if (i0 == 1)
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, off[q], real, make_double2(0.0, 0.0));
    for (int k = nb + p; k < N; k += 2) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], real, make_double2(0.0, 0.0));
    }
  }
}

// Two-sided elimination of the Dirichlet systems (used with NC = 1: 1-D and 2-D spaces).
// A CTA of four warps owns 32 work items: warps (p, side) with p the parity and side 0 / 1.
// Side 0 eliminates rows 0 .. h-1 top-down as k_solve_dirichlet does (h = ceil(n / 2)); side 1
// runs rows n-1 .. h bottom-up, writing each unknown and the tail sum T_i = sum_{j>=i} u_j as
// affine functions of the unknown above:
//     u_i = a_i + b_i u_{i-1},   T_i = A_i + B_i u_{i-1},
//     D_i = d_i + ell b_{i+1} + g_i B_{i+1},   a_i = (f_i - ell a_{i+1} - g_i A_{i+1}) / D_i,
//     b_i = -ell / D_i,   A_i = A_{i+1} + (1 + B_{i+1}) a_i,   B_i = (1 + B_{i+1}) b_i,
// from a_n = b_n = A_n = B_n = 0 (row i of the system: ell u_{i-1} + d_i u_i + ell u_{i+1} +
// g_i T_{i+1} = f_i).  For a = 0 (no ell terms) this is the ordinary back substitution of the
// upper-triangular stiffness rows; with a mass term |b_i| stays below one and B_i bounded.  The
// sides meet through shared memory at the reduced top row h-1,
//     u_{h-1} = (f'_{h-1} - ell a_h - g'_{h-1} A_h) / (d'_{h-1} + ell b_h + g'_{h-1} B_h),
// after which side 0 back-substitutes rows h-2 .. 0 and side 1 forward-substitutes rows h .. n-1.
// Each serial chain is half as long as in the one-sided kernel and twice as many warps run it.
template <typename T, int NC, typename TO = T>
__global__ void __launch_bounds__(128) k_solve_dirichlet2(const void* __restrict__ in, void* __restrict__ out, int N,
                                                          long ncols, int real, double a, double b,
                                                          const __grid_constant__ Wavenumbers wn,
                                                          const __grid_constant__ ColumnMap cm,
                                                          const double* __restrict__ tab, int ts,
                                                          double* __restrict__ scratch) {
  extern __shared__ double sh[];
  double* aA0 = sh;        // a * A0_k
  double* aG = sh + ts;    // a * G_k
  constexpr int XV = 6 * NC + 2;                     // exchange values per (parity, lane)
  double* xch = sh + 2 * ts;                         // [parity][lane][XV]
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    aA0[k] = a * tab[TD_A0 * ts + k];
    aG[k] = a * tab[TD_G * ts + k];
  }
  __syncthreads();
  constexpr int NV = 2 + 2 * NC;
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = warp & 1, side = warp >> 1;
  const long nwb = (cm.nitems + 31) / 32;
  const int nb = N - 2;
  const int n = (nb - p + 1) / 2, h = (n + 1) / 2;
  const double half_pi = 1.5707963267948966;
  const long rstep = 2 * ncols;
  const long sstep = (long)NV * nth;
  double* x = xch + (p * 32 + lane) * XV;
  for (long grp = blockIdx.x; grp < nwb; grp += gridDim.x) {
    const long item = grp * 32 + lane;
    const bool valid = item < cm.nitems;
    long cc[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) cc[q] = 0;
    if (valid) map_columns<NC>(cm, item, cc);
    const double k2 = valid ? kappa2_of(wn, cc[0]) : 0.0;
    const double aB = b - a * k2;
    const double ell = -aB * half_pi;
    const double aBpi = aB * 3.141592653589793;   // aB * B0_k for k > 0
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    double* s = scratch + gt;
    // reduced top row h-1 (side 0)
    double dl = 1.0, gl = 0.0;
    double2 fl[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) fl[q] = make_double2(0.0, 0.0);
    // right-hand sides come through a ring of DM rows of loads issued ahead (kept as loaded,
    // widened when used): a row's FP64 work is shorter than the load latency
    constexpr int DM = 4;
    cplx<T> fr[DM][NC];
    if (side == 0) {
      double pr = 0.0, pge = 0.0, pg = 0.0;
      double2 pf[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) pf[q] = make_double2(0.0, 0.0);
#pragma unroll
      for (int d = 0; d < DM; ++d)
        if (valid && d < h) {
#pragma unroll
          for (int q = 0; q < NC; ++q) fr[d][q] = ldraw<T>(in, off[q] + (long)d * rstep, real);
        }
      for (int i = 0; i < h; ++i) {
        const int k = p + 2 * i;
        double2 f[NC];
        const int slot = i % DM;
#pragma unroll
        for (int dd = 0; dd < DM; ++dd)
          if (dd == slot) {
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              f[q] = valid ? widen2<T>(fr[dd][q]) : make_double2(0.0, 0.0);
              if (valid && i + DM < h) fr[dd][q] = ldraw<T>(in, off[q] + (long)(i + DM) * rstep, real);
            }
          }
        double d = aA0[k] + (k == 0 ? aB * 4.71238898038469 : aBpi);
        double g = aG[k];
        if (i > 0) {
          const double mu = ell * pr;
          d = fma(-mu, pge, d);
          g = fma(-mu, pg, g);
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            f[q].x = fma(-mu, pf[q].x, f[q].x);
            f[q].y = fma(-mu, pf[q].y, f[q].y);
          }
        }
        const double r = rcp64(d);
        s[0] = r;
        s[nth] = g;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          s[(2 + 2 * q) * nth] = f[q].x;
          s[(3 + 2 * q) * nth] = f[q].y;
          pf[q] = f[q];
        }
        s += sstep;
        pr = r; pg = g; pge = g + ell;
        dl = d; gl = g;
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) fl[q] = pf[q];
    } else {
      double bn = 0.0, Bn = 0.0;
      double2 an[NC], An[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) an[q] = An[q] = make_double2(0.0, 0.0);
      // ring slot (n - 1 - i) % DM holds row i
#pragma unroll
      for (int d = 0; d < DM; ++d)
        if (valid && n - 1 - d >= h) {
#pragma unroll
          for (int q = 0; q < NC; ++q) fr[d][q] = ldraw<T>(in, off[q] + (long)(n - 1 - d) * rstep, real);
        }
      for (int i = n - 1; i >= h; --i) {
        const int k = p + 2 * i;
        double2 f[NC];
        const int slot = (n - 1 - i) % DM;
#pragma unroll
        for (int dd = 0; dd < DM; ++dd)
          if (dd == slot) {
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              f[q] = valid ? widen2<T>(fr[dd][q]) : make_double2(0.0, 0.0);
              if (valid && i - DM >= h) fr[dd][q] = ldraw<T>(in, off[q] + (long)(i - DM) * rstep, real);
            }
          }
        const double d = aA0[k] + (k == 0 ? aB * 4.71238898038469 : aBpi);
        const double g = aG[k];
        const double R = rcp64(fma(g, Bn, fma(ell, bn, d)));
        const double bi = -ell * R, onep = 1.0 + Bn;
        s[0] = bi;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          double2 ai;
          ai.x = fma(-g, An[q].x, fma(-ell, an[q].x, f[q].x)) * R;
          ai.y = fma(-g, An[q].y, fma(-ell, an[q].y, f[q].y)) * R;
          An[q].x = fma(onep, ai.x, An[q].x);
          An[q].y = fma(onep, ai.y, An[q].y);
          an[q] = ai;
          s[(1 + 2 * q) * nth] = ai.x;
          s[(2 + 2 * q) * nth] = ai.y;
        }
        s += sstep;
        bn = bi;
        Bn = onep * bi;
      }
      // hand (a_h, b_h, A_h, B_h) to side 0
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        x[4 * q] = an[q].x;
        x[4 * q + 1] = an[q].y;
        x[4 * q + 2] = An[q].x;
        x[4 * q + 3] = An[q].y;
      }
      x[4 * NC] = bn;
      x[4 * NC + 1] = Bn;
    }
    __syncthreads();
    // side 0 forms u_{h-1} from the reduced top row and side 1's (a_h, b_h, A_h, B_h); after one
    // synchronisation side 0 back-substitutes rows h-2 .. 0 while side 1 forward-substitutes rows
    // h .. n-1, each sweep reading its rows from the scratch through a ring of loads issued ahead
    double2 un[NC], Ts[NC];
    if (side == 0 && h > 0) {
      const double bh = x[4 * NC], Bh = x[4 * NC + 1];
      const double rd = rcp64(fma(gl, Bh, fma(ell, bh, dl)));
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const double2 ah = make_double2(x[4 * q], x[4 * q + 1]), Ah = make_double2(x[4 * q + 2], x[4 * q + 3]);
        double2 u;
        u.x = fma(-gl, Ah.x, fma(-ell, ah.x, fl[q].x)) * rd;
        u.y = fma(-gl, Ah.y, fma(-ell, ah.y, fl[q].y)) * rd;
        x[4 * NC + 2 + 2 * q] = u.x;           // u_{h-1} for side 1
        x[4 * NC + 3 + 2 * q] = u.y;
        // u_h = a_h + b_h u_{h-1},  T_h = A_h + B_h u_{h-1}
        un[q] = u;
        Ts[q] = make_double2(fma(Bh, u.x, Ah.x), fma(Bh, u.y, Ah.y));
        if (valid) st2<TO>(out, off[q] + (long)(h - 1) * rstep, real, u);
      }
    }
    __syncthreads();
    if (side == 0) {
      // back substitution of rows h-2 .. 0 (Ts = T_{i+1} after adding u_{i+1}); side 0 wrote row i
      // at scratch slot i; ring slot d of pass j0 holds row h - 2 - (j0 + d)
      constexpr int D0 = 2;
      const double* base0 = scratch + gt;
      double vb[D0][NV];
#pragma unroll
      for (int d = 0; d < D0; ++d)
        if (h - 2 - d >= 0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) vb[d][v] = base0[(long)(h - 2 - d) * sstep + v * nth];
        }
      for (int j0 = 0; j0 < h - 1; j0 += D0) {
#pragma unroll
        for (int d = 0; d < D0; ++d) {
          const int i = h - 2 - (j0 + d);
          if (i >= 0) {
            double v[NV];
#pragma unroll
            for (int t = 0; t < NV; ++t) v[t] = vb[d][t];
            if (i - D0 >= 0) {
#pragma unroll
              for (int t = 0; t < NV; ++t) vb[d][t] = base0[(long)(i - D0) * sstep + t * nth];
            }
            const double r = v[0], g = v[1];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              Ts[q].x += un[q].x;
              Ts[q].y += un[q].y;
              double2 u;
              u.x = fma(-g, Ts[q].x, fma(-ell, un[q].x, v[2 + 2 * q])) * r;
              u.y = fma(-g, Ts[q].y, fma(-ell, un[q].y, v[3 + 2 * q])) * r;
              if (valid) st2<TO>(out, off[q] + (long)i * rstep, real, u);
              un[q] = u;
            }
          }
        }
      }
      if (valid)
        for (int k = nb + p; k < N; k += 2) {
#pragma unroll
          for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], real, make_double2(0.0, 0.0));
        }
    } else {
      // forward substitution of rows h .. n-1 from u_{h-1}; side 1 wrote rows n-1 .. h at scratch
      // slots 0 .. n-1-h (row i is slot n-1-i); ring slot d of pass i0 holds row i0 + d
      constexpr int D1 = 4;
      double2 up[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q)
        up[q] = h > 0 ? make_double2(x[4 * NC + 2 + 2 * q], x[4 * NC + 3 + 2 * q]) : make_double2(0.0, 0.0);
      const double* base = scratch + gt;
      double rb[D1][1 + 2 * NC];
#pragma unroll
      for (int d = 0; d < D1; ++d)
        if (h + d < n) {
#pragma unroll
          for (int v = 0; v < 1 + 2 * NC; ++v) rb[d][v] = base[(long)(n - 1 - (h + d)) * sstep + v * nth];
        }
      for (int i0 = h; i0 < n; i0 += D1) {
#pragma unroll
        for (int d = 0; d < D1; ++d) {
          const int i = i0 + d;
          if (i < n) {
            double a[1 + 2 * NC];
#pragma unroll
            for (int t = 0; t < 1 + 2 * NC; ++t) a[t] = rb[d][t];
            if (i + D1 < n) {
#pragma unroll
              for (int t = 0; t < 1 + 2 * NC; ++t) rb[d][t] = base[(long)(n - 1 - (i + D1)) * sstep + t * nth];
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              double2 u;
              u.x = fma(a[0], up[q].x, a[1 + 2 * q]);
              u.y = fma(a[0], up[q].y, a[2 + 2 * q]);
              if (valid) st2<TO>(out, off[q] + (long)i * rstep, real, u);
              up[q] = u;
            }
          }
        }
      }
    }
    __syncthreads();   // the exchange slots are reused by the next group
  }
}

template <typename T, int NC, typename TO = T>
__global__ void __launch_bounds__(128) k_solve_biharmonic(const void* __restrict__ in, void* __restrict__ out,
                                                          int N, long ncols, int real, double a, double b,
                                                          double cc0, const __grid_constant__ Wavenumbers wn,
                                                          const __grid_constant__ ColumnMap cm,
                                                          const double* __restrict__ tab, int ts,
                                                          double* __restrict__ scratch) {
  // shared tables: a*S0, a*S1, a*S2, a*G0, a*G1 and the unscaled B0, B2, B4, Alo, A0, Aup, F0, F1
  extern __shared__ double sh[];
  enum { SS0 = 0, SS1, SS2, SG0, SG1, SB0, SB2, SB4, SALO, SA0, SAUP, SF0, SF1, SCOUNT };
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    sh[SS0 * ts + k] = a * tab[TB_S0 * ts + k];
    sh[SS1 * ts + k] = a * tab[TB_S1 * ts + k];
    sh[SS2 * ts + k] = a * tab[TB_S2 * ts + k];
    sh[SG0 * ts + k] = a * tab[TB_G0 * ts + k];
    sh[SG1 * ts + k] = a * tab[TB_G1 * ts + k];
    sh[SB0 * ts + k] = tab[TB_B0 * ts + k];
    sh[SB2 * ts + k] = tab[TB_B2 * ts + k];
    sh[SB4 * ts + k] = tab[TB_B4 * ts + k];
    sh[SALO * ts + k] = tab[TB_ALO * ts + k];
    sh[SA0 * ts + k] = tab[TB_A0 * ts + k];
    sh[SAUP * ts + k] = tab[TB_AUP * ts + k];
    sh[SF0 * ts + k] = tab[TB_F0 * ts + k];
    sh[SF1 * ts + k] = tab[TB_F1 * ts + k];
  }
  __syncthreads();
  auto tb = [&](int t, int k) -> double { return sh[t * ts + k]; };
  constexpr int NV = 5 + 2 * NC;
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const int nb = N - 4;
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const double k2 = kappa2_of(wn, cc[0]);
    const double aA = b - 2.0 * a * k2;
    const double aB = fma(a * k2, k2, fma(-b, k2, cc0));
    const int n = (nb - p + 1) / 2;
    // reduced rows i-1 (suffix 1) and i-2 (suffix 2); q4 = aB * B4 of rows i-1, i-2
    double r1 = 0, U11 = 0, U21 = 0, g01 = 0, g11 = 0, q41 = 0;
    double r2 = 0, U12 = 0, U22 = 0, g02 = 0, g12 = 0, q42 = 0;
    double2 f1[NC], f2[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { f1[q] = make_double2(0, 0); f2[q] = make_double2(0, 0); }
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    const long rstep = 2 * ncols;
    cplx<T> fn[NC];   // right-hand side of the next row, loaded one row ahead (widened when used)
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if (n > 0) fn[q] = ldraw<T>(in, off[q], real);
    double* s = scratch + gt;
    const long sstep = (long)NV * nth;
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double2 f[NC];
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        f[q] = widen2<T>(fn[q]);
        if (i + 1 < n) fn[q] = ldraw<T>(in, off[q] + (long)(i + 1) * rstep, real);
      }
      const double q4 = aB * tb(SB4, k);
      double D = fma(aA, tb(SA0, k), fma(aB, tb(SB0, k), tb(SS0, k)));
      double u1 = fma(aA, tb(SAUP, k), fma(aB, tb(SB2, k), tb(SS1, k)));
      double u2 = tb(SS2, k) + q4;
      double h0 = tb(SG0, k), h1 = tb(SG1, k);
      const double F0a = tb(SF0, k + 2), F1a = tb(SF1, k + 2);
      const double F0b = tb(SF0, k + 4), F1b = tb(SF1, k + 4);
      if (i >= 1) {
        double L1 = fma(aA, tb(SALO, k), aB * tb(SB2, k - 2));
        double mu1;
        if (i >= 2) {
          const double mu = q42 * r2;
          L1 = fma(-mu, U12, L1);
          D = fma(-mu, U22, D);
          u1 = fma(-mu, fma(g02, F0a, g12 * F1a), u1);
          u2 = fma(-mu, fma(g02, F0b, g12 * F1b), u2);
          h0 = fma(-mu, g02, h0);
          h1 = fma(-mu, g12, h1);
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            f[q].x = fma(-mu, f2[q].x, f[q].x);
            f[q].y = fma(-mu, f2[q].y, f[q].y);
          }
        }
        mu1 = L1 * r1;
        D = fma(-mu1, U11, D);
        u1 = fma(-mu1, U21, u1);
        u2 = fma(-mu1, fma(g01, F0b, g11 * F1b), u2);
        h0 = fma(-mu1, g01, h0);
        h1 = fma(-mu1, g11, h1);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          f[q].x = fma(-mu1, f1[q].x, f[q].x);
          f[q].y = fma(-mu1, f1[q].y, f[q].y);
        }
      }
      const double r = rcp64(D);
      s[0] = r; s[nth] = u1; s[2 * nth] = u2; s[3 * nth] = h0; s[4 * nth] = h1;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        s[(5 + 2 * q) * nth] = f[q].x;
        s[(6 + 2 * q) * nth] = f[q].y;
        f2[q] = f1[q];
        f1[q] = f[q];
      }
      s += sstep;
      r2 = r1; U12 = U11; U22 = U21; g02 = g01; g12 = g11; q42 = q41;
      r1 = r; U11 = u1; U21 = u2; g01 = h0; g11 = h1; q41 = q4;
    }
    // back substitution: u_{i+1}, u_{i+2}, u_{i+3} and the tail sums T0, T1 per column
    double2 ua[NC], ub[NC], uc[NC], T0[NC], T1[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      ua[q] = ub[q] = uc[q] = make_double2(0, 0);
      T0[q] = T1[q] = make_double2(0, 0);
    }
    double vn[NV];   // reduced row i, loaded one row ahead
    s -= sstep;      // row n-1
    if (n > 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) vn[v] = s[v * nth];
    }
    for (int i = n - 1; i >= 0; --i) {
      const int k = p + 2 * i;
      const double F0 = tb(SF0, k + 6), F1 = tb(SF1, k + 6);   // zero past the basis
      double v[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] = vn[j];
      if (i > 0) {
        s -= sstep;
#pragma unroll
        for (int j = 0; j < NV; ++j) vn[j] = s[j * nth];
      }
      const double r = v[0], u1 = v[1], u2 = v[2], h0 = v[3], h1 = v[4];
      // row i + 1 is stored one iteration late, so that its conversion to the output type
      // does not hold up this row's dependent FP64 chain
      if (i + 1 < n) {
#pragma unroll
        for (int q = 0; q < NC; ++q) st2<TO>(out, off[q] + (long)(i + 1) * rstep, real, ua[q]);
      }
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        T0[q].x = fma(F0, uc[q].x, T0[q].x); T0[q].y = fma(F0, uc[q].y, T0[q].y);
        T1[q].x = fma(F1, uc[q].x, T1[q].x); T1[q].y = fma(F1, uc[q].y, T1[q].y);
        double2 u;
        u.x = fma(-h1, T1[q].x, fma(-h0, T0[q].x, fma(-u2, ub[q].x, fma(-u1, ua[q].x, v[5 + 2 * q])))) * r;
        u.y = fma(-h1, T1[q].y, fma(-h0, T0[q].y, fma(-u2, ub[q].y, fma(-u1, ua[q].y, v[6 + 2 * q])))) * r;
        uc[q] = ub[q]; ub[q] = ua[q]; ua[q] = u;
      }
    }
    if (n > 0) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, off[q], real, ua[q]);
    }
    for (int k = nb + p; k < N; k += 2) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], real, make_double2(0.0, 0.0));
    }
  }
}

// ---- factored eliminations (3-D spaces) ---------------------------------------------------
// The factorisation of one (column, parity) system - reciprocal pivots, multipliers, the reduced
// super-diagonals and tail coefficients - depends only on the operator (a, b, c) and on kappa2,
// not on the right-hand side, just as the paper's Helmholtz and Biharmonic solver objects are
// built once from their matrices and then applied to many right-hand sides (Sec. 4).
// k_factor_* runs the top-down factorisation of the kernels above, one thread per pair of columns
// +-l1 (which share kappa2) and parity, and stores it in a table laid out [row][value][entry]
// (entry = 32 * warp + lane of that pair decomposition, so a warp reads 256 contiguous bytes per
// value); k_solve_*_f replays only the right-hand-side recurrences from the table, one thread per
// column and parity (NC = 1), both columns of a pair reading the pair's entry.  With no
// factorisation left to share between the columns of a thread, single columns give four times the
// warps of the four-column groups, to hide the FP64 latency and to share the SMs with a concurrent
// solve's kernels in small, even units (and a quarter of the registers).  FP64 operations per row
// and complex column: Dirichlet 10 (against 16 with the factorisation shared by a pair of
// columns), biharmonic 18 (against ~30 with it shared by four).  The multipliers and reciprocal
// pivots are the same FP64 values the kernels above compute; the back substitution adds the term
// of the unknown just solved last, so that its dependent chain is one FMA and one multiply per row.
enum { FD_MU = 0, FD_R, FD_G, FD_GE, FD_COUNT };                        // Dirichlet table values
enum { FB_MU = 0, FB_MU1, FB_R, FB_U1, FB_U2, FB_H0, FB_H1, FB_COUNT };  // biharmonic table values

template <int NC>
__global__ void __launch_bounds__(128) k_factor_dirichlet(int N, double a, double b,
                                                          const __grid_constant__ Wavenumbers wn,
                                                          const __grid_constant__ ColumnMap cm,
                                                          const double* __restrict__ tab, int ts,
                                                          double* __restrict__ fact) {
  extern __shared__ double sh[];
  double* aA0 = sh;
  double* aG = sh + ts;
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    aA0[k] = a * tab[TD_A0 * ts + k];
    aG[k] = a * tab[TD_G * ts + k];
  }
  __syncthreads();
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const long TT = 2 * nwb * 32;
  const int nb = N - 2;
  const double half_pi = 1.5707963267948966;
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const double k2 = kappa2_of(wn, cc[0]);
    const double aB = b - a * k2;
    const double ell = -aB * half_pi;
    const double aBpi = aB * 3.141592653589793;
    const int n = (nb - p + 1) / 2;
    double* fr = fact + w * 32 + lane;
    double pr = 0.0, pge = 0.0, pg = 0.0;
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double d = aA0[k] + (k == 0 ? aB * 4.71238898038469 : aBpi);
      double g = aG[k];
      double mu = 0.0;
      if (i > 0) {
        mu = ell * pr;
        d = fma(-mu, pge, d);
        g = fma(-mu, pg, g);
      }
      const double r = rcp64(d);
      fr[FD_MU * TT] = mu;
      fr[FD_R * TT] = r;
      fr[FD_G * TT] = g;
      fr[FD_GE * TT] = g + ell;
      fr += FD_COUNT * TT;
      pr = r; pg = g; pge = g + ell;
    }
  }
}

// Factorisation table of the factored solves: the columns (l1, l2) and (-l1, l2) have the same
// kappa2, so with kPairTable one table entry per pair +-l1 (written by k_factor_*<2>, the pair
// decomposition of the kernels above) serves both columns, whose threads read it at about the same
// time (the partner's read then hits L2); without it every column thread has its own entry
// (k_factor_*<1>).  table_items: the entries of a parity; table_thread: the entry of a column.
constexpr bool kPairTable = true;

__device__ __forceinline__ long table_items(const ColumnMap& cm) {
  if (!kPairTable) return cm.nitems;
  const int M1 = cm.pair_m1;
  return (1 + (M1 - 1) / 2 + (M1 % 2 == 0 ? 1 : 0)) * (long)cm.n2;
}
__device__ __forceinline__ long table_thread(const ColumnMap& cm, long w, int lane, long item, int p) {
  if (!kPairTable) return w * 32 + lane;
  const long i1 = item / cm.n2, i2 = item - i1 * cm.n2;
  const long g = 2 * i1 <= cm.pair_m1 ? i1 : cm.pair_m1 - i1;
  const long it = g * cm.n2 + i2;
  return (2 * (it >> 5) + p) * 32 + (it & 31);
}

// The factored sweeps do little FP64 work per row (the Dirichlet forward sweep 2 FMAs per
// column). Each sweep keeps a ring of D rows of operands in registers (the loads of row i + D are
// issued as row i is consumed; a slot is indexed by a compile-time position of the unrolled ring)
// and keeps them as loaded (widened when used). Every value is stored one row after it is
// computed: in-order issue would otherwise hold the store, and the warp behind it, until the FMA
// that produced the value completes. Depths: one row. Deeper rings (Dirichlet 4 rows forward and 2
// backward, biharmonic 2 forward) were measured on the 256^3 step: the Dirichlet solve alone 8 %
// faster, the two-stream step no faster and up to 8 % slower, with 30-40 more registers per thread.
constexpr int kDirFwdRows = 1, kDirBwdRows = 1, kBihFwdRows = 1, kBihBwdRows = 1;

template <typename T, int NC, typename TO, int DF, int DB>
__global__ void __launch_bounds__(128) k_solve_dirichlet_f(const void* __restrict__ in, void* __restrict__ out, int N,
                                                           long ncols, const __grid_constant__ ColumnMap cm,
                                                           const double* __restrict__ fact,
                                                           double* __restrict__ scratch) {
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const long TT = 2 * ((table_items(cm) + 31) / 32) * 32;
  const long fs = FD_COUNT * TT;   // table stride of one row
  const int nb = N - 2;
  const cplx<T>* src = reinterpret_cast<const cplx<T>*>(in);
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const int n = (nb - p + 1) / 2;
    const double* fr = fact + table_thread(cm, w, lane, item, p);
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    const long rstep = 2 * ncols;
    double* const s0 = scratch + gt;
    const long sstep = (long)(2 * NC) * nth;
    // forward: f'_i = f_i - mu_i f'_{i-1} into the scratch
    cplx<T> fb[DF][NC];
    double mb[DF];
#pragma unroll
    for (int d = 0; d < DF; ++d)
      if (d < n) {
#pragma unroll
        for (int q = 0; q < NC; ++q) fb[d][q] = src[off[q] + (long)d * rstep];
        mb[d] = fr[(long)d * fs + FD_MU * TT];
      }
    double2 pf[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) pf[q] = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < n; i0 += DF) {
#pragma unroll
      for (int d = 0; d < DF; ++d) {
        const int i = i0 + d;
        if (i < n) {
          const double mu = mb[d];
          double2 f[NC];
#pragma unroll
          for (int q = 0; q < NC; ++q) f[q] = widen2<T>(fb[d][q]);
          if (i + DF < n) {
#pragma unroll
            for (int q = 0; q < NC; ++q) fb[d][q] = src[off[q] + (long)(i + DF) * rstep];
            mb[d] = fr[(long)(i + DF) * fs + FD_MU * TT];
          }
          if (i > 0) {   // row i - 1
            double* s = s0 + (long)(i - 1) * sstep;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              s[(2 * q) * nth] = pf[q].x;
              s[(2 * q + 1) * nth] = pf[q].y;
            }
          }
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            f[q].x = fma(-mu, pf[q].x, f[q].x);
            f[q].y = fma(-mu, pf[q].y, f[q].y);
            pf[q] = f[q];
          }
        }
      }
    }
    if (n > 0) {
      double* s = s0 + (long)(n - 1) * sstep;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        s[(2 * q) * nth] = pf[q].x;
        s[(2 * q + 1) * nth] = pf[q].y;
      }
    }
    // backward: u_i = (f'_i - g_i sum_{j>=i+2} u_j - (g_i + ell) u_{i+1}) r_i, rows n-1 .. 0;
    // ring slot d of pass j0 holds row n - 1 - (j0 + d)
    double vb[DB][2 * NC], rb[DB], gb[DB], geb[DB];
    auto load_b = [&](int d, int i) {
      const double* s = s0 + (long)i * sstep;
#pragma unroll
      for (int v = 0; v < 2 * NC; ++v) vb[d][v] = s[v * nth];
      const double* fl = fr + (long)i * fs;
      rb[d] = fl[FD_R * TT];
      gb[d] = fl[FD_G * TT];
      geb[d] = fl[FD_GE * TT];
    };
#pragma unroll
    for (int d = 0; d < DB; ++d)
      if (d < n) load_b(d, n - 1 - d);
    double2 un[NC], Tp[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) { un[q] = make_double2(0.0, 0.0); Tp[q] = make_double2(0.0, 0.0); }
    for (int j0 = 0; j0 < n; j0 += DB) {
#pragma unroll
      for (int d = 0; d < DB; ++d) {
        const int j = j0 + d, i = n - 1 - j;
        if (j < n) {
          double v[2 * NC];
#pragma unroll
          for (int t = 0; t < 2 * NC; ++t) v[t] = vb[d][t];
          const double r = rb[d], g = gb[d], ge = geb[d];
          if (j + DB < n) load_b(d, i - DB);
          // row i + 1 is stored one iteration late
          if (i + 1 < n) {
#pragma unroll
            for (int q = 0; q < NC; ++q) st2<TO>(out, off[q] + (long)(i + 1) * rstep, false, un[q]);
          }
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            double2 u;
            u.x = fma(-ge, un[q].x, fma(-g, Tp[q].x, v[2 * q])) * r;
            u.y = fma(-ge, un[q].y, fma(-g, Tp[q].y, v[2 * q + 1])) * r;
            Tp[q].x += un[q].x;
            Tp[q].y += un[q].y;
            un[q] = u;
          }
        }
      }
    }
    if (n > 0) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, off[q], false, un[q]);
    }
    for (int k = nb + p; k < N; k += 2) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], false, make_double2(0.0, 0.0));
    }
  }
}

template <int NC>
__global__ void __launch_bounds__(128) k_factor_biharmonic(int N, double a, double b, double cc0,
                                                           const __grid_constant__ Wavenumbers wn,
                                                           const __grid_constant__ ColumnMap cm,
                                                           const double* __restrict__ tab, int ts,
                                                           double* __restrict__ fact) {
  extern __shared__ double sh[];
  enum { SS0 = 0, SS1, SS2, SG0, SG1, SB0, SB2, SB4, SALO, SA0, SAUP, SF0, SF1, SCOUNT };
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    sh[SS0 * ts + k] = a * tab[TB_S0 * ts + k];
    sh[SS1 * ts + k] = a * tab[TB_S1 * ts + k];
    sh[SS2 * ts + k] = a * tab[TB_S2 * ts + k];
    sh[SG0 * ts + k] = a * tab[TB_G0 * ts + k];
    sh[SG1 * ts + k] = a * tab[TB_G1 * ts + k];
    sh[SB0 * ts + k] = tab[TB_B0 * ts + k];
    sh[SB2 * ts + k] = tab[TB_B2 * ts + k];
    sh[SB4 * ts + k] = tab[TB_B4 * ts + k];
    sh[SALO * ts + k] = tab[TB_ALO * ts + k];
    sh[SA0 * ts + k] = tab[TB_A0 * ts + k];
    sh[SAUP * ts + k] = tab[TB_AUP * ts + k];
    sh[SF0 * ts + k] = tab[TB_F0 * ts + k];
    sh[SF1 * ts + k] = tab[TB_F1 * ts + k];
  }
  __syncthreads();
  auto tb = [&](int t, int k) -> double { return sh[t * ts + k]; };
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const long TT = 2 * nwb * 32;
  const int nb = N - 4;
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const double k2 = kappa2_of(wn, cc[0]);
    const double aA = b - 2.0 * a * k2;
    const double aB = fma(a * k2, k2, fma(-b, k2, cc0));
    const int n = (nb - p + 1) / 2;
    double r1 = 0, U11 = 0, U21 = 0, g01 = 0, g11 = 0, q41 = 0;
    double r2 = 0, U12 = 0, U22 = 0, g02 = 0, g12 = 0, q42 = 0;
    double* fr = fact + w * 32 + lane;
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      const double q4 = aB * tb(SB4, k);
      double D = fma(aA, tb(SA0, k), fma(aB, tb(SB0, k), tb(SS0, k)));
      double u1 = fma(aA, tb(SAUP, k), fma(aB, tb(SB2, k), tb(SS1, k)));
      double u2 = tb(SS2, k) + q4;
      double h0 = tb(SG0, k), h1 = tb(SG1, k);
      const double F0a = tb(SF0, k + 2), F1a = tb(SF1, k + 2);
      const double F0b = tb(SF0, k + 4), F1b = tb(SF1, k + 4);
      double mu = 0.0, mu1 = 0.0;
      if (i >= 1) {
        double L1 = fma(aA, tb(SALO, k), aB * tb(SB2, k - 2));
        if (i >= 2) {
          mu = q42 * r2;
          L1 = fma(-mu, U12, L1);
          D = fma(-mu, U22, D);
          u1 = fma(-mu, fma(g02, F0a, g12 * F1a), u1);
          u2 = fma(-mu, fma(g02, F0b, g12 * F1b), u2);
          h0 = fma(-mu, g02, h0);
          h1 = fma(-mu, g12, h1);
        }
        mu1 = L1 * r1;
        D = fma(-mu1, U11, D);
        u1 = fma(-mu1, U21, u1);
        u2 = fma(-mu1, fma(g01, F0b, g11 * F1b), u2);
        h0 = fma(-mu1, g01, h0);
        h1 = fma(-mu1, g11, h1);
      }
      const double r = rcp64(D);
      fr[FB_MU * TT] = mu;
      fr[FB_MU1 * TT] = mu1;
      fr[FB_R * TT] = r;
      fr[FB_U1 * TT] = u1;
      fr[FB_U2 * TT] = u2;
      fr[FB_H0 * TT] = h0;
      fr[FB_H1 * TT] = h1;
      fr += FB_COUNT * TT;
      r2 = r1; U12 = U11; U22 = U21; g02 = g01; g12 = g11; q42 = q41;
      r1 = r; U11 = u1; U21 = u2; g01 = h0; g11 = h1; q41 = q4;
    }
  }
}

template <typename T, int NC, typename TO, int DF, int DB>
__global__ void __launch_bounds__(128) k_solve_biharmonic_f(const void* __restrict__ in, void* __restrict__ out,
                                                            int N, long ncols, const __grid_constant__ ColumnMap cm,
                                                            const double* __restrict__ tab, int ts,
                                                            const double* __restrict__ fact,
                                                            double* __restrict__ scratch) {
  // shared: the rank-2 tail weights F0, F1 (zero past the basis)
  extern __shared__ double sh[];
  double* sF0 = sh;
  double* sF1 = sh + ts;
  for (int k = threadIdx.x; k < ts; k += blockDim.x) {
    sF0[k] = tab[TB_F0 * ts + k];
    sF1[k] = tab[TB_F1 * ts + k];
  }
  __syncthreads();
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long nwb = (cm.nitems + 31) / 32;
  const long TT = 2 * ((table_items(cm) + 31) / 32) * 32;
  const long fs = FB_COUNT * TT;
  const int nb = N - 4;
  const cplx<T>* src = reinterpret_cast<const cplx<T>*>(in);
  for (long w = gt / 32; w < 2 * nwb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long item = (w >> 1) * 32 + lane;
    if (item >= cm.nitems) continue;
    long cc[NC];
    map_columns<NC>(cm, item, cc);
    const int n = (nb - p + 1) / 2;
    const double* fr = fact + table_thread(cm, w, lane, item, p);
    long off[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) off[q] = (long)p * ncols + cc[q];
    const long rstep = 2 * ncols;
    double* const s0 = scratch + gt;
    const long sstep = (long)(2 * NC) * nth;
    // forward: f'_i = f_i - mu_i f'_{i-2} - mu1_i f'_{i-1} (the multipliers are zero where the
    // rows above do not exist)
    cplx<T> fb[DF][NC];
    double mb[DF], m1b[DF];
#pragma unroll
    for (int d = 0; d < DF; ++d)
      if (d < n) {
#pragma unroll
        for (int q = 0; q < NC; ++q) fb[d][q] = src[off[q] + (long)d * rstep];
        mb[d] = fr[(long)d * fs + FB_MU * TT];
        m1b[d] = fr[(long)d * fs + FB_MU1 * TT];
      }
    double2 f1[NC], f2[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) f1[q] = f2[q] = make_double2(0.0, 0.0);
    for (int i0 = 0; i0 < n; i0 += DF) {
#pragma unroll
      for (int d = 0; d < DF; ++d) {
        const int i = i0 + d;
        if (i < n) {
          const double mu = mb[d], mu1 = m1b[d];
          double2 f[NC];
#pragma unroll
          for (int q = 0; q < NC; ++q) f[q] = widen2<T>(fb[d][q]);
          if (i + DF < n) {
#pragma unroll
            for (int q = 0; q < NC; ++q) fb[d][q] = src[off[q] + (long)(i + DF) * rstep];
            mb[d] = fr[(long)(i + DF) * fs + FB_MU * TT];
            m1b[d] = fr[(long)(i + DF) * fs + FB_MU1 * TT];
          }
          if (i > 0) {   // row i - 1
            double* s = s0 + (long)(i - 1) * sstep;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              s[(2 * q) * nth] = f1[q].x;
              s[(2 * q + 1) * nth] = f1[q].y;
            }
          }
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            f[q].x = fma(-mu1, f1[q].x, fma(-mu, f2[q].x, f[q].x));
            f[q].y = fma(-mu1, f1[q].y, fma(-mu, f2[q].y, f[q].y));
            f2[q] = f1[q];
            f1[q] = f[q];
          }
        }
      }
    }
    if (n > 0) {
      double* s = s0 + (long)(n - 1) * sstep;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        s[(2 * q) * nth] = f1[q].x;
        s[(2 * q + 1) * nth] = f1[q].y;
      }
    }
    // backward: u_{i+1}, u_{i+2}, u_{i+3} and the tail sums T0, T1 per column; ring slot d of
    // pass j0 holds row n - 1 - (j0 + d): its right-hand side, r, u1, u2, h0, h1 and the tail
    // weights F0, F1 at k + 6 (k = p + 2i)
    double vb[DB][2 * NC], cb[DB][7];
    auto load_b = [&](int d, int i) {
      const double* s = s0 + (long)i * sstep;
#pragma unroll
      for (int v = 0; v < 2 * NC; ++v) vb[d][v] = s[v * nth];
      const double* fl = fr + (long)i * fs;
#pragma unroll
      for (int t = 0; t < 5; ++t) cb[d][t] = fl[(FB_R + t) * TT];
      cb[d][5] = sF0[p + 2 * i + 6];
      cb[d][6] = sF1[p + 2 * i + 6];
    };
#pragma unroll
    for (int d = 0; d < DB; ++d)
      if (d < n) load_b(d, n - 1 - d);
    double2 ua[NC], ub[NC], uc[NC], T0[NC], T1[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      ua[q] = ub[q] = uc[q] = make_double2(0, 0);
      T0[q] = T1[q] = make_double2(0, 0);
    }
    for (int j0 = 0; j0 < n; j0 += DB) {
#pragma unroll
      for (int d = 0; d < DB; ++d) {
        const int j = j0 + d, i = n - 1 - j;
        if (j < n) {
          double v[2 * NC];
#pragma unroll
          for (int t = 0; t < 2 * NC; ++t) v[t] = vb[d][t];
          const double r = cb[d][0], u1 = cb[d][1], u2 = cb[d][2], h0 = cb[d][3], h1 = cb[d][4];
          const double F0 = cb[d][5], F1 = cb[d][6];
          if (j + DB < n) load_b(d, i - DB);
          if (i + 1 < n) {
#pragma unroll
            for (int q = 0; q < NC; ++q) st2<TO>(out, off[q] + (long)(i + 1) * rstep, false, ua[q]);
          }
#pragma unroll
          for (int q = 0; q < NC; ++q) {
            T0[q].x = fma(F0, uc[q].x, T0[q].x); T0[q].y = fma(F0, uc[q].y, T0[q].y);
            T1[q].x = fma(F1, uc[q].x, T1[q].x); T1[q].y = fma(F1, uc[q].y, T1[q].y);
            double2 u;
            u.x = fma(-u1, ua[q].x, fma(-u2, ub[q].x, fma(-h0, T0[q].x, fma(-h1, T1[q].x, v[2 * q])))) * r;
            u.y = fma(-u1, ua[q].y, fma(-u2, ub[q].y, fma(-h0, T0[q].y, fma(-h1, T1[q].y, v[2 * q + 1])))) * r;
            uc[q] = ub[q]; ub[q] = ua[q]; ua[q] = u;
          }
        }
      }
    }
    if (n > 0) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, off[q], false, ua[q]);
    }
    for (int k = nb + p; k < N; k += 2) {
#pragma unroll
      for (int q = 0; q < NC; ++q) st2<TO>(out, (long)k * ncols + cc[q], false, make_double2(0.0, 0.0));
    }
  }
}

// Values per row per thread in the scratch for NC columns per thread.
int solve_scratch_values(int basis, int nc) {
  return basis == kDirichlet ? 2 + 2 * nc : basis == kNeumann ? 3 + 2 * nc : 5 + 2 * nc;
}

// Dynamic shared memory that lets at most max_per_sm CTAs of a kernel share an SM.  The 3-D
// biharmonic elimination runs one warp per SM sub-partition on 132 SMs, each warp's chain keeping
// its sub-partition's FP64 pipe busy.  A launch that meets SMs partly filled by other kernels (the
// elimination or transforms of a concurrent solve on another stream) would otherwise put two of
// its CTAs on some SMs, whose sub-partitions would then serve two chains each and finish last.
static size_t spread_smem(size_t need, int max_per_sm) {
  int dev = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || per_sm <= 0)
    return need;
  // every CTA also holds 1 KB of shared memory reserved by the system
  const size_t cap = (size_t)per_sm / (size_t)(max_per_sm + 1) + 1;
  return std::max(need, cap);
}

// CTAs of 128 threads for one elimination launch: one thread per work item and parity, at most
// the scratch_threads the space's scratch holds rows for (the kernels loop over the rest).
static unsigned solve_grid(const ColumnMap& cm, long scratch_threads) {
  const long warps_needed = 2 * ((cm.nitems + 31) / 32);
  long threads = std::min(scratch_threads, warps_needed * 32);
  threads = std::max(128L, ((threads + 127) / 128) * 128);
  threads = std::min(threads, std::max(128L, (scratch_threads / 128) * 128));
  return (unsigned)(threads / 128);
}

template <typename T, int NC, typename TO>
static cudaError_t solve_nc(int basis, bool real, double a, double b, double c, const void* in, void* out, int N,
                            long ncols, const Wavenumbers& wn, const ColumnMap& cm, const double* tab, double* scratch,
                            long scratch_threads, cudaStream_t s) {
  const unsigned grid = solve_grid(cm, scratch_threads);
  const int ts = N + 8;
  cudaError_t e;
  if (basis == kNeumann) {
    if constexpr (NC <= 2) {
      const size_t smem = sizeof(double) * 4 * ts;
      if (smem > 48 * 1024 &&
          (e = cudaFuncSetAttribute(k_solve_neumann<T, NC, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
              cudaSuccess)
        return e;
      k_solve_neumann<T, NC, TO><<<grid, 128, smem, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, wn, cm, tab, ts, scratch);
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (basis == kDirichlet && NC == 1) {
    // two-sided kernel for the one-column-per-thread spaces (1-D and 2-D, few columns, long
    // serial chains); the 3-D box keeps the one-sided kernel, whose pairs already fill the GPU.
    // Four warps per 32 work items, each thread at most ceil(n / 2) rows of
    // scratch; the grid is sized so that the scratch allocated for the one-sided kernel (N/2 + 1
    // rows per thread of scratch_threads) holds every thread's rows
    if constexpr (NC != 1) {
      return cudaErrorInvalidValue;
    } else {
      const long nwb = (cm.nitems + 31) / 32;
      const long rows_full = N / 2 + 1, n0 = (N - 2 + 1) / 2, rows_split = (n0 + 1) / 2 + 1;
      long cap = scratch_threads * rows_full / rows_split;
      cap = std::max(128L, (cap / 128) * 128);
      const long thr = std::min(cap, nwb * 128);
      const unsigned grid2 = (unsigned)std::max(1L, thr / 128);
      const size_t smem = sizeof(double) * (2 * ts + 2 * 32 * (6 * NC + 2));
      if (smem > 48 * 1024 &&
          (e = cudaFuncSetAttribute(k_solve_dirichlet2<T, NC, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess)
        return e;
      k_solve_dirichlet2<T, NC, TO><<<grid2, 128, smem, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, wn, cm, tab, ts,
                                                             scratch);
    }
  } else if (basis == kDirichlet) {
    const size_t smem = sizeof(double) * 2 * ts;
    if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k_solve_dirichlet<T, NC, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    k_solve_dirichlet<T, NC, TO><<<grid, 128, smem, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, wn, cm, tab, ts, scratch);
  } else {
    const size_t smem = NC == 4 ? spread_smem(sizeof(double) * 13 * ts, 1) : sizeof(double) * 13 * ts;
    if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k_solve_biharmonic<T, NC, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    k_solve_biharmonic<T, NC, TO><<<grid, 128, smem, s>>>(in, out, N, ncols, real ? 1 : 0, a, b, c, wn, cm, tab, ts, scratch);
  }
  return cudaGetLastError();
}

// Work decomposition of a call: NC = 4 with a group table (3-D, square Fourier box), NC = 2 on
// other 3-D spaces (pairs +l1 / -l1 along axis 1), NC = 1 on 1-D and 2-D spaces.
static ColumnMap column_map(long ncols, const Wavenumbers& wn, const int2* groups, long ngroups, int* nc) {
  ColumnMap cm;
  cm.pair_m1 = 0;
  cm.n2 = wn.n2;
  cm.nitems = ncols;
  cm.groups = groups;
  *nc = 1;
  if (wn.n1 > 1 && groups) {
    cm.pair_m1 = wn.n1;
    cm.nitems = ngroups;
    *nc = 4;
  } else if (wn.n1 > 1) {
    cm.pair_m1 = wn.n1;
    cm.nitems = (1 + (wn.n1 - 1) / 2 + (wn.n1 % 2 == 0 ? 1 : 0)) * (long)wn.n2;
    *nc = 2;
  }
  return cm;
}

// groups: device table of (a, b) for the four-column grouping, or nullptr; TO: type of the output
// spectral data (T, or float for FP64 input whose solution is rounded once to FP32)
template <typename T, typename TO>
cudaError_t launch_solve_to(int basis, bool real, double a, double b, double c, const void* in, void* out, int N,
                            long ncols, const Wavenumbers& wn, const double* tab, double* scratch, long scratch_threads,
                            const int2* groups, long ngroups, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  int nc = 1;
  const ColumnMap cm = column_map(ncols, wn, groups, ngroups, &nc);
  if (nc == 4)
    return solve_nc<T, 4, TO>(basis, real, a, b, c, in, out, N, ncols, wn, cm, tab, scratch, scratch_threads, s);
  if (nc == 2)
    return solve_nc<T, 2, TO>(basis, real, a, b, c, in, out, N, ncols, wn, cm, tab, scratch, scratch_threads, s);
  return solve_nc<T, 1, TO>(basis, real, a, b, c, in, out, N, ncols, wn, cm, tab, scratch, scratch_threads, s);
}

int solve_factor_values(int basis) { return basis == kDirichlet ? FD_COUNT : basis == kBiharmonic ? FB_COUNT : 0; }

// Work decomposition of the factored solves of 3-D spaces: one thread per column and parity.
static ColumnMap factored_map(long ncols, const Wavenumbers& wn, bool* ok) {
  ColumnMap cm;
  cm.pair_m1 = wn.n1;   // read by table_thread only
  cm.n2 = wn.n2;
  cm.nitems = ncols;
  cm.groups = nullptr;
  *ok = wn.n1 > 1;   // 1-D and 2-D spaces have no factored form
  return cm;
}

long solve_factor_threads(long ncols, const Wavenumbers& wn) {
  bool ok = false;
  const ColumnMap cm = factored_map(ncols, wn, &ok);
  if (!ok) return 0;
  if (kPairTable) {
    int nc = 0;
    return 2 * ((column_map(ncols, wn, nullptr, 0, &nc).nitems + 31) / 32) * 32;
  }
  return 2 * ((cm.nitems + 31) / 32) * 32;
}

long solve_factored_scratch_threads(long ncols, const Wavenumbers& wn) {
  bool ok = false;
  const ColumnMap cm = factored_map(ncols, wn, &ok);
  return ok ? 2 * ((cm.nitems + 31) / 32) * 32 : 0;
}

template <int NC>
static cudaError_t factor_nc(int basis, double a, double b, double c, int N, const Wavenumbers& wn,
                             const ColumnMap& cm, const double* tab, double* fact, cudaStream_t s) {
  const long threads = ((2 * ((cm.nitems + 31) / 32) * 32 + 127) / 128) * 128;
  const unsigned grid = (unsigned)std::max(1L, threads / 128);
  const int ts = N + 8;
  cudaError_t e;
  if (basis == kDirichlet) {
    const size_t smem = sizeof(double) * 2 * ts;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_factor_dirichlet<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
    k_factor_dirichlet<NC><<<grid, 128, smem, s>>>(N, a, b, wn, cm, tab, ts, fact);
  } else {
    const size_t smem = sizeof(double) * 13 * ts;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_factor_biharmonic<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
      return e;
    k_factor_biharmonic<NC><<<grid, 128, smem, s>>>(N, a, b, c, wn, cm, tab, ts, fact);
  }
  return cudaGetLastError();
}

cudaError_t launch_factor(int basis, double a, double b, double c, int N, long ncols, const Wavenumbers& wn,
                          const double* tab, double* fact, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  bool ok = false;
  const ColumnMap cm = factored_map(ncols, wn, &ok);
  if (!ok || solve_factor_values(basis) == 0) return cudaErrorInvalidValue;
  if (kPairTable) {
    int nc = 0;
    const ColumnMap cm2 = column_map(ncols, wn, nullptr, 0, &nc);
    return factor_nc<2>(basis, a, b, c, N, wn, cm2, tab, fact, s);
  }
  return factor_nc<1>(basis, a, b, c, N, wn, cm, tab, fact, s);
}

template <typename T, int NC, typename TO>
static cudaError_t solve_factored_nc(int basis, const void* in, void* out, int N, long ncols,
                                     const ColumnMap& cm, const double* tab, const double* fact, double* scratch,
                                     long scratch_threads, cudaStream_t s) {
  const unsigned grid = solve_grid(cm, scratch_threads);
  const int ts = N + 8;
  if (basis == kDirichlet) {
    k_solve_dirichlet_f<T, NC, TO, kDirFwdRows, kDirBwdRows><<<grid, 128, 0, s>>>(in, out, N, ncols, cm, fact, scratch);
  } else {
    const size_t smem = sizeof(double) * 2 * ts;
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_solve_biharmonic_f<T, NC, TO, kBihFwdRows, kBihBwdRows>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    k_solve_biharmonic_f<T, NC, TO, kBihFwdRows, kBihBwdRows><<<grid, 128, smem, s>>>(in, out, N, ncols, cm, tab, ts,
                                                                                      fact, scratch);
  }
  return cudaGetLastError();
}

template <typename T, typename TO>
cudaError_t launch_solve_factored_to(int basis, bool real, const void* in, void* out, int N, long ncols,
                                     const Wavenumbers& wn, const double* tab, const double* fact, double* scratch,
                                     long scratch_threads, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  bool ok = false;
  const ColumnMap cm = factored_map(ncols, wn, &ok);
  // 3-D spaces (complex spectral arrays)
  if (!ok || real || solve_factor_values(basis) == 0) return cudaErrorInvalidValue;
  return solve_factored_nc<T, 1, TO>(basis, in, out, N, ncols, cm, tab, fact, scratch, scratch_threads, s);
}

template cudaError_t launch_solve_factored_to<float, float>(int, bool, const void*, void*, int, long,
                                                            const Wavenumbers&, const double*, const double*,
                                                            double*, long, cudaStream_t);
template cudaError_t launch_solve_factored_to<double, double>(int, bool, const void*, void*, int, long,
                                                              const Wavenumbers&, const double*, const double*,
                                                              double*, long, cudaStream_t);
template cudaError_t launch_solve_factored_to<double, float>(int, bool, const void*, void*, int, long,
                                                             const Wavenumbers&, const double*, const double*,
                                                             double*, long, cudaStream_t);

template <typename T>
cudaError_t launch_solve(int basis, bool real, double a, double b, double c, const void* in, void* out, int N,
                         long ncols, const Wavenumbers& wn, const double* tab, double* scratch, long scratch_threads,
                         const int2* groups, long ngroups, cudaStream_t s) {
  return launch_solve_to<T, T>(basis, real, a, b, c, in, out, N, ncols, wn, tab, scratch, scratch_threads, groups,
                               ngroups, s);
}

cudaError_t launch_solve_f64_to_f32(int basis, double a, double b, double c, const void* in, void* out, int N, long ncols,
                                    const Wavenumbers& wn, const double* tab, double* scratch, long scratch_threads,
                                    const int2* groups, long ngroups, cudaStream_t s) {
  return launch_solve_to<double, float>(basis, false, a, b, c, in, out, N, ncols, wn, tab, scratch, scratch_threads,
                                        groups, ngroups, s);
}

template cudaError_t launch_solve<float>(int, bool, double, double, double, const void*, void*, int, long,
                                         const Wavenumbers&, const double*, double*, long, const int2*, long,
                                         cudaStream_t);
template cudaError_t launch_solve<double>(int, bool, double, double, double, const void*, void*, int, long,
                                          const Wavenumbers&, const double*, double*, long, const int2*, long,
                                          cudaStream_t);

}  // namespace sgm
