// legendre.cu - Legendre bases on axis 0: dense transforms, banded FP64 solves, and the host
// tables of both.  The bases (Sec. 3.1 lists them; Eq. legdirichlet; Eq. legbiharmonic, whose
// printed last term lacks its factor L_{l+4}, which phi(+-1) = phi'(+-1) = 0 requires):
//   regular      phi_l = L_l                                       l = 0..N-1
//   Dirichlet    phi_l = L_l - L_{l+2}                             l = 0..N-3
//   biharmonic   phi_l = L_l + beta_l L_{l+2} + gamma_l L_{l+4}    l = 0..N-5
//                beta_l = -2(2l+5)/(2l+7),  gamma_l = (2l+3)/(2l+7)
// on the Legendre-Gauss points x_j (descending) with weights w_j (weight function 1).
//
// Transforms.  No fast transform is known for Legendre series and the paper uses O(N^2) sums
// for them (Sec. 3.4.2), so each axis-0 operation is one dense N x N matrix applied to every
// column, Y = P X (complex data as interleaved real columns):
//   scalar product   P[k][j] = w_j phi_k(x_j)               rows past the basis are zero
//   backward         P[j][k] = phi_k(x_j)                   columns past the basis are zero
//   forward (L_k)    P[k][j] = (2k+1)/2 w_j L_k(x_j)         the mass matrix is diag(2/(2k+1))
// k_dense_axis0 is a tiled product: a 64 x 64 output tile per CTA, 16-deep slices of P and X
// staged in shared memory, 4 x 4 outputs per thread, accumulated in the space's precision.  FP32
// spaces of N <= 128 created with SGM_CHEB_TC or SGM_CHEB_AUTO can run the same products on the
// tensor cores instead: the images of these matrices feed the BF16x3 contraction of k_cheb_tc.cu.
//
// Solves.  With weight 1 the weak forms integrate by parts, (phi_l'', phi_m) = -(phi_l', phi_m')
// and (phi_l'''', phi_m) = (phi_l'', phi_m''), and the derivatives of the bases have one or two
// Legendre terms (from L_{n+1}' - L_{n-1}' = (2n+1) L_n):
//   Dirichlet    phi_k'  = -(2k+3) L_{k+1}
//   biharmonic   phi_k'  = c1_k L_{k+1} + c3_k L_{k+3},  c1_k = (2k+3)(beta_k + gamma_k),
//                                                       c3_k = (2k+7) gamma_k
//                phi_k'' = d_k L_{k+2},  d_k = (2k+5) c3_k
// (the L_k' terms cancel because 1 + beta_k + gamma_k = 0, the L_{k+1}' terms because
// c1_k + c3_k = 0).  With (L_i, L_j) = 2/(2i+1) delta_ij every matrix is banded within a parity:
//   Dirichlet    A_kk = -(4k+6);  B_kk = 2/(2k+1) + 2/(2k+5),  B_{k,k+2} = -2/(2k+5)
//   biharmonic   S_kk = 2 d_k^2/(2k+5)
//                A_kk = -(2 c1_k^2/(2k+3) + 2 c3_k^2/(2k+7)),  A_{k,k+2} = -2 c3_k c1_{k+2}/(2k+7)
//                B_kk = 2/(2k+1) + 2 beta_k^2/(2k+5) + 2 gamma_k^2/(2k+9)
//                B_{k,k+2} = 2 beta_k/(2k+5) + 2 gamma_k beta_{k+2}/(2k+9),  B_{k,k+4} = 2 gamma_k/(2k+9)
// Each (column, parity) system is therefore symmetric with at most two bands on either side in
// the parity's own index (i = (k - p)/2).  k_legendre_solve factors it as L U without pivoting
// (the Poisson and biharmonic systems are symmetric positive definite), U with a unit
// diagonal: per row the pivot mu_i, the two upper multipliers alpha_i, beta_i and the
// forward-substituted right-hand side z_i go to scratch, then the back substitution
// x_i = z_i - alpha_i x_{i+1} - beta_i x_{i+2} runs upwards.  All of it in FP64, one thread per
// (column, parity).
#include <cmath>
#include <vector>

#include "convert.cuh"
#include "space_internal.cuh"

namespace sgm {
namespace {

constexpr int kLegMaxN = 1024;          // dense N x N matrices per space
constexpr int kBandValues = 6;          // S_kk, A_kk, A_{k,k+2}, B_kk, B_{k,k+2}, B_{k,k+4}
constexpr int kSolveValues = 4;         // scratch per row: alpha, beta, Re z, Im z
const long double kPiL = 3.141592653589793238462643383279502884L;

// ---- host tables ------------------------------------------------------------------------------
// Legendre-Gauss points (descending) and weights: Newton's iteration on L_N from the
// asymptotic first guess cos(pi (j + 3/4) / (N + 1/2)), with L_N and L_N' from the three-term
// recurrence; w_j = 2 / ((1 - x_j^2) L_N'(x_j)^2).
void gauss_legendre(int N, std::vector<long double>& x, std::vector<long double>& w) {
  x.assign(N, 0.0L);
  w.assign(N, 0.0L);
  for (int j = 0; j < N; ++j) {
    long double z = std::cos(kPiL * (j + 0.75L) / (N + 0.5L));
    long double dp = 1.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = z;
      for (int n = 2; n <= N; ++n) {
        const long double p2 = ((2 * n - 1) * z * p1 - (n - 1) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (N == 1) p0 = 1.0L;  // L_0
      dp = N * (z * p1 - p0) / (z * z - 1.0L);
      const long double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-19L) break;
    }
    x[j] = z;
    w[j] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

// coefficients of phi_k in the Legendre basis: (1, beta, gamma) at L_k, L_{k+2}, L_{k+4}
void basis_terms(int kind, int k, long double& be, long double& ga) {
  be = ga = 0.0L;
  if (kind == SGM_LEGENDRE_DIRICHLET) {
    be = -1.0L;
  } else if (kind == SGM_LEGENDRE_BIHARMONIC) {
    be = -2.0L * (2 * k + 5) / (long double)(2 * k + 7);
    ga = (long double)(2 * k + 3) / (long double)(2 * k + 7);
  }
}

int num_basis(int kind, int N) {
  return kind == SGM_LEGENDRE_DIRICHLET ? N - 2 : kind == SGM_LEGENDRE_BIHARMONIC ? N - 4 : N;
}

// dense axis-0 matrices, row-major N x N, for the ChebMode modes (forward only for SGM_LEGENDRE)
std::vector<std::vector<long double>> dense_matrices(int kind, int N) {
  std::vector<long double> x, w;
  gauss_legendre(N, x, w);
  // L[j][n] = L_n(x_j), n = 0..N-1
  std::vector<long double> L((size_t)N * N);
  for (int j = 0; j < N; ++j) {
    long double p0 = 1.0L, p1 = x[j];
    L[(size_t)j * N] = 1.0L;
    if (N > 1) L[(size_t)j * N + 1] = p1;
    for (int n = 2; n < N; ++n) {
      const long double p2 = ((2 * n - 1) * x[j] * p1 - (n - 1) * p0) / n;
      L[(size_t)j * N + n] = p2;
      p0 = p1;
      p1 = p2;
    }
  }
  const int nb = num_basis(kind, N);
  auto phi = [&](int k, int j) {  // phi_k(x_j)
    long double be, ga;
    basis_terms(kind, k, be, ga);
    long double v = L[(size_t)j * N + k];
    if (be != 0.0L) v += be * L[(size_t)j * N + k + 2];
    if (ga != 0.0L) v += ga * L[(size_t)j * N + k + 4];
    return v;
  };
  std::vector<std::vector<long double>> out(3, std::vector<long double>((size_t)N * N, 0.0L));
  for (int k = 0; k < nb; ++k)
    for (int j = 0; j < N; ++j) {
      const long double v = phi(k, j);
      out[kChebScalar][(size_t)k * N + j] = w[j] * v;
      out[kChebBackward][(size_t)j * N + k] = v;
    }
  if (kind == SGM_LEGENDRE)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        out[kChebForwardT][(size_t)k * N + j] = 0.5L * (2 * k + 1) * w[j] * L[(size_t)j * N + k];
  return out;
}

// band entries per basis row k (kBandValues doubles): S_kk, A_kk, A_{k,k+2}, B_kk, B_{k,k+2},
// B_{k,k+4}; entries that reach past the basis are zero
long double lsq(int i) { return 2.0L / (2 * i + 1); }  // (L_i, L_i)

std::vector<double> band_table(int kind, int N) {
  const int nb = num_basis(kind, N);
  std::vector<double> t((size_t)nb * kBandValues, 0.0);
  for (int k = 0; k < nb; ++k) {
    long double S = 0, Ad = 0, Ao = 0, Bd = 0, Bo2 = 0, Bo4 = 0;
    if (kind == SGM_LEGENDRE_DIRICHLET) {
      Ad = -(4.0L * k + 6.0L);
      Bd = lsq(k) + lsq(k + 2);
      if (k + 2 < nb) Bo2 = -lsq(k + 2);
    } else if (kind == SGM_LEGENDRE_BIHARMONIC) {
      long double be, ga, be2, ga2;
      basis_terms(kind, k, be, ga);
      basis_terms(kind, k + 2, be2, ga2);
      const long double c1 = (2 * k + 3) * (be + ga), c3 = (2 * k + 7) * ga;
      const long double c1n = (2 * k + 7) * (be2 + ga2);  // c1 of row k + 2
      const long double d = (2 * k + 5) * c3;
      S = d * d * lsq(k + 2);
      Ad = -(c1 * c1 * lsq(k + 1) + c3 * c3 * lsq(k + 3));
      Bd = lsq(k) + be * be * lsq(k + 2) + ga * ga * lsq(k + 4);
      if (k + 2 < nb) {
        Ao = -c3 * c1n * lsq(k + 3);
        Bo2 = be * lsq(k + 2) + ga * be2 * lsq(k + 4);
      }
      if (k + 4 < nb) Bo4 = ga * lsq(k + 4);
    } else {
      Bd = lsq(k);
    }
    const long double v[kBandValues] = {S, Ad, Ao, Bd, Bo2, Bo4};
    for (int i = 0; i < kBandValues; ++i) t[(size_t)k * kBandValues + i] = (double)v[i];
  }
  return t;
}

// ---- dense axis-0 product ---------------------------------------------------------------------
template <typename TO, typename TI> __device__ __forceinline__ TO cvt(TI v);
template <> __device__ __forceinline__ float cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ double cvt<double, float>(float v) { return widen_f32(v); }
template <> __device__ __forceinline__ float cvt<float, double>(double v) { return narrow_f64(v); }

constexpr int kBM = 64, kBN = 64, kBK = 16, kDenseThreads = 256;

// Y[r][c] = sum_j P[r][j] X[j][c], r, j < N, c < C; P in the accumulation type T, X of type TI,
// Y of type TO.  Grid: x over 64-column tiles, y over 64-row tiles.
template <typename T, typename TI, typename TO>
__global__ void __launch_bounds__(kDenseThreads)
k_dense_axis0(const T* __restrict__ P, const TI* __restrict__ X, TO* __restrict__ Y, int N, long C) {
  __shared__ T Ps[kBK][kBM];  // Ps[kk][r] = P[r0 + r][k0 + kk]
  __shared__ T Xs[kBK][kBN];  // Xs[kk][c] = X[k0 + kk][c0 + c]
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.y * kBM;
  const long c0 = (long)blockIdx.x * kBN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < N; k0 += kBK) {
    for (int e = threadIdx.x; e < kBM * kBK; e += kDenseThreads) {
      const int r = e / kBK, kk = e % kBK;
      const int gr = r0 + r, gk = k0 + kk;
      Ps[kk][r] = (gr < N && gk < N) ? P[(long)gr * N + gk] : T(0);
    }
    for (int e = threadIdx.x; e < kBK * kBN; e += kDenseThreads) {
      const int kk = e / kBN, c = e % kBN;
      const int gk = k0 + kk;
      const long gc = c0 + c;
      Xs[kk][c] = (gk < N && gc < C) ? cvt<T, TI>(X[(long)gk * C + gc]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ps[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Xs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = r0 + ty * 4 + i;
    if (gr >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long gc = c0 + tx + 16 * j;
      if (gc < C) Y[(long)gr * C + gc] = cvt<TO, T>(acc[i][j]);
    }
  }
}

// ---- banded FP64 solve ------------------------------------------------------------------------
// One work item = (column, parity); items = 2 * ncols, parity-major so that a warp holds one
// parity of adjacent columns.  TS: spectral data type (float or double), R: 1 (real) or 2
// (complex) components.  band: kBandValues per basis row; scratch: [row][kSolveValues][thread]
// for nthreads threads that stride over the items.
template <typename TS, int R>
__global__ void __launch_bounds__(128)
k_legendre_solve(const TS* __restrict__ in, TS* __restrict__ out, int N, int nb, long ncols, double a, double b,
                 double c, Wavenumbers wn, const double* __restrict__ band, double* __restrict__ scratch,
                 long nthreads) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  const long stride = ncols * R;
  for (long item = t; item < 2 * ncols; item += nthreads) {
    const int par = (int)(item / ncols);
    const long col = item - (long)par * ncols;
    const int np = (nb - par + 1) / 2;  // rows of this parity
    if (np <= 0) continue;
    const double k2 = kappa2_of(wn, col);
    // M = a (S - 2 k2 A + k2^2 B) + b (A - k2 B) + c B, band by band
    const double cS = a, cA = -2.0 * a * k2 + b, cB = a * k2 * k2 - b * k2 + c;
    auto row = [&](int i, double& d, double& u1, double& u2) {  // diagonal, +1, +2 of row i
      const double* e = band + (long)(par + 2 * i) * kBandValues;
      d = cS * e[0] + cA * e[1] + cB * e[3];
      u1 = cA * e[2] + cB * e[4];
      u2 = cB * e[5];
    };
    // forward elimination: L has e_i (i, i-2), g_i (i, i-1), mu_i; U has 1, alpha_i, beta_i
    double al1 = 0, al2 = 0, bt1 = 0, bt2 = 0;         // alpha, beta of rows i-1, i-2
    double up1_1 = 0, up2_1 = 0, up2_2 = 0;            // M(i-1, i), M(i-2, i): the lower entries
    double z1[R], z2[R];
#pragma unroll
    for (int l = 0; l < R; ++l) z1[l] = z2[l] = 0.0;
    for (int i = 0; i < np; ++i) {
      double d, u1, u2;
      row(i, d, u1, u2);
      const double e = up2_2;                          // M(i, i-2) = M(i-2, i)
      const double g = up1_1 - al2 * e;                // M(i, i-1) - e alpha_{i-2}
      const double mu = d - bt2 * e - al1 * g;
      const double rmu = 1.0 / mu;
      const double al = (u1 - bt1 * g) * rmu;
      const double bt = u2 * rmu;
      const long k = par + 2 * i;
      double y[R], z[R];
      if constexpr (R == 2) {
        const cplx<TS> v = *reinterpret_cast<const cplx<TS>*>(in + k * stride + col * 2);
        y[0] = widen<TS>(v.x);
        y[1] = widen<TS>(v.y);
      } else {
        y[0] = widen<TS>(in[k * stride + col]);
      }
#pragma unroll
      for (int l = 0; l < R; ++l) z[l] = (y[l] - e * z2[l] - g * z1[l]) * rmu;
      double* sc = scratch + (long)i * kSolveValues * nthreads + t;
      sc[0] = al;
      sc[nthreads] = bt;
#pragma unroll
      for (int l = 0; l < R; ++l) sc[(2 + l) * nthreads] = z[l];
      al2 = al1;
      al1 = al;
      bt2 = bt1;
      bt1 = bt;
      up2_2 = up2_1;
      up2_1 = u2;
      up1_1 = u1;
#pragma unroll
      for (int l = 0; l < R; ++l) {
        z2[l] = z1[l];
        z1[l] = z[l];
      }
    }
    // back substitution x_i = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
    double x1[R], x2[R];
#pragma unroll
    for (int l = 0; l < R; ++l) x1[l] = x2[l] = 0.0;
    for (int i = np - 1; i >= 0; --i) {
      const double* sc = scratch + (long)i * kSolveValues * nthreads + t;
      const double al = sc[0], bt = sc[nthreads];
      double x[R];
#pragma unroll
      for (int l = 0; l < R; ++l) x[l] = sc[(2 + l) * nthreads] - al * x1[l] - bt * x2[l];
      const long k = par + 2 * i;
      if constexpr (R == 2)
        *reinterpret_cast<cplx<TS>*>(out + k * stride + col * 2) = mk<cplx<TS>>(narrow<TS>(x[0]), narrow<TS>(x[1]));
      else
        out[k * stride + col] = narrow<TS>(x[0]);
#pragma unroll
      for (int l = 0; l < R; ++l) {
        x2[l] = x1[l];
        x1[l] = x[l];
      }
    }
    // rows past the basis are zero (only parity-owned rows are written, so each row once)
    for (int k = nb + ((nb & 1) != par ? 1 : 0); k < N; k += 2) {
      if constexpr (R == 2)
        *reinterpret_cast<cplx<TS>*>(out + (long)k * stride + col * 2) = mk<cplx<TS>>(TS(0), TS(0));
      else
        out[(long)k * stride + col] = TS(0);
    }
  }
}

// ---- host side --------------------------------------------------------------------------------
template <typename T>
int upload(const std::vector<long double>& m, void** out) {
  std::vector<T> h(m.size());
  for (size_t i = 0; i < m.size(); ++i) h[i] = (T)m[i];
  cudaError_t e = cudaMalloc(out, sizeof(T) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(*out, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre matrices: %s", cudaGetErrorString(e));
  return SGM_OK;
}

template <typename T, typename TI, typename TO>
cudaError_t launch_dense(const void* P, const void* in, void* out, int N, long C, cudaStream_t s) {
  const dim3 grid((unsigned)((C + kBN - 1) / kBN), (unsigned)((N + kBM - 1) / kBM));
  k_dense_axis0<T, TI, TO><<<grid, kDenseThreads, 0, s>>>((const T*)P, (const TI*)in, (TO*)out, N, C);
  return cudaGetLastError();
}

}  // namespace

int legendre_build(sgm_space* s, bool tc_images) {
  const int N = (int)s->n[0], kind = s->kinds[0];
  if (N > kLegMaxN) return set_error(SGM_ERR_SIZE, "Legendre bases need N <= %d (got %d)", kLegMaxN, N);
  const auto mats = dense_matrices(kind, N);
  for (int mode : {kChebScalar, kChebBackward, kChebForwardT}) {
    if (mode == kChebForwardT && kind != SGM_LEGENDRE) continue;
    const int st = s->prec == SGM_F32 ? upload<float>(mats[mode], &s->leg_mat[mode])
                                      : upload<double>(mats[mode], &s->leg_mat[mode]);
    if (st != SGM_OK) return st;
    if (tc_images && s->prec == SGM_F32 && N <= kTcMaxN) {  // BF16x3 contraction images (k_cheb_tc.cu)
      const std::vector<uint16_t> img = tc_matrix_image(mats[mode], N);
      cudaError_t e = cudaMalloc(&s->tc_img[mode], img.size() * 2);
      if (e == cudaSuccess) e = cudaMemcpy(s->tc_img[mode], img.data(), img.size() * 2, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre contraction matrix: %s", cudaGetErrorString(e));
    }
  }
  if (kind == SGM_LEGENDRE) return SGM_OK;  // no solves on the regular basis
  const std::vector<double> band = band_table(kind, N);
  cudaError_t e = cudaMalloc(&s->leg_band, sizeof(double) * band.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(s->leg_band, band.data(), sizeof(double) * band.size(), cudaMemcpyHostToDevice);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre band table: %s", cudaGetErrorString(e));
  const long items = 2 * (s->nspec / N);
  s->leg_threads = std::min((long)std::max(1, sms) * 256, ((items + 127) / 128) * 128);
  const long rows = (num_basis(kind, N) + 1) / 2;
  e = cudaMalloc(&s->leg_scratch, sizeof(double) * rows * kSolveValues * s->leg_threads);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre solve scratch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

int legendre_pass(sgm_space* s, int mode, const void* in, void* out, cudaStream_t st, bool wide) {
  const int N = (int)s->n[0];
  const void* P = (mode >= 0 && mode < 3) ? s->leg_mat[mode] : nullptr;
  if (!P) return set_error(SGM_ERR_STATE, "this Legendre basis has no matrix for axis-0 mode %d", mode);
  long inner = 1;
  for (int d = 1; d < s->ndim; ++d) inner *= s->spec[d];
  const long C = inner * (s->real_spec ? 1 : 2);
  cudaError_t e;
  if (s->prec == SGM_F64)
    e = launch_dense<double, double, double>(P, in, out, N, C, st);
  else if (!wide)
    e = launch_dense<float, float, float>(P, in, out, N, C, st);
  else if (mode == kChebBackward)
    e = launch_dense<float, double, float>(P, in, out, N, C, st);   // FP64 spectral in
  else
    e = launch_dense<float, float, double>(P, in, out, N, C, st);   // FP64 spectral out
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre axis-0 pass: %s", cudaGetErrorString(e));
  return SGM_OK;
}

template <typename TS>
int legendre_solve(sgm_space* s, double a, double b, double c, const void* in, void* out, const Wavenumbers& wn,
                   cudaStream_t st) {
  if (!s->leg_band || !s->leg_scratch) return set_error(SGM_ERR_STATE, "this Legendre basis has no solver");
  const int N = (int)s->n[0];
  const int nb = num_basis(s->kinds[0], N);
  const long ncols = s->nspec / N;
  const unsigned grid = (unsigned)((s->leg_threads + 127) / 128);
  if (s->real_spec)
    k_legendre_solve<TS, 1><<<grid, 128, 0, st>>>((const TS*)in, (TS*)out, N, nb, ncols, a, b, c, wn, s->leg_band,
                                                   s->leg_scratch, s->leg_threads);
  else
    k_legendre_solve<TS, 2><<<grid, 128, 0, st>>>((const TS*)in, (TS*)out, N, nb, ncols, a, b, c, wn, s->leg_band,
                                                   s->leg_scratch, s->leg_threads);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Legendre solve: %s", cudaGetErrorString(e));
  return SGM_OK;
}

template int legendre_solve<float>(sgm_space*, double, double, double, const void*, void*, const Wavenumbers&,
                                   cudaStream_t);
template int legendre_solve<double>(sgm_space*, double, double, double, const void*, void*, const Wavenumbers&,
                                    cudaStream_t);

}  // namespace sgm
