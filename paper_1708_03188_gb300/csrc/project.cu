// project.cu - projected derivatives, project(Dx(u, axis, m), W0) of Sec. 5 of the paper:
// the kernel, its coefficient table and the C ABI entry point sgm_project_dx.
//
// W0 is the space of u with axis 0 replaced by the regular Chebyshev basis (the space itself
// when all axes are Fourier axes).  Every polynomial degree involved stays below N and
// Gauss-Chebyshev quadrature with N points integrates degree 2N - 1 exactly, so the Galerkin
// projection onto W0 of the derivative of u = sum_l u_hat_l phi_l is the Chebyshev expansion
// of the derivative itself:
//   1. basis stencil, the Shen-to-Chebyshev map of Eq. fast_shen:
//        a_q = u_hat_q + beta_{q-2} u_hat_{q-2} + gamma_{q-4} u_hat_{q-4},
//      Dirichlet beta = -1, gamma = 0; biharmonic beta_j = -2(j+2)/(j+3), gamma_j = (j+1)/(j+3)
//      (Eq. chebbiharmonic); regular Chebyshev a = u_hat.  Rows of u_hat at or past the basis
//      size read as zero;
//   2. a derivative along axis 0 applies the Chebyshev derivative recurrence m times:
//        c_k b_k = b_{k+2} + 2(k+1) a_{k+1},  c_0 = 2, c_k = 1 (k > 0),  b_N = b_{N+1} = 0,
//      or, for the Legendre bases (W0 the regular Legendre basis, the same stencil form with the
//      Legendre coefficients), b_k / (2k+1) = b_{k+2} / (2k+5) + a_{k+1};
//   3. a derivative along a Fourier axis multiplies by (i k)^m, k = 2 pi l / L with the stored
//      wavenumber l (FFT order; an R2C axis keeps l = 0..M/2).
//
// Work split.  Level j (the j-th derivative) at row r uses level j at row r + 2 and level j-1
// at row r + 1, so the output rows of one parity depend only on the input rows of the other
// parity (odd m) or the same parity (even m).  One thread takes one column (both components
// of a complex column) and one output parity, and sweeps its rows downwards: at output row k
// it holds level j at row k + m - j for every j, plus one previous value per level.  A warp
// covers 32 adjacent columns, so each row it reads or writes is one contiguous segment.
// Input rows stream through registers in chunks of kChunk rows (16 FP32, 8 FP64), the next
// chunk's loads issued before the current chunk is consumed.
//
// Arithmetic.  FP64 spaces use plain FP64.  FP32 spaces carry every intermediate as an
// unevaluated pair of floats hi + lo: exact products through one FMA (Dekker 1971, "A
// floating-point technique for extending the available precision"), Knuth's two-sum, and the
// errors summed in lo without renormalising (the cascaded sums of Ogita, Rump and Oishi 2005,
// "Accurate sum and dot product").  The result is as accurate as a computation in about twice
// FP32 precision rounded once, and the FP64 pipe (1/64 of the FP32 rate on this GPU) stays idle.
#include <algorithm>
#include <cmath>
#include <vector>

#include "space_internal.cuh"

#define PROJECT_TRY(expr)        \
  do {                           \
    const int _st = (expr);      \
    if (_st != SGM_OK) return _st; \
  } while (0)

namespace sgm {
namespace {

// input rows per register chunk: two chunks are in flight per thread; FP32 pairs leave room for
// a deeper look-ahead than FP64
template <typename T> constexpr int kChunkOf = sizeof(T) == 4 ? 16 : 8;
constexpr int kMaxOrder = 4;  // largest derivative order
constexpr int kThreads = 128;

// Fourier-axis factor of a derivative along axis d: the column index c of the kernel runs
// over the axes after the Chebyshev axis (all axes of a Fourier-only space) in C order, so
// the axis-d index is (c / inner) % n.
struct FourierDx {
  long inner;    // product of the stored extents of the axes after d
  int n;         // stored extent of axis d
  int M;         // transform length of axis d
  int r2c;       // axis d is R2C (index = wavenumber)
  int order;     // m
  double scale;  // 2 pi / L_d
};

template <typename T> struct Pair { T hi, lo; };

// ---- error-free transforms in FP32 (round-to-nearest intrinsics, never contracted) ----------
// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ Pair<float> two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// Level 0, the Chebyshev coefficient a_q = w0 + beta w2 + gamma w4 of the basis stencil.  The
// stencil is where accuracy is decided: phi_l is close to a second difference of Chebyshev
// polynomials, so derivatives of the coefficients cancel strongly and would amplify a plain
// FP32 rounding of a_q.  The products with the (hi, lo) coefficients are exact up to the lo
// terms (Dekker's product via one FMA); the sum is a cascaded two-sum whose errors collect in lo.
__device__ __forceinline__ Pair<float> stencil(float w0, float w2, float w4, Pair<float> be, Pair<float> ga) {
  const float p1 = __fmul_rn(be.hi, w2);
  const float e1 = __fmaf_rn(be.lo, w2, __fmaf_rn(be.hi, w2, -p1));
  const float p2 = __fmul_rn(ga.hi, w4);
  const float e2 = __fmaf_rn(ga.lo, w4, __fmaf_rn(ga.hi, w4, -p2));
  const Pair<float> s1 = two_sum(w0, p1);
  const Pair<float> s2 = two_sum(s1.hi, p2);
  return {s2.hi, __fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(e1, e2))};
}
__device__ __forceinline__ Pair<double> stencil(double w0, double w2, double w4, Pair<double> be, Pair<double> ga) {
  return {fma(ga.hi, w4, fma(be.hi, w2, w0)), 0.0};
}

// One step of the derivative recurrence, prev + c cur with c = 2(r+1) exact.  The pair stays
// unnormalised: hi carries the running FP32 sum and lo the exact errors of its products and
// additions (the cascaded dot product "Dot2" of Ogita, Rump and Oishi, 2005).
__device__ __forceinline__ Pair<float> level(Pair<float> prev, float c, Pair<float> cur) {
  const float p = __fmul_rn(c, cur.hi);
  const float pe = __fmaf_rn(c, cur.hi, -p);
  const Pair<float> s = two_sum(prev.hi, p);
  return {s.hi, __fadd_rn(prev.lo, __fadd_rn(s.lo, __fmaf_rn(c, cur.lo, pe)))};
}
__device__ __forceinline__ Pair<double> level(Pair<double> prev, double c, Pair<double> cur) {
  return {fma(c, cur.hi, prev.hi), 0.0};
}

// the output value (K (hi + lo) for a Fourier-axis factor K = Kh + Kl), rounded once
__device__ __forceinline__ float round_out(Pair<float> v) { return __fadd_rn(v.hi, v.lo); }
__device__ __forceinline__ double round_out(Pair<double> v) { return v.hi; }
__device__ __forceinline__ float scale_out(Pair<float> K, Pair<float> v) {
  const float p = __fmul_rn(K.hi, v.hi);
  return __fadd_rn(p, __fmaf_rn(K.hi, v.lo, __fmaf_rn(K.lo, v.hi, __fmaf_rn(K.hi, v.hi, -p))));
}
__device__ __forceinline__ double scale_out(Pair<double> K, Pair<double> v) { return K.hi * v.hi; }

// c (hi + lo) with c an integer-valued T: the product of hi exactly (one FMA), lo rounded
__device__ __forceinline__ Pair<float> pscale(float c, Pair<float> v) {
  const float p = __fmul_rn(c, v.hi);
  return {p, __fmaf_rn(c, v.lo, __fmaf_rn(c, v.hi, -p))};
}
__device__ __forceinline__ Pair<double> pscale(double c, Pair<double> v) { return {c * v.hi, 0.0}; }

template <typename T> __device__ __forceinline__ Pair<T> pval(T x) { return {x, T(0)}; }
template <typename T> __device__ __forceinline__ Pair<T> phalf(Pair<T> a) { return {a.hi * T(0.5), a.lo * T(0.5)}; }

// one input row of one column: R components, zero outside 0 <= r < nb
template <typename T, int R>
__device__ __forceinline__ void load_row(const T* __restrict__ src, long stride, int r, int nb, T (&v)[R]) {
  if (r >= 0 && r < nb) {
    if constexpr (R == 2) {
      const cplx<T> c = *reinterpret_cast<const cplx<T>*>(src + (long)r * stride);
      v[0] = c.x;
      v[1] = c.y;
    } else {
      v[0] = src[(long)r * stride];
    }
  } else {
#pragma unroll
    for (int l = 0; l < R; ++l) v[l] = T(0);
  }
}

// T: float or double.  R: 1 (the real spectral array of a 1-D Chebyshev space) or 2 (complex).
// M0: derivative order along axis 0.  LEG: axis 0 is a Legendre basis, whose derivative
// recurrence is (2r+1)^-1 b_r = (2r+5)^-1 b_{r+2} + a_{r+1}: each level keeps the running sum
// c_r = c_{r+2} + a_{r+1} and hands b_r = (2r+1) c_r on (no c_0 factor).  FAX: multiply by the Fourier factor
// (i k)^m of fx (then M0 = 0).  tab: per row j the stencil coefficients (beta_j hi, beta_j lo,
// gamma_j hi, gamma_j lo); NULL for a Fourier-only space, which has one row (N = nb = 1).
// Grid: x covers the columns, y the two output parities.
template <typename T, int R, int M0, bool FAX, bool LEG>
__global__ void __launch_bounds__(kThreads)
k_project_dx(const T* __restrict__ in, T* __restrict__ out, int N, int nb, long ncols, const T* __restrict__ tab,
             FourierDx fx) {
  const long col = (long)blockIdx.x * kThreads + threadIdx.x;
  const int par = (int)blockIdx.y;
  if (col >= ncols) return;
  const int ktop = ((N - 1) & 1) == par ? N - 1 : N - 2;  // highest output row of this parity
  if (ktop < 0) return;
  constexpr int kChunk = kChunkOf<T>;
  const long stride = ncols * R;  // elements per row
  const T* src = in + col * R;
  T* dst = out + col * R;

  Pair<T> K = pval<T>(T(1));
  int rot = 0;
  if constexpr (FAX) {
    const int idx = (int)((col / fx.inner) % fx.n);
    const double kk = fx.scale * (double)signed_wavenumber(idx, fx.M, fx.r2c);
    double kd = 1.0;
    for (int j = 0; j < fx.order; ++j) kd *= kk;
    K.hi = (T)kd;
    K.lo = (T)(kd - (double)K.hi);
    rot = fx.order & 3;
  }

  // lev[j][l], j >= 1: level j of component l at row (k + M0 - j) + 2, i.e. its previous value
  Pair<T> lev[M0 + 1][R];
#pragma unroll
  for (int j = 0; j <= M0; ++j)
#pragma unroll
    for (int l = 0; l < R; ++l) lev[j][l] = pval<T>(T(0));

  // window of u_hat rows (q + 2, q, q - 2) before step q shifts in row q - 4
  const int qtop = ktop + M0;
  T w[3][R];
  load_row<T, R>(src, stride, qtop + 2, nb, w[0]);
  load_row<T, R>(src, stride, qtop, nb, w[1]);
  load_row<T, R>(src, stride, qtop - 2, nb, w[2]);
  T buf[kChunk][R], nxt[kChunk][R];
  int row = qtop - 4;  // input row consumed by the next step
#pragma unroll
  for (int i = 0; i < kChunk; ++i) load_row<T, R>(src, stride, row - 2 * i, nb, buf[i]);

  for (int k0 = ktop; k0 >= 0; k0 -= 2 * kChunk) {
#pragma unroll
    for (int i = 0; i < kChunk; ++i) load_row<T, R>(src, stride, row - 2 * (kChunk + i), nb, nxt[i]);
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int k = k0 - 2 * i;
      if (k < 0) break;
      const int q = k + M0;  // row of level 0 at this step
#pragma unroll
      for (int l = 0; l < R; ++l) {
        w[0][l] = w[1][l];
        w[1][l] = w[2][l];
        w[2][l] = buf[i][l];
      }
      Pair<T> be = pval<T>(T(0)), ga = pval<T>(T(0));
      if (q >= 2 && q - 2 < nb) be = Pair<T>{tab[4 * (q - 2)], tab[4 * (q - 2) + 1]};
      if (q >= 4 && q - 4 < nb) ga = Pair<T>{tab[4 * (q - 4) + 2], tab[4 * (q - 4) + 3]};
      T o[R];
#pragma unroll
      for (int l = 0; l < R; ++l) {
        // level 0: Chebyshev coefficient a_q (the basis stencil)
        Pair<T> cur = stencil(w[0][l], w[1][l], w[2][l], be, ga);
        // level j at row r = q - j: b_r = b_{r+2} + 2 (r + 1) (level j-1 at row r + 1)
#pragma unroll
        for (int j = 1; j <= M0; ++j) {
          if constexpr (LEG) {
            const Pair<T> c = level(lev[j][l], T(1), cur);
            lev[j][l] = c;
            cur = pscale(T(2 * (q - j) + 1), c);
          } else {
            const Pair<T> v = level(lev[j][l], T(2 * (q - j + 1)), cur);
            lev[j][l] = v;
            cur = v;
          }
        }
        if (!LEG && M0 >= 1 && k == 0) cur = phalf(cur);  // c_0 = 2
        if constexpr (FAX)
          o[l] = scale_out(K, cur);
        else
          o[l] = round_out(cur);
      }
      if constexpr (FAX && R == 2) {  // times i^m
        const T x = o[0], y = o[1];
        if (rot == 1) {
          o[0] = -y;
          o[1] = x;
        } else if (rot == 2) {
          o[0] = -x;
          o[1] = -y;
        } else if (rot == 3) {
          o[0] = y;
          o[1] = -x;
        }
      }
      if constexpr (R == 2)
        *reinterpret_cast<cplx<T>*>(dst + (long)k * stride) = mk<cplx<T>>(o[0], o[1]);
      else
        dst[(long)k * stride] = o[0];
    }
    row -= 2 * kChunk;
#pragma unroll
    for (int i = 0; i < kChunk; ++i)
#pragma unroll
      for (int l = 0; l < R; ++l) buf[i][l] = nxt[i][l];
  }
}

template <typename T, int R, int M0, bool FAX, bool LEG>
cudaError_t launch_one(const void* in, void* out, int N, int nb, long ncols, const void* tab, const FourierDx& fx,
                       cudaStream_t s) {
  const dim3 grid((unsigned)((ncols + kThreads - 1) / kThreads), 2);
  k_project_dx<T, R, M0, FAX, LEG><<<grid, kThreads, 0, s>>>((const T*)in, (T*)out, N, nb, ncols, (const T*)tab, fx);
  return cudaGetLastError();
}

template <typename T, int R, bool LEG>
cudaError_t launch_order(int m0, const void* in, void* out, int N, int nb, long ncols, const void* tab,
                         const FourierDx& fx, cudaStream_t s) {
  switch (m0) {
    case 0: return launch_one<T, R, 0, false, LEG>(in, out, N, nb, ncols, tab, fx, s);
    case 1: return launch_one<T, R, 1, false, LEG>(in, out, N, nb, ncols, tab, fx, s);
    case 2: return launch_one<T, R, 2, false, LEG>(in, out, N, nb, ncols, tab, fx, s);
    case 3: return launch_one<T, R, 3, false, LEG>(in, out, N, nb, ncols, tab, fx, s);
    case 4: return launch_one<T, R, 4, false, LEG>(in, out, N, nb, ncols, tab, fx, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int R>
cudaError_t launch_project(int m0, bool fax, bool leg, const void* in, void* out, int N, int nb, long ncols,
                           const void* tab, const FourierDx& fx, cudaStream_t s) {
  if (fax) {  // the stencil alone, then the Fourier factor: the same for both families
    if constexpr (R == 2) return launch_one<T, 2, 0, true, false>(in, out, N, nb, ncols, tab, fx, s);
    return cudaErrorInvalidValue;
  }
  return leg ? launch_order<T, R, true>(m0, in, out, N, nb, ncols, tab, fx, s)
             : launch_order<T, R, false>(m0, in, out, N, nb, ncols, tab, fx, s);
}

template <typename T>
int upload_table(sgm_space* s, const std::vector<long double>& be, const std::vector<long double>& ga) {
  const size_t n = be.size();
  std::vector<T> h(4 * n);
  for (size_t j = 0; j < n; ++j) {
    const T bh = (T)be[j], gh = (T)ga[j];
    h[4 * j] = bh;
    h[4 * j + 1] = (T)(be[j] - (long double)bh);
    h[4 * j + 2] = gh;
    h[4 * j + 3] = (T)(ga[j] - (long double)gh);
  }
  cudaError_t e = cudaMalloc(&s->pdx_tab, sizeof(T) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(s->pdx_tab, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "derivative stencil table: %s", cudaGetErrorString(e));
  return SGM_OK;
}

// Projection onto a Shen space W (Sec. 5, project with a composite target basis).  Given the
// regular coefficients d (T_k or L_k) of a function, its Galerkin projection onto W has the
// scalar products S_k = (sum_j d_j T_j, psi_k)_w, and (T_j, T_k)_w = w_k delta_jk with
// w_k = pi c_k / 2 (Chebyshev, c_0 = 2) or 2 / (2k + 1) (Legendre), so for
// psi_k = T_k + beta_k T_{k+2} + gamma_k T_{k+4}
//   S_k = w_k d_k + beta_k w_{k+2} d_{k+2} + gamma_k w_{k+4} d_{k+4},   k < nt (rows past: 0),
// exact, since Gauss quadrature with N points integrates these degree < 2N - 1 products
// exactly.  The coefficients follow from the mass solve B c = S (space_mass_solve_f64).  S is
// formed in FP64 from the (FP32 or FP64) d, one thread per (row, column) with consecutive
// threads on consecutive columns.
struct ShenStencil {
  int legendre;    // 1: Legendre weights 2/(2k+1)
  int kind;        // kDirichlet, kNeumann or kBiharmonic (target basis)
};

__device__ __forceinline__ double series_weight(int legendre, int k) {
  if (legendre) return 2.0 / (2.0 * k + 1.0);
  return k == 0 ? 3.141592653589793 : 1.5707963267948966;
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_shen_scalar_of_series(const T* __restrict__ d, double* __restrict__ S, int N,
                                                              int nt, long ncols, ShenStencil st) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)N * ncols) return;
  const int k = (int)(idx / ncols);
  const long c = idx - (long)k * ncols;
  double out[R];
#pragma unroll
  for (int r = 0; r < R; ++r) out[r] = 0.0;
  if (k < nt) {
    double be, ga = 0.0;
    if (st.kind == kDirichlet) {
      be = -1.0;
    } else if (st.kind == kNeumann) {
      be = -neumann_q<double>(k);
    } else if (st.legendre) {
      be = -2.0 * (2 * k + 5) / (double)(2 * k + 7);
      ga = (double)(2 * k + 3) / (double)(2 * k + 7);
    } else {
      be = -2.0 * (k + 2) / (double)(k + 3);
      ga = (double)(k + 1) / (double)(k + 3);
    }
    const double w0 = series_weight(st.legendre, k), w2 = be * series_weight(st.legendre, k + 2),
                 w4 = ga * series_weight(st.legendre, k + 4);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double a0 = (double)d[((long)k * ncols + c) * R + r];
      const double a2 = k + 2 < N ? (double)d[((long)(k + 2) * ncols + c) * R + r] : 0.0;
      const double a4 = k + 4 < N ? (double)d[((long)(k + 4) * ncols + c) * R + r] : 0.0;
      out[r] = fma(w4, a4, fma(w2, a2, w0 * a0));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) S[idx * R + r] = out[r];
}

// FP64 -> T, n values (round to nearest)
template <typename T>
__global__ void __launch_bounds__(256) k_narrow_copy(const double* __restrict__ in, T* __restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

}  // namespace

int build_project_table(sgm_space* s) {
  if (!s->cheb) return SGM_OK;
  const int N = (int)s->n[0];
  std::vector<long double> be(N, 0.0L), ga(N, 0.0L);
  for (int j = 0; j < N; ++j) {
    if (s->kinds[0] == SGM_SHEN_DIRICHLET || s->kinds[0] == SGM_LEGENDRE_DIRICHLET) {
      be[j] = -1.0L;
    } else if (s->kinds[0] == SGM_SHEN_NEUMANN) {
      const long double r = (long double)j / (long double)(j + 2);
      be[j] = -r * r;
    } else if (s->kinds[0] == SGM_SHEN_BIHARMONIC) {
      be[j] = -2.0L * (j + 2) / (long double)(j + 3);
      ga[j] = (long double)(j + 1) / (long double)(j + 3);
    } else if (s->kinds[0] == SGM_LEGENDRE_BIHARMONIC) {
      be[j] = -2.0L * (2 * j + 5) / (long double)(2 * j + 7);
      ga[j] = (long double)(2 * j + 3) / (long double)(2 * j + 7);
    }
  }
  return s->prec == SGM_F32 ? upload_table<float>(s, be, ga) : upload_table<double>(s, be, ga);
}

}  // namespace sgm

using namespace sgm;

namespace {

// project(Dx(u, axis, order), W0) with W0 the regular basis: writes the regular coefficients to
// `out` (spectral layout of s, type of s's precision).  Arguments checked by the callers.
int project_regular(sgm_space* s, int axis, int order, const void* u_hat, void* out, cudaStream_t cs) {
  const int N = s->cheb ? (int)s->n[0] : 1;
  int nb = 1;
  if (s->cheb)
    nb = (s->kinds[0] == SGM_SHEN_DIRICHLET || s->kinds[0] == SGM_LEGENDRE_DIRICHLET ||
          s->kinds[0] == SGM_SHEN_NEUMANN)                                                   ? N - 2
         : (s->kinds[0] == SGM_SHEN_BIHARMONIC || s->kinds[0] == SGM_LEGENDRE_BIHARMONIC) ? N - 4
                                                                                           : N;
  const long ncols = s->nspec / N;
  const bool cheb_axis = s->cheb && axis == 0;
  const int m0 = cheb_axis ? order : 0;
  const bool fax = !cheb_axis && order > 0;
  FourierDx fx{1, 1, 1, 0, 0, 0.0};
  if (fax) {
    fx.inner = 1;
    for (int d = axis + 1; d < s->ndim; ++d) fx.inner *= s->spec[d];
    fx.n = (int)s->spec[axis];
    fx.M = (int)s->n[axis];
    fx.r2c = s->kinds[axis] == SGM_FOURIER_R2C;
    fx.order = order;
    fx.scale = 2.0 * 3.14159265358979323846 / (s->dom[2 * axis + 1] - s->dom[2 * axis]);
  }
  cudaError_t e;
  if (s->prec == SGM_F32)
    e = s->real_spec ? launch_project<float, 1>(m0, fax, s->legendre, u_hat, out, N, nb, ncols, s->pdx_tab, fx, cs)
                     : launch_project<float, 2>(m0, fax, s->legendre, u_hat, out, N, nb, ncols, s->pdx_tab, fx, cs);
  else
    e = s->real_spec ? launch_project<double, 1>(m0, fax, s->legendre, u_hat, out, N, nb, ncols, s->pdx_tab, fx, cs)
                     : launch_project<double, 2>(m0, fax, s->legendre, u_hat, out, N, nb, ncols, s->pdx_tab, fx, cs);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "project_dx: %s", cudaGetErrorString(e));
  return SGM_OK;
}

int project_args(sgm_space* s, int axis, int order, const void* u_hat, const void* du_hat) {
  const int st = space_check(s);
  if (st != SGM_OK) return st;
  if (axis < 0 || axis >= s->ndim) return set_error(SGM_ERR_ARG, "axis %d outside 0..%d", axis, s->ndim - 1);
  if (order < 0 || order > kMaxOrder) return set_error(SGM_ERR_ARG, "order %d outside 0..%d", order, kMaxOrder);
  if (!u_hat || !du_hat) return set_error(SGM_ERR_NULL, "NULL data pointer");
  if (((uintptr_t)u_hat & 15) || ((uintptr_t)du_hat & 15))
    return set_error(SGM_ERR_ALIGN, "data pointers must be 16-byte aligned");
  const char* a = (const char*)u_hat;
  const char* b = (const char*)du_hat;
  if (a < b + s->spec_bytes && b < a + s->spec_bytes) return set_error(SGM_ERR_ALIAS, "u_hat and du_hat overlap");
  if (s->cheb && !s->inner && !s->pdx_tab) return set_error(SGM_ERR_STATE, "space has no derivative stencil table");
  return SGM_OK;
}

bool is_regular(int kind) { return kind == SGM_CHEBYSHEV || kind == SGM_LEGENDRE; }
bool is_legendre_kind(int kind) {
  return kind == SGM_LEGENDRE || kind == SGM_LEGENDRE_DIRICHLET || kind == SGM_LEGENDRE_BIHARMONIC;
}

}  // namespace

extern "C" int sgm_project_dx(sgm_space* s, int axis, int order, const void* u_hat, void* du_hat, void* stream) {
  const int st = project_args(s, axis, order, u_hat, du_hat);
  if (st != SGM_OK) return st;
  if (s->inner) {  // a permuted space (axes.cu): the canonical call on canonical copies
    cudaStream_t cs = (cudaStream_t)stream;
    PROJECT_TRY(to_canonical(s, SGM_SPECTRAL, u_hat, s->P1, cs));
    PROJECT_TRY(sgm_project_dx(s->inner, s->perm[axis], order, s->P1, s->P2, stream));
    return from_canonical(s, SGM_SPECTRAL, s->P2, du_hat, cs);
  }
  return project_regular(s, axis, order, u_hat, du_hat, (cudaStream_t)stream);
}

extern "C" int sgm_project(sgm_space* s, int axis, int order, const void* u_hat, sgm_space* target, void* out_hat,
                           void* stream) {
  int st = project_args(s, axis, order, u_hat, out_hat);
  if (st != SGM_OK) return st;
  st = space_check(target);
  if (st != SGM_OK) return st;
  if (s->inner || target->inner) {  // permuted spaces (axes.cu): both in the same axis order
    if (!s->inner || !target->inner || target->ndim != s->ndim)
      return set_error(SGM_ERR_STATE, "target space has another axis order");
    for (int d = 0; d < s->ndim; ++d)
      if (target->perm[d] != s->perm[d]) return set_error(SGM_ERR_STATE, "target space has another axis order");
    cudaStream_t cs = (cudaStream_t)stream;
    PROJECT_TRY(to_canonical(s, SGM_SPECTRAL, u_hat, s->P1, cs));
    PROJECT_TRY(sgm_project(s->inner, s->perm[axis], order, s->P1, target->inner, target->P2, stream));
    return from_canonical(target, SGM_SPECTRAL, target->P2, out_hat, cs);
  }
  if (target->ndim != s->ndim || target->prec != s->prec || target->cheb != s->cheb)
    return set_error(SGM_ERR_STATE, "target space differs in dimension, precision or axis-0 family");
  for (int d = 0; d < s->ndim; ++d) {
    if (target->n[d] != s->n[d] || target->dom[2 * d] != s->dom[2 * d] || target->dom[2 * d + 1] != s->dom[2 * d + 1])
      return set_error(SGM_ERR_STATE, "target space differs in size or domain along axis %d", d);
    if (d > 0 || !s->cheb)
      if (target->kinds[d] != s->kinds[d]) return set_error(SGM_ERR_STATE, "target space differs along Fourier axis %d", d);
  }
  const char* a = (const char*)u_hat;
  const char* b = (const char*)out_hat;
  if (a < b + target->spec_bytes && b < a + target->spec_bytes) return set_error(SGM_ERR_ALIAS, "u_hat and out_hat overlap");
  cudaStream_t cs = (cudaStream_t)stream;
  if (!s->cheb || is_regular(target->kinds[0])) {
    if (s->cheb && is_legendre_kind(target->kinds[0]) != (bool)s->legendre)
      return set_error(SGM_ERR_STATE, "target basis is of another polynomial family");
    return project_regular(s, axis, order, u_hat, out_hat, cs);
  }
  if (is_legendre_kind(target->kinds[0]) != (bool)s->legendre)
    return set_error(SGM_ERR_STATE, "target basis is of another polynomial family");
  // regular coefficients of the derivative in s->W1, the target's scalar products in FP64 in
  // target->W2, the FP64 mass solve in place, then the result in the space's precision
  PROJECT_TRY(project_regular(s, axis, order, u_hat, s->W1, cs));
  const int N = (int)s->n[0];
  const long ncols = s->nspec / N;
  const int tk = target->kinds[0];
  ShenStencil sst{target->legendre ? 1 : 0,
                  (tk == SGM_SHEN_DIRICHLET || tk == SGM_LEGENDRE_DIRICHLET) ? (int)kDirichlet
                  : tk == SGM_SHEN_NEUMANN                                   ? (int)kNeumann
                                                                             : (int)kBiharmonic};
  const int nt = basis_count(sst.kind, N);
  const long total = (long)N * ncols;
  const unsigned grid = (unsigned)((total + 255) / 256);
  const int R = s->real_spec ? 1 : 2;
  void* S = (s->prec == SGM_F64) ? out_hat : target->W2;
  if (s->prec == SGM_F32) {
    if (R == 1) k_shen_scalar_of_series<float, 1><<<grid, 256, 0, cs>>>((const float*)s->W1, (double*)S, N, nt, ncols, sst);
    else k_shen_scalar_of_series<float, 2><<<grid, 256, 0, cs>>>((const float*)s->W1, (double*)S, N, nt, ncols, sst);
  } else {
    if (R == 1) k_shen_scalar_of_series<double, 1><<<grid, 256, 0, cs>>>((const double*)s->W1, (double*)S, N, nt, ncols, sst);
    else k_shen_scalar_of_series<double, 2><<<grid, 256, 0, cs>>>((const double*)s->W1, (double*)S, N, nt, ncols, sst);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "project: %s", cudaGetErrorString(e));
  PROJECT_TRY(space_mass_solve_f64(target, S, cs));
  if (s->prec == SGM_F32) {
    const long nv = total * R;
    k_narrow_copy<float><<<(unsigned)std::min<long>((nv + 255) / 256, 152L * 16), 256, 0, cs>>>((const double*)S, (float*)out_hat, nv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "project: %s", cudaGetErrorString(e));
  }
  return SGM_OK;
}
