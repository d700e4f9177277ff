// common.cuh - complex helpers, FFT plan and launcher declarations shared by the
// libsgm kernels.  Host and device code; no torch types anywhere.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sgm {

// ---- complex arithmetic on float2 / double2 -------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using cplx = typename cvec<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
  return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// ---- FFT plan ---------------------------------------------------------------------------
// A length-L transform is a sequence of Stockham radix passes; the product of the
// radices is L.  `tw` points at exp(-2 pi i k / L), k = 0..L-1, in the transform's
// precision.
constexpr int kMaxPasses = 24;
// dynamic shared memory a staged-tile kernel may request (of the 227 KB per CTA)
constexpr long kSmemBudget = 160 * 1024;
struct FftPlan {
  int L;
  int npass;
  int radix[kMaxPasses];
};

// ---- Shen basis kinds (mirror of sgm.h) -------------------------------------------------
enum Basis { kCheb = 0, kDirichlet = 1, kBiharmonic = 2, kC2C = 3, kR2C = 4, kNeumann = 8 };
// Shen Neumann basis phi_k = T_k - q_k T_{k+2}, q_k = (k / (k + 2))^2
template <typename T> __host__ __device__ __forceinline__ T neumann_q(int k) {
  const T r = (T)k / (T)(k + 2);
  return r * r;
}
// number of basis functions of a Chebyshev-family axis of N points
__host__ __device__ __forceinline__ int basis_count(int basis, int N) {
  return (basis == kDirichlet || basis == kNeumann) ? N - 2 : (basis == kBiharmonic ? N - 4 : N);
}

// Fourier wavenumber layout of the columns of a spectral array (used by the solves):
// a column index c = i1 * n2 + i2 (3-D) or c = i2 (2-D) or c = 0 (1-D);
// kappa^2 = s1 * l1^2 + s2 * l2^2 with l the signed wavenumber of the index.
struct Wavenumbers {
  int n1, n2;        // stored extents of axes 1 and 2 (1 if absent)
  int m1, m2;        // transform lengths (for signed wavenumbers of C2C axes)
  int r2c1, r2c2;    // 1 if that axis is R2C (index = wavenumber)
  double s1, s2;     // (2 pi / L)^2 per axis (0 if absent)
};

__host__ __device__ __forceinline__ int signed_wavenumber(int idx, int m, int r2c) {
  return (r2c || idx < (m + 1) / 2) ? idx : idx - m;
}

__device__ __forceinline__ double kappa2_of(const Wavenumbers& w, long c) {
  int i1 = (int)(c / w.n2), i2 = (int)(c - (long)i1 * w.n2);
  double l1 = signed_wavenumber(i1, w.m1, w.r2c1), l2 = signed_wavenumber(i2, w.m2, w.r2c2);
  return w.s1 * l1 * l1 + w.s2 * l2 * l2;
}

// ---- error reporting (space.cu): sets the thread-local message of sgm_last_error ---------
int set_error(int code, const char* fmt, ...);
// radix sequence of the runtime engine for length L (space.cu)
FftPlan host_plan(int L);

// ---- launchers (defined in k_fourier.cu, k_cheb.cu, k_solve.cu) --------------------------
// All return cudaGetLastError() after the launch.
enum RowMode { kRowR2C = 0, kRowC2R = 1, kRowC2CFwd = 2, kRowC2CInv = 3 };

template <typename T>
cudaError_t launch_rows(int mode, const void* in, void* out, long nrows, int L, const FftPlan& plan,
                        const cplx<T>* tw_plan, const cplx<T>* tw_L, cudaStream_t s);

template <typename T>
cudaError_t launch_strided(bool inverse, const void* in, void* out, long outer, int L, long inner,
                           const FftPlan& plan, const cplx<T>* tw, cudaStream_t s);

enum ChebMode { kChebScalar = 0, kChebBackward = 1, kChebForwardT = 2 };
template <typename T>
cudaError_t launch_cheb(int mode, int basis, bool real, const void* in, void* out, int N, long inner,
                        const FftPlan& plan, const cplx<T>* tw, const cplx<T>* dctw, cudaStream_t s,
                        bool wide = false);

// FP64 values per Chebyshev row per thread in the elimination scratch (k_solve.cu), for nc
// columns per thread.
int solve_scratch_values(int basis, int nc);
// compile-time-length transforms (k_fast_*.cu), for lengths with fast_compiled(L)
bool fast_compiled(int L);
template <typename T>
cudaError_t launch_rows_fast(int mode, const void* in, void* out, long nrows, int L, const cplx<T>* twf,
                             const cplx<T>* tw_L, cudaStream_t s);
template <typename T>
cudaError_t launch_strided_fast(bool inverse, const void* in, void* out, long outer, int L, long inner,
                                const cplx<T>* twf, cudaStream_t s);
template <typename T>
cudaError_t launch_cheb_fast(int mode, int basis, bool real, const void* in, void* out, int N, long inner,
                             const cplx<T>* twf, const cplx<T>* dctw, cudaStream_t s, bool wide);

// dense Chebyshev-axis contraction on the tensor cores (k_cheb_tc.cu), N <= 128: input and
// output are [N][ncols] real arrays (complex data as interleaved real columns); img is the
// device copy of tc_cheb_image(mode, basis, N)
template <typename TI, typename TO>
cudaError_t launch_cheb_tc(const void* in, void* out, long ncols, int N, const void* img, cudaStream_t s);
constexpr int kTcMaxN = 128;
int tc_pad16(int n);
// number of uint16 in the image is 2 * tc_pad16(N)^2
std::vector<uint16_t> tc_cheb_image(int mode, int basis, int N);
// the same image of any N x N matrix P (row-major, row = output row), N <= kTcMaxN
std::vector<uint16_t> tc_matrix_image(const std::vector<long double>& P, int N);
int tc_timeouts(bool reset);
int stream_timeouts(bool reset);   // k_stream.cu
int cnn_tc_timeouts(bool reset);   // k_cnn_tc.cu

template <typename T>
cudaError_t launch_solve(int basis, bool real, double a, double b, double c, const void* in, void* out,
                         int N, long ncols, const Wavenumbers& wn, const double* tab, double* scratch,
                         long scratch_threads, const int2* groups, long ngroups, cudaStream_t s);
// the same solve on FP64 spectral input (complex) with the solution rounded once to complex64
cudaError_t launch_solve_f64_to_f32(int basis, double a, double b, double c, const void* in, void* out, int N, long ncols,
                                    const Wavenumbers& wn, const double* tab, double* scratch, long scratch_threads,
                                    const int2* groups, long ngroups, cudaStream_t s);
// Factored eliminations of 3-D spaces (k_solve.cu): FP64 values per row and work thread of a
// factorisation table (0: the basis has none), work threads of the table for a call's column
// layout (0: a 1-D or 2-D space, no factored form), the work threads of the solve itself (one per
// column and parity; their scratch rows), the factorisation of the operator (a, b, c)
// into a table of rows x values x threads doubles, and the solve replaying a table (TI, TO:
// spectral input and output types; the table must come from launch_factor with the same basis, N,
// columns and wavenumbers; scratch_threads: threads the scratch holds 2 doubles per row for).
int solve_factor_values(int basis);
long solve_factor_threads(long ncols, const Wavenumbers& wn);
long solve_factored_scratch_threads(long ncols, const Wavenumbers& wn);   // threads of the solve
cudaError_t launch_factor(int basis, double a, double b, double c, int N, long ncols, const Wavenumbers& wn,
                          const double* tab, double* fact, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_solve_factored_to(int basis, bool real, const void* in, void* out, int N, long ncols,
                                     const Wavenumbers& wn, const double* tab, const double* fact, double* scratch,
                                     long scratch_threads, cudaStream_t s);

}  // namespace sgm
