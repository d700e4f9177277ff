// noalloc.cu - sgm_helmholtz_solve_noalloc: the Shen-Dirichlet Helmholtz solve without a
// space object and without any device allocation.
//
// Who needs it: callers that must not allocate device memory themselves.  Examples are
// programs whose device memory is owned by one memory manager (a framework's caching
// allocator, or a fixed budget that has claimed the HBM in advance), and latency-critical
// loops that cannot risk the time or the failure of a cudaMalloc.  sgm_space_create
// allocates tables, workspaces and elimination scratch, so such callers cannot use the
// space API for this step.
//
// How: the elimination scratch of k_solve_dirichlet (one FP64 record per row per thread)
// lives in a file-scope __device__ array of fixed size (kStaticScratchBytes).  Under CUDA's
// lazy module loading the array is reserved on a device when this module is first used there
// (the first call's address lookup), and it is then held until the process exits.  The
// Galerkin coefficients are evaluated inline from their closed forms instead of being
// read from a table, so no other device memory is needed.  Host code cannot use the
// array's name as a device address: on the first call on each device (with that device
// current) the entry point looks its address up with cudaGetSymbolAddress, checks the
// result and caches it per device; that first call must therefore come before any stream
// capture, and before a caller with a fixed memory budget claims the rest of the device.
// The cached address belongs to the device's primary context: after cudaDeviceReset the
// library must be reloaded before this entry point is called again.  Calls reuse the same array and it keeps the last call's contents; nothing in it
// needs clearing, because every value a thread reads back was written earlier by the same
// thread in the same call.  Calls whose kernels overlap on the GPU (for example on two
// streams) race on the array and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/sgm.h"
#include "common.cuh"

namespace sgm {
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr size_t kStaticScratchDoubles = kStaticScratchBytes / sizeof(double);
constexpr int kNoallocMaxN = 2048;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once per device).
int static_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(SGM_ERR_STATE, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(SGM_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SGM_OK;
}

__device__ __forceinline__ double rcp64_seeded(double x) {
  const float xf = (float)x;
  const float ax = fabsf(xf);
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Same elimination as k_solve_dirichlet (k_solve.cu), with the coefficients of row k taken
// from their closed forms: B_kk = pi/2 (c_k + 1), A_kk = -2 pi (k+1)(k+2), tail -4 pi (k+1).
template <typename T>
__global__ void __launch_bounds__(128) k_solve_dirichlet_static(const void* __restrict__ in, void* __restrict__ out,
                                                                int N, long ncols, int real, double a, double b,
                                                                const __grid_constant__ Wavenumbers wn,
                                                                double* __restrict__ scratch) {
  const double pi = 3.141592653589793;
  const long nth = (long)gridDim.x * blockDim.x;
  const long gt = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long ncb = (ncols + 31) / 32;
  const int nb = N - 2;
  for (long w = gt / 32; w < 2 * ncb; w += nth / 32) {
    const int p = (int)(w & 1);
    const long c = (w >> 1) * 32 + lane;
    if (c >= ncols) continue;
    const double k2 = kappa2_of(wn, c);
    const double aB = b - a * k2;
    const double ell = -aB * 0.5 * pi;
    const int n = (nb - p + 1) / 2;
    double pr = 0.0, pg = 0.0, pfx = 0.0, pfy = 0.0;
    for (int i = 0; i < n; ++i) {
      const int k = p + 2 * i;
      double fx, fy = 0.0;
      if (real) {
        fx = (double)reinterpret_cast<const T*>(in)[(long)k * ncols + c];
      } else {
        const cplx<T> v = reinterpret_cast<const cplx<T>*>(in)[(long)k * ncols + c];
        fx = (double)v.x;
        fy = (double)v.y;
      }
      const double kp1 = (double)(k + 1);
      double d = a * (-2.0 * pi * kp1 * (kp1 + 1.0)) + aB * (0.5 * pi * ((k == 0 ? 2.0 : 1.0) + 1.0));
      double g = a * (-4.0 * pi * kp1);
      if (i > 0) {
        const double mu = ell * pr;
        d = fma(-mu, pg + ell, d);
        g = fma(-mu, pg, g);
        fx = fma(-mu, pfx, fx);
        fy = fma(-mu, pfy, fy);
      }
      const double r = rcp64_seeded(d);
      double* s = scratch + (long)i * 4 * nth + gt;
      s[0] = r;
      s[nth] = g;
      s[2 * nth] = fx;
      s[3 * nth] = fy;
      pr = r; pg = g; pfx = fx; pfy = fy;
    }
    double ux = 0.0, uy = 0.0, tx = 0.0, ty = 0.0;
    for (int i = n - 1; i >= 0; --i) {
      const int k = p + 2 * i;
      const double* s = scratch + (long)i * 4 * nth + gt;
      const double r = s[0], g = s[nth];
      tx += ux;
      ty += uy;
      const double vx = (s[2 * nth] - ell * ux - g * tx) * r;
      const double vy = (s[3 * nth] - ell * uy - g * ty) * r;
      if (real) {
        reinterpret_cast<T*>(out)[(long)k * ncols + c] = (T)vx;
      } else {
        cplx<T> o; o.x = (T)vx; o.y = (T)vy;
        reinterpret_cast<cplx<T>*>(out)[(long)k * ncols + c] = o;
      }
      ux = vx;
      uy = vy;
    }
    for (int k = nb + p; k < N; k += 2) {
      if (real) {
        reinterpret_cast<T*>(out)[(long)k * ncols + c] = (T)0;
      } else {
        cplx<T> o; o.x = (T)0; o.y = (T)0;
        reinterpret_cast<cplx<T>*>(out)[(long)k * ncols + c] = o;
      }
    }
  }
}

}  // namespace
}  // namespace sgm

using namespace sgm;

extern "C" int sgm_helmholtz_solve_noalloc(int ndim, const int* kinds, const int64_t* n, const double* domain,
                                           int precision, double a, double b, const void* f_tilde, void* u_hat,
                                           void* stream) {
  if (!kinds || !n || !f_tilde || !u_hat) return set_error(SGM_ERR_NULL, "kinds, n, f_tilde and u_hat must be non-NULL");
  if (ndim < 1 || ndim > 3) return set_error(SGM_ERR_SIZE, "ndim must be 1..3 (got %d)", ndim);
  if (precision != SGM_F32 && precision != SGM_F64) return set_error(SGM_ERR_ARG, "precision must be SGM_F32 or SGM_F64");
  if (kinds[0] != SGM_SHEN_DIRICHLET) return set_error(SGM_ERR_STATE, "axis 0 must be SGM_SHEN_DIRICHLET");
  if (n[0] < 4 || n[0] > kNoallocMaxN)
    return set_error(SGM_ERR_SIZE, "N = %lld outside 4..%d, the largest size whose elimination scratch fits the "
                     "%zu-byte static array", (long long)n[0], kNoallocMaxN, kStaticScratchBytes);
  if (domain && (domain[0] != -1.0 || domain[1] != 1.0))
    return set_error(SGM_ERR_ARG, "the Chebyshev axis is defined on [-1, 1] only");
  for (int d = 1; d < ndim; ++d) {
    if (kinds[d] != SGM_FOURIER_C2C && kinds[d] != SGM_FOURIER_R2C)
      return set_error(SGM_ERR_SIZE, "axis %d must be a Fourier axis", d);
    if (kinds[d] == SGM_FOURIER_R2C && d != ndim - 1) return set_error(SGM_ERR_SIZE, "only the last axis may be R2C");
    if (n[d] < 1 || n[d] > 4096) return set_error(SGM_ERR_SIZE, "axis %d: size outside 1..4096", d);
    if (kinds[d] == SGM_FOURIER_R2C && n[d] < 2) return set_error(SGM_ERR_SIZE, "R2C axis needs M >= 2");
    if (domain && !(domain[2 * d + 1] > domain[2 * d])) return set_error(SGM_ERR_ARG, "axis %d: empty domain", d);
  }
  if (!std::isfinite(a) || !std::isfinite(b)) return set_error(SGM_ERR_ARG, "coefficients must be finite");
  if (a == 0.0 && b == 0.0) return set_error(SGM_ERR_ARG, "a = b = 0 gives a singular system");

  // spectral layout and wavenumbers, as for a space with these axes
  const int N = (int)n[0];
  int64_t spec[3] = {n[0], 1, 1};
  for (int d = 1; d < ndim; ++d) spec[d] = (kinds[d] == SGM_FOURIER_R2C) ? n[d] / 2 + 1 : n[d];
  const long ncols = (long)(spec[1] * spec[2]);
  const bool real = ndim == 1;
  const size_t elem = real ? (precision == SGM_F32 ? 4 : 8) : (precision == SGM_F32 ? 8 : 16);
  const size_t bytes = (size_t)N * ncols * elem;
  if (((uintptr_t)f_tilde & 15) || ((uintptr_t)u_hat & 15)) return set_error(SGM_ERR_ALIGN, "pointers must be 16-byte aligned");
  const char* pa = (const char*)f_tilde;
  const char* pb = (const char*)u_hat;
  if (pa != pb && pa < pb + bytes && pb < pa + bytes) return set_error(SGM_ERR_ALIAS, "f_tilde and u_hat overlap");

  Wavenumbers wn;
  wn.n1 = wn.n2 = wn.m1 = wn.m2 = 1;
  wn.r2c1 = wn.r2c2 = 0;
  wn.s1 = wn.s2 = 0.0;
  auto scale = [&](int d) {
    const double L = domain ? domain[2 * d + 1] - domain[2 * d] : 2.0 * 3.141592653589793;
    const double k = 2.0 * 3.141592653589793 / L;
    return k * k;
  };
  if (ndim == 2) {
    wn.n2 = (int)spec[1]; wn.m2 = (int)n[1]; wn.r2c2 = kinds[1] == SGM_FOURIER_R2C; wn.s2 = scale(1);
  } else if (ndim == 3) {
    wn.n1 = (int)spec[1]; wn.m1 = (int)n[1]; wn.s1 = scale(1);
    wn.n2 = (int)spec[2]; wn.m2 = (int)n[2]; wn.r2c2 = kinds[2] == SGM_FOURIER_R2C; wn.s2 = scale(2);
  }

  double* scratch = nullptr;
  int st = static_scratch(&scratch);
  if (st != SGM_OK) return st;

  // threads: as many 128-thread blocks as the static scratch holds (4 doubles per row per
  // thread, N/2 + 1 rows per parity), and no more than there are (column, parity) warps.
  const long rows = N / 2 + 1;
  long cap = (long)(kStaticScratchDoubles / (size_t)(rows * 4));
  cap = (cap / 128) * 128;
  long need = 2 * ((ncols + 31) / 32) * 32;
  need = ((need + 127) / 128) * 128;
  const long threads = std::min(cap, need);
  if (threads < 128) return set_error(SGM_ERR_SIZE, "static scratch too small for N = %d", N);
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)(threads / 128);
  if (precision == SGM_F32)
    k_solve_dirichlet_static<float><<<grid, 128, 0, s>>>(f_tilde, u_hat, N, ncols, real ? 1 : 0, a, b, wn, scratch);
  else
    k_solve_dirichlet_static<double><<<grid, 128, 0, s>>>(f_tilde, u_hat, N, ncols, real ? 1 : 0, a, b, wn, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}
