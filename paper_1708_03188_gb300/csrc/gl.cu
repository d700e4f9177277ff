// gl.cu - host side of the Ginzburg-Landau stepper (Sec. 6 of the paper): object, tables and
// the C ABI entry points sgm_gl_*.  Kernels in k_gl.cuh.
#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "k_gl.cuh"
#include "space_internal.cuh"

using namespace sgm;

struct sgm_gl {
  static constexpr uint32_t kMagic = 0x53474c31u;
  uint32_t magic = kMagic;
  int device = 0;
  int M = 0, MP = 0;
  int prec = SGM_F64;
  int scheme = SGM_GL_RK4;
  double beta = 0, gamma = 0, dt = 0, length = 0;
  void* P = nullptr;    // M x MP workspace (padded rows)
  void* V = nullptr;    // stage input
  void* A = nullptr;    // RK4 accumulator
  void* E = nullptr;    // exp(L(k) dt / 2), integrating-factor scheme only
  void* twf = nullptr;  // pass tables for length MP
};

namespace {

void free_gl(sgm_gl* g) {
  cudaFree(g->P);
  cudaFree(g->V);
  cudaFree(g->A);
  cudaFree(g->E);
  cudaFree(g->twf);
  g->magic = 0;
  delete g;
}

int check_gl(const sgm_gl* g) {
  if (!g) return set_error(SGM_ERR_NULL, "gl is NULL");
  if (g->magic != sgm_gl::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_gl");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
    return set_error(SGM_ERR_STATE, "stepper was created on device %d, current device is %d", g->device, dev);
  return SGM_OK;
}

template <typename T> int upload_E(sgm_gl* g) {
  const int M = g->M;
  std::vector<cplx<T>> h((size_t)M * M);
  const long double ks = 2.0L * 3.141592653589793238462643383279502884L / g->length;
  for (int r = 0; r < M; ++r)
    for (int j = 0; j < M; ++j) {
      const long double lr = r < (M + 1) / 2 ? r : r - M, lj = j < (M + 1) / 2 ? j : j - M;
      const long double k2 = ks * ks * (lr * lr + lj * lj);
      const long double h2 = 0.5L * g->dt;
      const long double mag = expl(h2 * (1.0L - k2)), ph = -h2 * g->beta * k2;
      h[(size_t)r * M + j].x = (T)(mag * cosl(ph));
      h[(size_t)r * M + j].y = (T)(mag * sinl(ph));
    }
  cudaError_t e = cudaMalloc(&g->E, sizeof(cplx<T>) * h.size());
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  e = cudaMemcpy(g->E, h.data(), sizeof(cplx<T>) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
  return SGM_OK;
}

template <typename T> int launch(sgm_gl* g, int mode, bool pad_first, bool pad_next, const void* Vin, void* Vout,
                                 void* S, void* out, int stage, cudaStream_t st) {
  GlParams prm;
  prm.beta = g->beta;
  prm.gamma = g->gamma;
  prm.dt = g->dt;
  prm.kscale = 2.0 * 3.141592653589793 / g->length;
  prm.stage = stage;
  cudaError_t e = gl_launch<T>(g->M, mode, pad_first, pad_next, (const cplx<T>*)Vin, (cplx<T>*)Vout, (cplx<T>*)g->A, (cplx<T>*)S,
                               (const cplx<T>*)g->E, (cplx<T>*)out, (cplx<T>*)g->P, prm, (const cplx<T>*)g->twf, st);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "Ginzburg-Landau launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

template <typename T> int step_impl(sgm_gl* g, void* u, int nsteps, cudaStream_t st) {
  const int mode = g->scheme == SGM_GL_IFRK4 ? kGlIfRk4 : kGlRk4;
  // one run of 4 * nsteps stages: only the first pads its input itself; every stage but the last
  // leaves the padded, back-transformed input of the next stage in P
  const long total = 4L * nsteps;
  long i = 0;
  for (int n = 0; n < nsteps; ++n)
    for (int s = 0; s < 4; ++s, ++i) {
      int r = launch<T>(g, mode, i == 0, i + 1 < total, s == 0 ? u : g->V, g->V, u, nullptr, s, st);
      if (r != SGM_OK) return r;
    }
  return SGM_OK;
}

}  // namespace

extern "C" {

int sgm_gl_create(sgm_gl** out, const sgm_space* space, double padding, double beta, double gamma, double dt,
                  int scheme) {
  if (!out) return set_error(SGM_ERR_NULL, "out is NULL");
  *out = nullptr;
  int st = space_check(space);
  if (st != SGM_OK) return st;
  if (space->ndim != 2 || space->kinds[0] != SGM_FOURIER_C2C || space->kinds[1] != SGM_FOURIER_C2C)
    return set_error(SGM_ERR_SIZE, "the Ginzburg-Landau stepper needs a 2-D C2C x C2C space");
  const int M = (int)space->n[0];
  const double L0 = space->dom[1] - space->dom[0], L1 = space->dom[3] - space->dom[2];
  if (space->n[1] != M || !(std::fabs(L0 - L1) <= 1e-12 * std::fabs(L0)))
    return set_error(SGM_ERR_SIZE, "the stepper needs a square grid on a square domain");
  if (!(M == 32 || M == 64 || M == 128 || M == 256 || M == 512 || M == 1024))
    return set_error(SGM_ERR_SIZE, "grid size %d not supported (32, 64, ..., 1024)", M);
  if (padding != 1.5) return set_error(SGM_ERR_ARG, "padding factor must be 1.5 (the 3/2 rule)");
  if (!std::isfinite(beta) || !std::isfinite(gamma) || !(dt > 0.0) || !std::isfinite(dt))
    return set_error(SGM_ERR_ARG, "beta, gamma must be finite and dt > 0");
  if (scheme != SGM_GL_RK4 && scheme != SGM_GL_IFRK4) return set_error(SGM_ERR_ARG, "unknown scheme %d", scheme);
  sgm_gl* g = new (std::nothrow) sgm_gl;
  if (!g) return set_error(SGM_ERR_ALLOC, "host allocation failed");
  g->device = space->device;
  g->M = M;
  g->MP = 3 * M / 2;
  g->prec = space->prec;
  g->scheme = scheme;
  g->beta = beta;
  g->gamma = gamma;
  g->dt = dt;
  g->length = L0;
  const size_t ce = g->prec == SGM_F32 ? 8 : 16;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&g->P, ce * (size_t)M * g->MP);
  if (e == cudaSuccess) e = cudaMalloc(&g->V, ce * (size_t)M * M);
  if (e == cudaSuccess) e = cudaMalloc(&g->A, ce * (size_t)M * M);
  if (e != cudaSuccess) {
    free_gl(g);
    return set_error(SGM_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
  }
  st = make_fast_twiddles(g->prec, g->MP, &g->twf);
  if (st == SGM_OK && scheme == SGM_GL_IFRK4) st = g->prec == SGM_F32 ? upload_E<float>(g) : upload_E<double>(g);
  if (st != SGM_OK) {
    free_gl(g);
    return st;
  }
  *out = g;
  return SGM_OK;
}

int sgm_gl_destroy(sgm_gl* gl) {
  if (!gl) return SGM_OK;
  if (gl->magic != sgm_gl::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_gl");
  free_gl(gl);
  return SGM_OK;
}

int sgm_gl_rhs(sgm_gl* gl, const void* u_hat, void* rhs, void* stream) {
  int st = check_gl(gl);
  if (st != SGM_OK) return st;
  if (!u_hat || !rhs) return set_error(SGM_ERR_NULL, "NULL data pointer");
  const size_t bytes = (gl->prec == SGM_F32 ? 8 : 16) * (size_t)gl->M * gl->M;
  const char* a = (const char*)u_hat;
  const char* b = (const char*)rhs;
  if (a < b + bytes && b < a + bytes) return set_error(SGM_ERR_ALIAS, "u_hat and rhs overlap");
  cudaStream_t s = (cudaStream_t)stream;
  return gl->prec == SGM_F32 ? launch<float>(gl, kGlRhs, true, false, u_hat, nullptr, nullptr, rhs, 0, s)
                             : launch<double>(gl, kGlRhs, true, false, u_hat, nullptr, nullptr, rhs, 0, s);
}

int sgm_gl_step(sgm_gl* gl, void* u_hat, int nsteps, void* stream) {
  int st = check_gl(gl);
  if (st != SGM_OK) return st;
  if (!u_hat) return set_error(SGM_ERR_NULL, "NULL data pointer");
  if (nsteps < 0) return set_error(SGM_ERR_ARG, "nsteps must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  return gl->prec == SGM_F32 ? step_impl<float>(gl, u_hat, nsteps, s) : step_impl<double>(gl, u_hat, nsteps, s);
}

}  // extern "C"
