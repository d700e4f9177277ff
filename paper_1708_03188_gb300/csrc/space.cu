// space.cu - host side of libsgm: the tensor-product space object, its device tables
// (FFT twiddles, DCT twiddles, Galerkin coefficient tables), workspaces, and the C ABI
// entry points declared in include/sgm.h.
//
// Pipelines (Sec. 4 of the paper, transform order: Fourier axes first on the way in):
//   scalar product  rows(R2C|C2C fwd, last axis) -> strided C2C (middle axis, in place)
//                   -> Chebyshev DCT-II + stencil (axis 0)
//   forward         scalar product -> FP64 mass-matrix elimination (in place)
//   backward        stencil + DCT-III (axis 0) -> strided inverse C2C -> rows (C2R|C2C inv)
//   solve           FP64 elimination per Fourier column (k_solve.cu)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "fft_fast.cuh"
#include "space_internal.cuh"

using namespace sgm;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define SGM_CU(call)                                                                       \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(SGM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define SGM_TRY(expr)            \
  do {                           \
    int st_ = (expr);            \
    if (st_ != SGM_OK) return st_; \
  } while (0)

const long double kPi = 3.141592653589793238462643383279502884L;

FftPlan make_plan(int L) {
  FftPlan p;
  memset(&p, 0, sizeof p);
  p.L = L;
  int m = L;
  auto push = [&](int r) { p.radix[p.npass++] = r; m /= r; };
  while (m % 8 == 0 && p.npass < kMaxPasses) push(8);
  if (m % 4 == 0) push(4);
  if (m % 2 == 0) push(2);
  while (m % 3 == 0) push(3);
  while (m % 5 == 0) push(5);
  for (int q = 7; m > 1; q += 2)
    while (m % q == 0) push(q);
  return p;
}

}  // namespace

FftPlan sgm::host_plan(int L) { return make_plan(L); }

int sgm::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}


namespace {

template <typename T> int upload_twiddles(sgm_space* s, int L, void** out) {
  std::vector<cplx<T>> h(L);
  for (int k = 0; k < L; ++k) {
    long double a = -2.0L * kPi * (long double)k / (long double)L;
    h[k].x = (T)cosl(a);
    h[k].y = (T)sinl(a);
  }
  SGM_CU(cudaMalloc(out, sizeof(cplx<T>) * L));
  SGM_CU(cudaMemcpy(*out, h.data(), sizeof(cplx<T>) * L, cudaMemcpyHostToDevice));
  return SGM_OK;
}

int need_tw(sgm_space* s, int L) {
  if (s->tw.count(L)) return SGM_OK;
  void* p = nullptr;
  int st = s->prec == SGM_F32 ? upload_twiddles<float>(s, L, &p) : upload_twiddles<double>(s, L, &p);
  if (st != SGM_OK) return st;
  s->tw[L] = p;
  return SGM_OK;
}

template <typename T> int upload_fast_twiddles(int L, void** out) {
  std::vector<cplx<T>> h(fast_table_size(L));
  fill_fast_table(L, h.data(), [&](long j) {
    const long double a = -2.0L * kPi * (long double)j / (long double)L;
    cplx<T> w;
    w.x = (T)cosl(a);
    w.y = (T)sinl(a);
    return w;
  });
  SGM_CU(cudaMalloc(out, sizeof(cplx<T>) * h.size()));
  SGM_CU(cudaMemcpy(*out, h.data(), sizeof(cplx<T>) * h.size(), cudaMemcpyHostToDevice));
  return SGM_OK;
}

}  // namespace

int sgm::make_fast_twiddles(int precision, int L, void** out) {
  return precision == SGM_F32 ? upload_fast_twiddles<float>(L, out) : upload_fast_twiddles<double>(L, out);
}

// pass tables for the compile-time engine when L has a compiled kernel (else nullptr)
int sgm::need_twf(sgm_space* s, int L, const void** out) {
  *out = nullptr;
  if (!fast_compiled(L)) return SGM_OK;
  if (!s->twf.count(L)) {
    void* p = nullptr;
    int st = s->prec == SGM_F32 ? upload_fast_twiddles<float>(L, &p) : upload_fast_twiddles<double>(L, &p);
    if (st != SGM_OK) return st;
    s->twf[L] = p;
  }
  *out = s->twf[L];
  return SGM_OK;
}

namespace {

template <typename T> int upload_dctw(sgm_space* s, int N) {
  std::vector<cplx<T>> h(N);
  for (int k = 0; k < N; ++k) {
    long double a = -kPi * (long double)k / (2.0L * N);
    h[k].x = (T)cosl(a);
    h[k].y = (T)sinl(a);
  }
  SGM_CU(cudaMalloc(&s->dctw, sizeof(cplx<T>) * N));
  SGM_CU(cudaMemcpy(s->dctw, h.data(), sizeof(cplx<T>) * N, cudaMemcpyHostToDevice));
  return SGM_OK;
}

// Galerkin coefficient tables, closed forms evaluated in long double.
//   (T_a, T_b)_w = pi/2 c_a delta_ab;   (T_a'', T_b)_w = pi/2 a (a^2 - b^2), b < a, same parity;
//   (T_a'''', T_b)_w = pi/2 a/24 [a^2 (a^2-4)^2 - 3 a^4 b^2 + 3 a^2 b^4 - b^2 (b^2-4)^2], b <= a-4.
long double d2(int a, int b) {
  if (b < a && ((a - b) & 1) == 0) return 0.5L * kPi * a * ((long double)a * a - (long double)b * b);
  return 0.0L;
}
long double d4(int a, int b) {
  if (b <= a - 4 && ((a - b) & 1) == 0) {
    long double A = a, B = b;
    long double P = A * A * (A * A - 4) * (A * A - 4) - 3 * A * A * A * A * B * B + 3 * A * A * B * B * B * B -
                    B * B * (B * B - 4) * (B * B - 4);
    return 0.5L * kPi * A / 24.0L * P;
  }
  return 0.0L;
}
struct Term { int idx; long double c; };
void bih_terms(int k, Term t[3]) {
  t[0] = {k, 1.0L};
  t[1] = {k + 2, -2.0L * (k + 2) / (k + 3)};
  t[2] = {k + 4, (long double)(k + 1) / (k + 3)};
}

int build_tables(sgm_space* s) {
  const int N = (int)s->n[0];
  const int ts = N + 8;
  std::vector<double> h;
  if (s->kinds[0] == SGM_SHEN_NEUMANN) {
    // TN_B0, TN_BUP, TN_A0, TN_G of k_solve_neumann (k_solve.cu)
    h.assign(4 * ts, 0.0);
    for (int k = 0; k < N - 2; ++k) {
      const long double q = ((long double)k / (k + 2)) * ((long double)k / (k + 2));
      h[0 * ts + k] = (double)(0.5L * kPi * ((k == 0 ? 2 : 1) + q * q));
      h[1 * ts + k] = (double)(-0.5L * kPi * q);
      h[2 * ts + k] = (double)(-2.0L * kPi * k * k * (k + 1) / (k + 2));
      h[3 * ts + k] = (double)(-4.0L * kPi * (k + 1) / ((long double)(k + 2) * (k + 2)));
    }
  } else if (s->kinds[0] == SGM_SHEN_DIRICHLET) {
    h.assign(3 * ts, 0.0);
    for (int k = 0; k < N - 2; ++k) {
      h[0 * ts + k] = (double)(0.5L * kPi * ((k == 0 ? 2 : 1) + 1));
      h[1 * ts + k] = (double)(-2.0L * kPi * (k + 1) * (k + 2));
      h[2 * ts + k] = (double)(-4.0L * kPi * (k + 1));
    }
  } else if (s->kinds[0] == SGM_SHEN_BIHARMONIC) {
    enum { B0, B2, B4, ALO, A0, AUP, S0, S1, S2, G0, G1, F0, F1, COUNT };
    h.assign(COUNT * ts, 0.0);
    const int nb = N - 4;
    auto pair = [&](int m, int l, long double (*f)(int, int)) {
      Term tm[3], tl[3];
      bih_terms(m, tm);
      bih_terms(l, tl);
      long double acc = 0;
      for (auto& x : tl)
        for (auto& y : tm) acc += x.c * y.c * f(x.idx, y.idx);
      return acc;
    };
    for (int k = 0; k < nb; ++k) {
      Term t[3];
      bih_terms(k, t);
      const long double ck = (k == 0) ? 2 : 1;
      const long double be = t[1].c, ga = t[2].c;
      const long double be2 = -2.0L * (k + 4) / (k + 5);
      h[B0 * ts + k] = (double)(0.5L * kPi * (ck + be * be + ga * ga));
      h[B2 * ts + k] = (double)(0.5L * kPi * (be + ga * be2));
      h[B4 * ts + k] = (double)(0.5L * kPi * ga);
      h[A0 * ts + k] = (double)pair(k, k, d2);
      h[AUP * ts + k] = (double)pair(k, k + 2, d2);
      h[ALO * ts + k] = k >= 2 ? (double)pair(k, k - 2, d2) : 0.0;
      h[S0 * ts + k] = (double)pair(k, k, d4);
      h[S1 * ts + k] = (double)pair(k, k + 2, d4);
      h[S2 * ts + k] = (double)pair(k, k + 4, d4);
      long double g0 = 0, g1 = 0, f0 = 0, f1 = 0;
      for (auto& x : t) {
        long double b2 = (long double)x.idx * x.idx;
        g0 += x.c * b2 * b2;
        g1 += x.c * b2 * b2 * b2;
        f0 += x.c * x.idx / 24.0L * (3 * b2 + 8);
        f1 += x.c * x.idx / 24.0L * (-1.0L);
      }
      h[G0 * ts + k] = (double)g0;
      h[G1 * ts + k] = (double)g1;
      h[F0 * ts + k] = (double)(0.5L * kPi * f0);
      h[F1 * ts + k] = (double)(0.5L * kPi * f1);
    }
  } else {
    return SGM_OK;
  }
  SGM_CU(cudaMalloc(&s->tab, sizeof(double) * h.size()));
  SGM_CU(cudaMemcpy(s->tab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
  return SGM_OK;
}

int check_space(const sgm_space* s) {
  if (!s) return fail(SGM_ERR_NULL, "space is NULL");
  if (s->magic != sgm_space::kMagic) return fail(SGM_ERR_STATE, "not a live sgm_space");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device)
    return fail(SGM_ERR_STATE, "space was created on device %d, current device is %d", s->device, dev);
  return SGM_OK;
}

int check_ptrs(const void* in, size_t in_bytes, const void* out, size_t out_bytes, bool allow_same) {
  if (!in || !out) return fail(SGM_ERR_NULL, "NULL data pointer");
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return fail(SGM_ERR_ALIGN, "data pointers must be 16-byte aligned");
  const char* a = (const char*)in;
  const char* b = (const char*)out;
  if (allow_same && a == b) return SGM_OK;
  if (a < b + out_bytes && b < a + in_bytes) return fail(SGM_ERR_ALIAS, "input and output overlap");
  return SGM_OK;
}

int wrap(cudaError_t e, const char* what) {
  if (e != cudaSuccess) return fail(SGM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return SGM_OK;
}

int first_fourier(const sgm_space* s) { return s->cheb ? 1 : 0; }

// Fourier forward on axes first_fourier..ndim-1: in (physical) -> out (complex).
template <typename T> int fourier_forward(sgm_space* s, const void* in, void* out, cudaStream_t st) {
  const int d = s->ndim - 1;
  const int L = (int)s->n[d];
  long nrows = 1;
  for (int i = 0; i < d; ++i) nrows *= s->n[i];
  const bool r2c = s->kinds[d] == SGM_FOURIER_R2C;
  const int fl = (r2c && L % 2 == 0) ? L / 2 : L;
  FftPlan p = make_plan(fl);
  SGM_TRY(need_tw(s, fl));
  SGM_TRY(need_tw(s, L));
  const void* twf = nullptr;
  SGM_TRY(need_twf(s, fl, &twf));
  const int mode = r2c ? kRowR2C : kRowC2CFwd;
  if (twf && (!r2c || L % 2 == 0))
    SGM_TRY(wrap(launch_rows_fast<T>(mode, in, out, nrows, L, (const cplx<T>*)twf, (const cplx<T>*)s->tw[L], st),
                 "rows forward"));
  else
    SGM_TRY(wrap(launch_rows<T>(mode, in, out, nrows, L, p, (const cplx<T>*)s->tw[fl], (const cplx<T>*)s->tw[L], st),
                 "rows forward"));
  for (int a = d - 1; a >= first_fourier(s); --a) {
    long outer = 1, inner = 1;
    for (int i = 0; i < a; ++i) outer *= s->spec[i];
    for (int i = a + 1; i < s->ndim; ++i) inner *= s->spec[i];
    const int La = (int)s->n[a];
    FftPlan pa = make_plan(La);
    SGM_TRY(need_tw(s, La));
    const void* twf = nullptr;
    SGM_TRY(need_twf(s, La, &twf));
    if (twf)
      SGM_TRY(wrap(launch_strided_fast<T>(false, out, out, outer, La, inner, (const cplx<T>*)twf, st), "strided forward"));
    else
      SGM_TRY(wrap(launch_strided<T>(false, out, out, outer, La, inner, pa, (const cplx<T>*)s->tw[La], st),
                   "strided forward"));
  }
  return SGM_OK;
}

// Fourier backward: in (complex spectral-like) -> out (physical).  `in` is read only if
// at most one Fourier axis exists, or copied through W1 otherwise (W1 may equal in).
template <typename T> int fourier_backward(sgm_space* s, const void* in, void* out, cudaStream_t st) {
  const int d = s->ndim - 1;
  const void* cur = in;
  for (int a = first_fourier(s); a < d; ++a) {
    long outer = 1, inner = 1;
    for (int i = 0; i < a; ++i) outer *= s->spec[i];
    for (int i = a + 1; i < s->ndim; ++i) inner *= s->spec[i];
    const int La = (int)s->n[a];
    FftPlan pa = make_plan(La);
    SGM_TRY(need_tw(s, La));
    const void* twf = nullptr;
    SGM_TRY(need_twf(s, La, &twf));
    if (twf)
      SGM_TRY(wrap(launch_strided_fast<T>(true, cur, s->W1, outer, La, inner, (const cplx<T>*)twf, st),
                   "strided backward"));
    else
      SGM_TRY(wrap(launch_strided<T>(true, cur, s->W1, outer, La, inner, pa, (const cplx<T>*)s->tw[La], st),
                   "strided backward"));
    cur = s->W1;
  }
  const int L = (int)s->n[d];
  long nrows = 1;
  for (int i = 0; i < d; ++i) nrows *= s->n[i];
  const bool r2c = s->kinds[d] == SGM_FOURIER_R2C;
  const int fl = (r2c && L % 2 == 0) ? L / 2 : L;
  FftPlan p = make_plan(fl);
  SGM_TRY(need_tw(s, fl));
  SGM_TRY(need_tw(s, L));
  const void* twf = nullptr;
  SGM_TRY(need_twf(s, fl, &twf));
  const int mode = r2c ? kRowC2R : kRowC2CInv;
  if (twf && (!r2c || L % 2 == 0))
    return wrap(launch_rows_fast<T>(mode, cur, out, nrows, L, (const cplx<T>*)twf, (const cplx<T>*)s->tw[L], st),
                "rows backward");
  return wrap(launch_rows<T>(mode, cur, out, nrows, L, p, (const cplx<T>*)s->tw[fl], (const cplx<T>*)s->tw[L], st),
              "rows backward");
}

// the Chebyshev-axis pass as the dense tensor-core contraction (FP32 spaces)
int cheb_pass_tc(sgm_space* s, int mode, const void* in, void* out, cudaStream_t st, bool wide) {
  const int N = (int)s->n[0];
  long ncols = s->real_spec ? 1 : 2;
  for (int i = 1; i < s->ndim; ++i) ncols *= s->spec[i];
  const void* img = s->tc_img[mode];
  cudaError_t e;
  if (mode == kChebBackward)
    e = wide ? launch_cheb_tc<double, float>(in, out, ncols, N, img, st)
             : launch_cheb_tc<float, float>(in, out, ncols, N, img, st);
  else
    e = wide ? launch_cheb_tc<float, double>(in, out, ncols, N, img, st)
             : launch_cheb_tc<float, float>(in, out, ncols, N, img, st);
  return wrap(e, "chebyshev contraction");
}

template <typename T>
int cheb_pass(sgm_space* s, int mode, const void* in, void* out, cudaStream_t st, bool wide = false) {
  const int N = (int)s->n[0];
  if (sizeof(T) == 4 && s->cheb_tc) return cheb_pass_tc(s, mode, in, out, st, wide);
  if (s->legendre) return legendre_pass(s, mode, in, out, st, wide);
  long inner = 1;
  for (int i = 1; i < s->ndim; ++i) inner *= s->spec[i];
  FftPlan p = make_plan(N);
  SGM_TRY(need_tw(s, N));
  const void* twf = nullptr;
  SGM_TRY(need_twf(s, N, &twf));
  if (twf)
    return wrap(launch_cheb_fast<T>(mode, s->kinds[0], s->real_spec, in, out, N, inner, (const cplx<T>*)twf,
                                    (const cplx<T>*)s->dctw, st, wide),
                "chebyshev pass");
  return wrap(launch_cheb<T>(mode, s->kinds[0], s->real_spec, in, out, N, inner, p, (const cplx<T>*)s->tw[N],
                             (const cplx<T>*)s->dctw, st, wide),
              "chebyshev pass");
}

Wavenumbers wavenumbers(const sgm_space* s) {
  Wavenumbers w;
  memset(&w, 0, sizeof w);
  w.n1 = w.n2 = 1;
  w.m1 = w.m2 = 1;
  auto scale = [&](int ax) {
    double L = s->dom[2 * ax + 1] - s->dom[2 * ax];
    double k = 2.0 * 3.14159265358979323846 / L;
    return k * k;
  };
  if (s->ndim == 2) {
    w.n2 = (int)s->spec[1];
    w.m2 = (int)s->n[1];
    w.r2c2 = s->kinds[1] == SGM_FOURIER_R2C;
    w.s2 = scale(1);
  } else if (s->ndim == 3) {
    w.n1 = (int)s->spec[1];
    w.m1 = (int)s->n[1];
    w.r2c1 = 0;
    w.s1 = scale(1);
    w.n2 = (int)s->spec[2];
    w.m2 = (int)s->n[2];
    w.r2c2 = s->kinds[2] == SGM_FOURIER_R2C;
    w.s2 = scale(2);
  }
  return w;
}

bool stream_capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// The elimination of one solve call (TI, TO: spectral input and output types).  Spaces with
// factorisation slots (3-D Dirichlet and biharmonic) replay, one thread per column and parity, a
// stored factorisation of the operator
// (a, b, c), computing it first into the least recently used slot when neither slot holds it for
// this column layout; the factorisation kernel then runs on the caller's stream ahead of the
// solve, so stream order keeps the slot consistent for every later call on that space.  Inside a
// stream capture the self-contained kernels run instead, so that a captured graph never depends
// on slot contents that later calls may replace.
template <typename TI, typename TO>
int eliminate(sgm_space* s, int basis, double a, double b, double c, const void* in, void* out, long ncols,
              const Wavenumbers& wn, cudaStream_t st) {
  const int N = (int)s->n[0];
  if (s->fact[0] && s->fact[1] && solve_factor_values(basis) > 0 && !stream_capturing(st) &&
      solve_factor_threads(ncols, wn) <= s->fact_threads) {
    const double key[5] = {(double)basis, a, b, c, (double)wn.n2};
    int slot = -1;
    for (int i = 0; i < 2; ++i)
      if (s->fact_valid[i] && std::memcmp(key, s->fact_key[i], sizeof key) == 0) slot = i;
    if (slot < 0) {
      slot = !s->fact_valid[0] ? 0 : !s->fact_valid[1] ? 1 : s->fact_use[0] <= s->fact_use[1] ? 0 : 1;
      s->fact_valid[slot] = false;
      SGM_TRY(wrap(launch_factor(basis, a, b, c, N, ncols, wn, s->tab, s->fact[slot], st), "factorisation"));
      std::memcpy(s->fact_key[slot], key, sizeof key);
      s->fact_valid[slot] = true;
    }
    s->fact_use[slot] = ++s->fact_clock;
    return wrap(launch_solve_factored_to<TI, TO>(basis, s->real_spec, in, out, N, ncols, wn, s->tab, s->fact[slot],
                                                 s->scratch, s->fact_scratch_threads, st),
                "solve");
  }
  if constexpr (std::is_same<TI, TO>::value)
    return wrap(launch_solve<TI>(basis, s->real_spec, a, b, c, in, out, N, ncols, wn, s->tab, s->scratch,
                                 s->scratch_threads, s->groups, s->ngroups, st),
                "solve");
  else
    return wrap(launch_solve_f64_to_f32(basis, a, b, c, in, out, N, ncols, wn, s->tab, s->scratch,
                                        s->scratch_threads, s->groups, s->ngroups, st),
                "solve");
}

template <typename T>
int solve_impl(sgm_space* s, int basis, double a, double b, double c, const void* in, void* out, cudaStream_t st) {
  // the Legendre kernel takes the biharmonic form a S + (b - 2 a k2) A + (a k2^2 - b k2 + c) B;
  // a lap(u) + b u is that form with (0, a, b)
  if (s->legendre)
    return basis == kDirichlet ? legendre_solve<T>(s, 0.0, a, b, in, out, wavenumbers(s), st)
                               : legendre_solve<T>(s, a, b, c, in, out, wavenumbers(s), st);
  long ncols = 1;
  for (int i = 1; i < s->ndim; ++i) ncols *= s->spec[i];
  if (s->kinds[0] == SGM_SHEN_NEUMANN) basis = kNeumann;
  return eliminate<T, T>(s, basis, a, b, c, in, out, ncols, wavenumbers(s), st);
}

// wide: write the spectral result in FP64 (FP32 spaces, internal intermediates only)
template <typename T>
int scalar_impl(sgm_space* s, const void* f, void* out, cudaStream_t st, int mode, bool wide = false) {
  if (!s->cheb) return fourier_forward<T>(s, f, out, st);
  if (s->ndim == 1) return cheb_pass<T>(s, mode, f, out, st, wide);
  SGM_TRY(fourier_forward<T>(s, f, s->W1, st));
  return cheb_pass<T>(s, mode, s->W1, out, st, wide);
}

template <typename T> int forward_impl(sgm_space* s, const void* u, void* out, cudaStream_t st) {
  if (!s->cheb) return fourier_forward<T>(s, u, out, st);
  const int basis = s->kinds[0];
  if (basis == SGM_CHEBYSHEV || basis == SGM_LEGENDRE) return scalar_impl<T>(s, u, out, st, kChebForwardT);
  SGM_TRY(scalar_impl<T>(s, u, out, st, kChebScalar));
  if (basis == SGM_SHEN_DIRICHLET || basis == SGM_LEGENDRE_DIRICHLET || basis == SGM_SHEN_NEUMANN)
    return solve_impl<T>(s, kDirichlet, 0.0, 1.0, 0.0, out, out, st);
  return solve_impl<T>(s, kBiharmonic, 0.0, 0.0, 1.0, out, out, st);
}

// wide: the spectral input is FP64 (FP32 spaces, internal intermediates only)
template <typename T> int backward_impl(sgm_space* s, const void* uh, void* u, cudaStream_t st, bool wide = false) {
  if (!s->cheb) return fourier_backward<T>(s, uh, u, st);
  if (s->ndim == 1) return cheb_pass<T>(s, kChebBackward, uh, u, st, wide);
  SGM_TRY(cheb_pass<T>(s, kChebBackward, uh, s->W1, st, wide));
  return fourier_backward<T>(s, s->W1, u, st);
}

}  // namespace

int sgm::space_check(const sgm_space* s) { return check_space(s); }

// The mass solve of the forward transform (a = 0 systems) on FP64 spectral data of any space
// with a Shen basis on axis 0, in place: B u = data.
int sgm::space_mass_solve_f64(sgm_space* s, void* data, cudaStream_t st) {
  const int k = s->kinds[0];
  if (k == SGM_SHEN_DIRICHLET || k == SGM_LEGENDRE_DIRICHLET || k == SGM_SHEN_NEUMANN)
    return solve_impl<double>(s, kDirichlet, 0.0, 1.0, 0.0, data, data, st);
  return solve_impl<double>(s, kBiharmonic, 0.0, 0.0, 1.0, data, data, st);
}

namespace {

void free_space(sgm_space* s) {
  if (s->inner) {
    sgm_space_destroy(s->inner);
    cudaFree(s->P1);
    cudaFree(s->P2);
    s->magic = 0;
    delete s;
    return;
  }
  for (auto& kv : s->tw) cudaFree(kv.second);
  s->tw.clear();
  for (auto& kv : s->twf) cudaFree(kv.second);
  s->twf.clear();
  cudaFree(s->dctw);
  cudaFree(s->tab);
  cudaFree(s->W1);
  cudaFree(s->W2);
  cudaFree(s->scratch);
  cudaFree(s->fact[0]);
  cudaFree(s->fact[1]);
  cudaFree(s->groups);
  for (void* p : s->tc_img) cudaFree(p);
  cudaFree(s->pdx_tab);
  for (void* p : s->leg_mat) cudaFree(p);
  cudaFree(s->leg_band);
  cudaFree(s->leg_scratch);
  s->magic = 0;
  delete s;
}

// time the scalar product and backward passes of both Chebyshev-axis methods on this space's
// workspaces (the pair that the physical-to-physical solves run), keep the faster method;
// returns 1 (contraction), 0 (FFT) or -1 (CUDA error, message set)
int autotune_cheb(sgm_space* s) {
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int result = -1;
  float best[2] = {0, 0};
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    fail(SGM_ERR_CUDA, "autotune: stream or event creation failed");
    goto done;
  }
  if (cudaMemsetAsync(s->W1, 0, (size_t)s->nspec * s->celem(), st) != cudaSuccess ||
      cudaMemsetAsync(s->W2, 0, (size_t)s->nspec * 16, st) != cudaSuccess) {
    fail(SGM_ERR_CUDA, "autotune: workspace clear failed");
    goto done;
  }
  for (int m = 0; m < 2; ++m) {
    s->cheb_tc = m;
    best[m] = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) goto cuda_fail;
      if (cheb_pass<float>(s, kChebScalar, s->W1, s->W2, st, true) != SGM_OK) goto done;
      if (cheb_pass<float>(s, kChebBackward, s->W2, s->W1, st, true) != SGM_OK) goto done;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto cuda_fail;
      float ms = 0;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) goto cuda_fail;
      if (rep > 0 && ms < best[m]) best[m] = ms;   // the first run includes one-time set-up
    }
  }
  result = best[1] < best[0] ? 1 : 0;
  goto done;
cuda_fail:
  fail(SGM_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (result < 0) s->cheb_tc = 0;
  return result;
}

}  // namespace

// one call on a permuted space (axes.cu): input of layout `win` -> P1 -> the canonical call
// (P1 -> P2, or P1 in place) -> output of layout `wout`
template <typename F>
static int permuted_call(sgm_space* s, int win, const void* in, int wout, void* out, cudaStream_t st, F call) {
  SGM_TRY(to_canonical(s, win, in, s->P1, st));
  SGM_TRY(call(s->P1, s->P2));
  return from_canonical(s, wout, s->P2, out, st);
}

extern "C" {

const char* sgm_last_error(void) { return g_err.c_str(); }

const char* sgm_status_string(int status) {
  switch (status) {
    case SGM_OK: return "ok";
    case SGM_ERR_NULL: return "NULL pointer";
    case SGM_ERR_SIZE: return "unsupported size or basis combination";
    case SGM_ERR_ARG: return "invalid argument";
    case SGM_ERR_ALIAS: return "input and output overlap";
    case SGM_ERR_ALIGN: return "misaligned pointer";
    case SGM_ERR_CUDA: return "CUDA error";
    case SGM_ERR_ALLOC: return "allocation failed";
    case SGM_ERR_STATE: return "invalid object state";
    default: return "unknown status";
  }
}

int sgm_space_create(sgm_space** out, int ndim, const int* kinds, const int64_t* n, const double* domain,
                     int precision) {
  if (!out || !kinds || !n) return fail(SGM_ERR_NULL, "out, kinds and n must be non-NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > 3) return fail(SGM_ERR_SIZE, "ndim must be 1..3 (got %d)", ndim);
  if (!canonical_axes(ndim, kinds)) return permuted_create(out, ndim, kinds, n, domain, precision);
  const int cheb_flags = precision & (SGM_CHEB_TC | SGM_CHEB_AUTO);
  precision &= ~(SGM_CHEB_TC | SGM_CHEB_AUTO);
  if (precision != SGM_F32 && precision != SGM_F64) return fail(SGM_ERR_ARG, "precision must be SGM_F32 or SGM_F64");
  if (cheb_flags == (SGM_CHEB_TC | SGM_CHEB_AUTO)) return fail(SGM_ERR_ARG, "SGM_CHEB_TC and SGM_CHEB_AUTO exclude each other");
  if (cheb_flags && precision != SGM_F32) return fail(SGM_ERR_ARG, "Chebyshev-axis method flags need an SGM_F32 space");
  auto polynomial = [](int k) {
    return k == SGM_CHEBYSHEV || k == SGM_SHEN_DIRICHLET || k == SGM_SHEN_BIHARMONIC || k == SGM_SHEN_NEUMANN ||
           k == SGM_LEGENDRE ||
           k == SGM_LEGENDRE_DIRICHLET || k == SGM_LEGENDRE_BIHARMONIC;
  };
  const bool cheb = polynomial(kinds[0]);
  const bool legendre = kinds[0] == SGM_LEGENDRE || kinds[0] == SGM_LEGENDRE_DIRICHLET || kinds[0] == SGM_LEGENDRE_BIHARMONIC;
  for (int d = 0; d < ndim; ++d) {
    const int k = kinds[d];
    if (k < SGM_CHEBYSHEV || k > SGM_SHEN_NEUMANN) return fail(SGM_ERR_ARG, "axis %d: unknown basis kind %d", d, k);
    if (d > 0 && polynomial(k)) return fail(SGM_ERR_SIZE, "axis %d: a Chebyshev or Legendre basis must be axis 0", d);
    if (k == SGM_FOURIER_R2C && d != ndim - 1) return fail(SGM_ERR_SIZE, "axis %d: only the last axis may be R2C", d);
    if (n[d] < 1 || n[d] > 4096) return fail(SGM_ERR_SIZE, "axis %d: size %lld outside 1..4096", d, (long long)n[d]);
  }
  if (kinds[0] == SGM_SHEN_DIRICHLET && n[0] < 4) return fail(SGM_ERR_SIZE, "Dirichlet basis needs N >= 4");
  if (kinds[0] == SGM_SHEN_NEUMANN && n[0] < 4) return fail(SGM_ERR_SIZE, "Neumann basis needs N >= 4");
  if (kinds[0] == SGM_SHEN_BIHARMONIC && n[0] < 6) return fail(SGM_ERR_SIZE, "biharmonic basis needs N >= 6");
  // the biharmonic elimination stages 13 coefficient tables of N + 8 doubles in shared memory
  if (kinds[0] == SGM_SHEN_BIHARMONIC && n[0] > 2048)
    return fail(SGM_ERR_SIZE, "biharmonic basis needs N <= 2048 (got %lld)", (long long)n[0]);
  if (kinds[0] == SGM_CHEBYSHEV && n[0] < 2) return fail(SGM_ERR_SIZE, "Chebyshev basis needs N >= 2");
  if (kinds[0] == SGM_LEGENDRE && n[0] < 2) return fail(SGM_ERR_SIZE, "Legendre basis needs N >= 2");
  if (kinds[0] == SGM_LEGENDRE_DIRICHLET && n[0] < 4) return fail(SGM_ERR_SIZE, "Legendre Dirichlet basis needs N >= 4");
  if (kinds[0] == SGM_LEGENDRE_BIHARMONIC && n[0] < 6) return fail(SGM_ERR_SIZE, "Legendre biharmonic basis needs N >= 6");
  // the Legendre transforms are dense N x N matrices held by the space
  if (legendre && n[0] > 1024) return fail(SGM_ERR_SIZE, "Legendre bases need N <= 1024 (got %lld)", (long long)n[0]);
  if (kinds[ndim - 1] == SGM_FOURIER_R2C && n[ndim - 1] < 2) return fail(SGM_ERR_SIZE, "R2C axis needs M >= 2");
  if ((cheb_flags & SGM_CHEB_TC) && (!cheb || n[0] > kTcMaxN))
    return fail(SGM_ERR_SIZE, "SGM_CHEB_TC needs a Chebyshev axis of at most %d points", kTcMaxN);
  if (cheb && domain && (domain[0] != -1.0 || domain[1] != 1.0))
    return fail(SGM_ERR_ARG, "the Chebyshev or Legendre axis domain must be [-1, 1]");
  if (domain)
    for (int d = 0; d < ndim; ++d)
      if (!(domain[2 * d + 1] > domain[2 * d])) return fail(SGM_ERR_ARG, "axis %d: empty domain", d);

  sgm_space* s = new (std::nothrow) sgm_space;
  if (!s) return fail(SGM_ERR_ALLOC, "host allocation failed");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    delete s;
    return fail(SGM_ERR_CUDA, "no CUDA device");
  }
  s->device = dev;
  s->ndim = ndim;
  s->prec = precision;
  s->cheb = cheb;
  s->legendre = legendre;
  for (int d = 0; d < ndim; ++d) {
    s->kinds[d] = kinds[d];
    s->n[d] = n[d];
    s->spec[d] = n[d];
    const bool cax = (d == 0 && cheb);
    s->dom[2 * d] = domain ? domain[2 * d] : (cax ? -1.0 : 0.0);
    s->dom[2 * d + 1] = domain ? domain[2 * d + 1] : (cax ? 1.0 : 2.0 * 3.14159265358979323846);
  }
  if (kinds[ndim - 1] == SGM_FOURIER_R2C) s->spec[ndim - 1] = n[ndim - 1] / 2 + 1;
  s->real_phys = kinds[ndim - 1] == SGM_FOURIER_R2C || (cheb && ndim == 1);
  s->real_spec = cheb && ndim == 1;
  s->nphys = 1;
  s->nspec = 1;
  for (int d = 0; d < ndim; ++d) {
    s->nphys *= n[d];
    s->nspec *= s->spec[d];
  }
  s->phys_bytes = s->nphys * (s->real_phys ? s->relem() : s->celem());
  s->spec_bytes = s->nspec * (s->real_spec ? s->relem() : s->celem());

  int st = SGM_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == SGM_OK) st = fail(SGM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  };
  // The streaming pipeline (k_stream.cu) of the physical-to-physical solves: FP32 spaces with a
  // Shen Dirichlet or biharmonic axis 0 of a streaming length, its Chebyshev pass by the FFT, and
  // Fourier axes C2C (axis 1 of a 3-D space) and R2C (last axis, even length) with streaming kernels.
  if (cheb && !legendre && precision == SGM_F32 && !(cheb_flags && n[0] <= kTcMaxN) &&
      (kinds[0] == SGM_SHEN_DIRICHLET || kinds[0] == SGM_SHEN_BIHARMONIC || kinds[0] == SGM_SHEN_NEUMANN) &&
      cheb_stream_length((int)n[0]) &&
      kinds[ndim - 1] == SGM_FOURIER_R2C && n[ndim - 1] % 2 == 0 && rows_stream_length((int)(n[ndim - 1] / 2)) &&
      (ndim == 2 || (ndim == 3 && kinds[1] == SGM_FOURIER_C2C && strided_stream_length((int)n[1])))) {
    s->stream = true;
    s->hp = (int)(n[ndim - 1] / 2 + 2);   // H + 1 coefficients rounded up to an even count
    s->inner_p = (ndim == 3 ? n[1] : 1) * (long)s->hp;
  }
  const size_t npad = s->stream ? (size_t)n[0] * s->inner_p : 0;
  const size_t wbytes = std::max({s->spec_bytes, (size_t)s->nspec * s->celem(), npad * s->celem()});
  chk(cudaMalloc(&s->W1, wbytes), "workspace");
  // W2 holds the spectral intermediate of the physical-to-physical solves: FP64 on the
  // one-tile-per-CTA kernels, complex64 on the streaming pipeline
  chk(cudaMalloc(&s->W2, std::max((size_t)s->nspec, npad) * 16), "workspace");
  if (st == SGM_OK && legendre) {
    st = legendre_build(s, cheb_flags != 0 && n[0] <= kTcMaxN);
    if (st == SGM_OK) st = build_project_table(s);
  } else if (st == SGM_OK && cheb) {
    const int N = (int)n[0];
    st = precision == SGM_F32 ? upload_dctw<float>(s, N) : upload_dctw<double>(s, N);
    if (st == SGM_OK) st = build_tables(s);
    if (st == SGM_OK) st = build_project_table(s);
    if (st == SGM_OK && (kinds[0] == SGM_SHEN_DIRICHLET || kinds[0] == SGM_SHEN_BIHARMONIC ||
                         kinds[0] == SGM_SHEN_NEUMANN)) {
      int sms = 0;
      chk(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
      long ncols = s->stream ? s->inner_p : s->nspec / N;
      long items = ncols;
      s->solve_nc = 1;
      if (ndim == 3) {
        const double L1 = s->dom[3] - s->dom[2], L2 = s->dom[5] - s->dom[4];
        const bool square = kinds[2] == SGM_FOURIER_R2C && n[1] == n[2] && std::fabs(L1 - L2) <= 1e-12 * std::fabs(L1);
        // The self-contained eliminations (inside stream capture; the factored solves take one
        // column per thread):
        // four columns per factorisation leave one warp per SM sub-partition on a 256^3 box, too
        // few to hide the latency of dependent FP64 instructions; the Dirichlet elimination, whose
        // per-column work is small next to its factorisation, runs faster with pairs and twice the
        // warps.  The biharmonic elimination keeps the groups of four.
        if (square && kinds[0] == SGM_SHEN_BIHARMONIC) {
          // columns (+-a, b), (+-b, a) share kappa2: one elimination thread per (a, b), a <= b
          const int M = (int)n[1], h = M / 2;
          std::vector<int2> g;
          for (int a = 0; a <= h; ++a)
            for (int b = a; b <= h; ++b) g.push_back(make_int2(a, b));
          s->ngroups = (long)g.size();
          chk(cudaMalloc(&s->groups, sizeof(int2) * g.size()), "group table");
          if (st == SGM_OK) chk(cudaMemcpy(s->groups, g.data(), sizeof(int2) * g.size(), cudaMemcpyHostToDevice), "group table");
          items = s->ngroups;
          s->solve_nc = 4;
        } else {
          // the streaming pipeline solves its padded columns too (n2 = hp)
          items = (1 + (n[1] - 1) / 2 + (n[1] % 2 == 0 ? 1 : 0)) * (s->stream ? (long)s->hp : s->spec[2]);
          s->solve_nc = 2;
        }
      }
      long need = 2 * ((items + 31) / 32) * 32;
      need = ((need + 127) / 128) * 128;
      s->scratch_threads = std::min((long)std::max(1, sms) * 256, need);
      const long rows = N / 2 + 1;
      const int nv = solve_scratch_values(kinds[0] == SGM_SHEN_DIRICHLET ? kDirichlet
                                          : kinds[0] == SGM_SHEN_NEUMANN ? kNeumann
                                                                         : kBiharmonic,
                                          s->solve_nc);
      size_t scratch_bytes = sizeof(double) * rows * nv * s->scratch_threads;
      // factorisation slots of the 3-D Dirichlet and biharmonic eliminations.  The factored solves
      // run one thread per column and parity (the four-column groups pay off only while the
      // factorisation is recomputed), for either column layout (spectral arrays; the padded
      // streaming intermediates); their scratch holds 2 values per row and thread
      const int nvf = kinds[0] == SGM_SHEN_DIRICHLET ? solve_factor_values(kDirichlet)
                      : kinds[0] == SGM_SHEN_BIHARMONIC ? solve_factor_values(kBiharmonic)
                                                        : 0;
      if (st == SGM_OK && ndim == 3 && nvf > 0) {
        Wavenumbers wn = wavenumbers(s);
        long thr = solve_factor_threads(s->nspec / N, wn);
        long sthr = solve_factored_scratch_threads(s->nspec / N, wn);
        if (s->stream) {
          wn.n2 = s->hp;
          thr = std::max(thr, solve_factor_threads(s->inner_p, wn));
          sthr = std::max(sthr, solve_factored_scratch_threads(s->inner_p, wn));
        }
        s->fact_threads = thr;
        s->fact_scratch_threads = ((sthr + 127) / 128) * 128;
        scratch_bytes = std::max(scratch_bytes, sizeof(double) * rows * 2 * s->fact_scratch_threads);
        for (int i = 0; i < 2 && st == SGM_OK; ++i)
          chk(cudaMalloc(&s->fact[i], sizeof(double) * rows * nvf * s->fact_threads), "factorisation table");
      }
      chk(cudaMalloc(&s->scratch, scratch_bytes), "solve scratch");
    }
  }
  if (st == SGM_OK && cheb && cheb_flags && n[0] <= kTcMaxN) {
    const int N = (int)n[0];
    // a Legendre space got the images of its dense matrices from legendre_build
    for (int mode : {kChebScalar, kChebBackward, kChebForwardT}) {
      if (legendre) continue;
      const std::vector<uint16_t> img = tc_cheb_image(mode, kinds[0], N);
      chk(cudaMalloc(&s->tc_img[mode], img.size() * 2), "contraction matrix");
      if (st == SGM_OK)
        chk(cudaMemcpy(s->tc_img[mode], img.data(), img.size() * 2, cudaMemcpyHostToDevice), "contraction matrix");
    }
    if (st == SGM_OK) s->cheb_tc = (cheb_flags & SGM_CHEB_TC) ? 1 : autotune_cheb(s);
    if (s->cheb_tc < 0) st = SGM_ERR_CUDA;
  }
  if (st == SGM_OK && s->stream) {
    const uint64_t N0 = (uint64_t)n[0], ip = (uint64_t)s->inner_p;
    const uint64_t dc[2] = {ip * 2, N0};
    const uint32_t boxc[2] = {32, (uint32_t)N0};
    const uint64_t sc1[1] = {ip * 8};
    bool ok = encode_tiled_map(&s->map_w1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, s->W1, dc, sc1, boxc) == cudaSuccess;
    if (ok && ndim == 3) {
      const uint64_t M1 = (uint64_t)n[1], hp = (uint64_t)s->hp;
      const uint64_t ds[3] = {hp * 2, M1, N0};
      const uint64_t ss[2] = {hp * 8, M1 * hp * 8};
      const uint32_t boxs[3] = {32, (uint32_t)M1, 1};
      ok = encode_tiled_map(&s->map_w1s, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, s->W1, ds, ss, boxs) == cudaSuccess;
    }
    if (!ok) st = fail(SGM_ERR_CUDA, "tensor map of the streaming pipeline rejected");
  }
  if (st != SGM_OK) {
    free_space(s);
    return st;
  }
  *out = s;
  return SGM_OK;
}

int sgm_space_solve_events(sgm_space* space, void* begin, void* end) {
  if (!space) return fail(SGM_ERR_NULL, "NULL space");
  if (space->magic != sgm_space::kMagic) return fail(SGM_ERR_STATE, "not a live sgm_space");
  if ((begin == nullptr) != (end == nullptr)) return fail(SGM_ERR_ARG, "give both events or neither");
  if (space->inner) return sgm_space_solve_events(space->inner, begin, end);
  space->ev_solve_begin = (cudaEvent_t)begin;
  space->ev_solve_end = (cudaEvent_t)end;
  return SGM_OK;
}

int sgm_space_cheb_method(const sgm_space* space, int* method) {
  if (!space || !method) return fail(SGM_ERR_NULL, "NULL argument");
  if (space->magic != sgm_space::kMagic) return fail(SGM_ERR_STATE, "not a live sgm_space");
  if (space->inner) return sgm_space_cheb_method(space->inner, method);
  *method = space->cheb_tc;
  return SGM_OK;
}

int sgm_tc_wait_timeouts(int* count, int reset) {
  if (!count) return fail(SGM_ERR_NULL, "NULL argument");
  const int v = tc_timeouts(reset != 0), w = cnn_tc_timeouts(reset != 0), x = stream_timeouts(reset != 0);
  if (v < 0 || w < 0 || x < 0) return fail(SGM_ERR_CUDA, "reading the device wait counters failed");
  *count = v + w + x;
  return SGM_OK;
}

int sgm_space_destroy(sgm_space* space) {
  if (!space) return SGM_OK;
  if (space->magic != sgm_space::kMagic) return fail(SGM_ERR_STATE, "not a live sgm_space");
  free_space(space);
  return SGM_OK;
}

int sgm_space_shape(const sgm_space* space, int which, int64_t* shape_out) {
  if (!space || !shape_out) return fail(SGM_ERR_NULL, "NULL argument");
  if (space->magic != sgm_space::kMagic) return fail(SGM_ERR_STATE, "not a live sgm_space");
  if (which != SGM_PHYSICAL && which != SGM_SPECTRAL) return fail(SGM_ERR_ARG, "which must be PHYSICAL or SPECTRAL");
  for (int d = 0; d < space->ndim; ++d) shape_out[d] = which == SGM_PHYSICAL ? space->n[d] : space->spec[d];
  return SGM_OK;
}

int sgm_scalar_product(sgm_space* s, const void* f, void* f_tilde, void* stream) {
  SGM_TRY(check_space(s));
  SGM_TRY(check_ptrs(f, s->phys_bytes, f_tilde, s->spec_bytes, false));
  if (s->inner)
    return permuted_call(s, SGM_PHYSICAL, f, SGM_SPECTRAL, f_tilde, (cudaStream_t)stream,
                         [&](void* a, void* b) { return sgm_scalar_product(s->inner, a, b, stream); });
  cudaStream_t st = (cudaStream_t)stream;
  return s->prec == SGM_F32 ? scalar_impl<float>(s, f, f_tilde, st, kChebScalar)
                            : scalar_impl<double>(s, f, f_tilde, st, kChebScalar);
}

int sgm_forward(sgm_space* s, const void* u, void* u_hat, void* stream) {
  SGM_TRY(check_space(s));
  SGM_TRY(check_ptrs(u, s->phys_bytes, u_hat, s->spec_bytes, false));
  if (s->inner)
    return permuted_call(s, SGM_PHYSICAL, u, SGM_SPECTRAL, u_hat, (cudaStream_t)stream,
                         [&](void* a, void* b) { return sgm_forward(s->inner, a, b, stream); });
  cudaStream_t st = (cudaStream_t)stream;
  return s->prec == SGM_F32 ? forward_impl<float>(s, u, u_hat, st) : forward_impl<double>(s, u, u_hat, st);
}

int sgm_backward(sgm_space* s, const void* u_hat, void* u, void* stream) {
  SGM_TRY(check_space(s));
  SGM_TRY(check_ptrs(u_hat, s->spec_bytes, u, s->phys_bytes, false));
  if (s->inner)
    return permuted_call(s, SGM_SPECTRAL, u_hat, SGM_PHYSICAL, u, (cudaStream_t)stream,
                         [&](void* a, void* b) { return sgm_backward(s->inner, a, b, stream); });
  cudaStream_t st = (cudaStream_t)stream;
  return s->prec == SGM_F32 ? backward_impl<float>(s, u_hat, u, st) : backward_impl<double>(s, u_hat, u, st);
}

// the Helmholtz solver needs a Dirichlet basis, the biharmonic solver a biharmonic one (either family)
static bool solver_matches(const sgm_space* s, int basis) {
  const int k = s->inner ? s->inner->kinds[0] : s->kinds[0];
  if (basis == kDirichlet) return k == SGM_SHEN_DIRICHLET || k == SGM_SHEN_NEUMANN || k == SGM_LEGENDRE_DIRICHLET;
  return k == SGM_SHEN_BIHARMONIC || k == SGM_LEGENDRE_BIHARMONIC;
}

static int solve_entry(sgm_space* s, int basis, double a, double b, double c, const void* f, void* u, void* stream) {
  SGM_TRY(check_space(s));
  if (!solver_matches(s, basis)) return fail(SGM_ERR_STATE, "axis 0 basis does not match this solver");
  if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c))
    return fail(SGM_ERR_ARG, "coefficients must be finite");
  if (basis == kDirichlet && a == 0.0 && b == 0.0) return fail(SGM_ERR_ARG, "a = b = 0 gives a singular system");
  if (basis == kBiharmonic && a == 0.0 && b == 0.0 && c == 0.0)
    return fail(SGM_ERR_ARG, "a = b = c = 0 gives a singular system");
  SGM_TRY(check_ptrs(f, s->spec_bytes, u, s->spec_bytes, true));
  cudaStream_t st = (cudaStream_t)stream;
  if (s->inner)
    return permuted_call(s, SGM_SPECTRAL, f, SGM_SPECTRAL, u, st, [&](void* x, void* y) {
      return solve_entry(s->inner, basis, a, b, c, x, y, stream);
    });
  return s->prec == SGM_F32 ? solve_impl<float>(s, basis, a, b, c, f, u, st)
                            : solve_impl<double>(s, basis, a, b, c, f, u, st);
}

int sgm_helmholtz_solve(sgm_space* s, double a, double b, const void* f_tilde, void* u_hat, void* stream) {
  return solve_entry(s, kDirichlet, a, b, 0.0, f_tilde, u_hat, stream);
}

int sgm_biharmonic_solve(sgm_space* s, double a, double b, double c, const void* f_tilde, void* u_hat,
                         void* stream) {
  return solve_entry(s, kBiharmonic, a, b, c, f_tilde, u_hat, stream);
}

// Physical -> physical on the streaming pipeline (FP32 spaces, see sgm_space::stream): R2C rows
// into the padded W1, the strided C2C axis in place, the Chebyshev scalar product (FP32 moments and
// stencil) into the padded W2 as complex64, the FP64 solve from W2 (inputs widened exactly, the
// result rounded once into W1; the padding columns are solved as dummy columns), and the Chebyshev,
// strided and C2R passes backwards from W1.
static int stream_entry(sgm_space* s, int basis, double a, double b, double c, const void* f, void* u,
                        cudaStream_t st) {
  const int nd = s->ndim;
  const int N0 = (int)s->n[0], M2 = (int)s->n[nd - 1], LF = M2 / 2;
  const long nrows = nd == 3 ? s->n[0] * s->n[1] : s->n[0];
  const void *twN = nullptr, *twLF = nullptr, *twM1 = nullptr;
  SGM_TRY(need_twf(s, N0, &twN));
  SGM_TRY(need_twf(s, LF, &twLF));
  SGM_TRY(need_tw(s, M2));
  if (nd == 3) SGM_TRY(need_twf(s, (int)s->n[1], &twM1));
  const float2* twL = (const float2*)s->tw[M2];
  float2* w1 = (float2*)s->W1;
  SGM_TRY(wrap(launch_rows_stream(kRowR2C, LF, f, w1, nrows, s->hp, (const float2*)twLF, twL, st),
               "rows forward"));
  if (nd == 3)
    SGM_TRY(wrap(launch_strided_stream(false, (int)s->n[1], s->map_w1s, w1, s->n[0], s->hp, (const float2*)twM1,
                                       st),
                 "strided forward"));
  SGM_TRY(wrap(launch_cheb_stream(kChebScalar, N0, s->map_w1, s->W2, s->inner_p, s->kinds[0], (const float2*)twN,
                                  (const float2*)s->dctw, st),
               "chebyshev pass"));
  Wavenumbers wn = wavenumbers(s);
  wn.n2 = s->hp;
  if (s->kinds[0] == SGM_SHEN_NEUMANN) basis = kNeumann;
  if (s->ev_solve_begin) SGM_TRY(wrap(cudaEventRecord(s->ev_solve_begin, st), "solve event"));
  SGM_TRY((eliminate<float, float>(s, basis, a, b, c, s->W2, w1, s->inner_p, wn, st)));
  if (s->ev_solve_end) SGM_TRY(wrap(cudaEventRecord(s->ev_solve_end, st), "solve event"));
  SGM_TRY(wrap(launch_cheb_stream(kChebBackward, N0, s->map_w1, w1, s->inner_p, s->kinds[0], (const float2*)twN,
                                  (const float2*)s->dctw, st),
               "chebyshev pass"));
  if (nd == 3)
    SGM_TRY(wrap(launch_strided_stream(true, (int)s->n[1], s->map_w1s, w1, s->n[0], s->hp, (const float2*)twM1,
                                       st),
                 "strided backward"));
  return wrap(launch_rows_stream(kRowC2R, LF, w1, u, nrows, s->hp, (const float2*)twLF, twL, st),
              "rows backward");
}

// Physical -> physical: scalar product into W2 (FP64 spectral intermediate), FP64 solve in
// place, backward from W2.  On FP32 spaces the transforms stay FP32 and only the
// Chebyshev kernels widen/narrow the intermediate.
static int full_entry(sgm_space* s, int basis, double a, double b, double c, const void* f, void* u, void* stream) {
  SGM_TRY(check_space(s));
  if (!solver_matches(s, basis)) return fail(SGM_ERR_STATE, "axis 0 basis does not match this solver");
  if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c))
    return fail(SGM_ERR_ARG, "coefficients must be finite");
  if (basis == kDirichlet && a == 0.0 && b == 0.0) return fail(SGM_ERR_ARG, "a = b = 0 gives a singular system");
  if (basis == kBiharmonic && a == 0.0 && b == 0.0 && c == 0.0)
    return fail(SGM_ERR_ARG, "a = b = c = 0 gives a singular system");
  SGM_TRY(check_ptrs(f, s->phys_bytes, u, s->phys_bytes, false));
  cudaStream_t st = (cudaStream_t)stream;
  if (s->inner)
    return permuted_call(s, SGM_PHYSICAL, f, SGM_PHYSICAL, u, st, [&](void* x, void* y) {
      return full_entry(s->inner, basis, a, b, c, x, y, stream);
    });
  if (s->prec == SGM_F32 && s->stream) return stream_entry(s, basis, a, b, c, f, u, st);
  auto solve = [&]() -> int {
    if (s->ev_solve_begin) SGM_TRY(wrap(cudaEventRecord(s->ev_solve_begin, st), "solve event"));
    SGM_TRY(solve_impl<double>(s, basis, a, b, c, s->W2, s->W2, st));
    if (s->ev_solve_end) SGM_TRY(wrap(cudaEventRecord(s->ev_solve_end, st), "solve event"));
    return SGM_OK;
  };
  if (s->prec == SGM_F32) {
    SGM_TRY(scalar_impl<float>(s, f, s->W2, st, kChebScalar, true));
    SGM_TRY(solve());
    return backward_impl<float>(s, s->W2, u, st, true);
  }
  SGM_TRY(scalar_impl<double>(s, f, s->W2, st, kChebScalar));
  SGM_TRY(solve());
  return backward_impl<double>(s, s->W2, u, st);
}

int sgm_helmholtz(sgm_space* s, double a, double b, const void* f, void* u, void* stream) {
  return full_entry(s, kDirichlet, a, b, 0.0, f, u, stream);
}

int sgm_biharmonic(sgm_space* s, double a, double b, double c, const void* f, void* u, void* stream) {
  return full_entry(s, kBiharmonic, a, b, c, f, u, stream);
}

}  // extern "C"
