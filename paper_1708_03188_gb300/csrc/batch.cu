// batch.cu - host side of the batched 1-D Helmholtz problems (kernels in k_batch.cu):
// problem table sorted by size, per-size FFT plans and twiddle pools, warp-interleaved FP64
// buffers, and the C ABI entry points sgm_batch_*.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/sgm.h"
#include "common.cuh"

namespace sgm {
struct BatchProblemH {  // host mirror of BatchProblem in k_batch.cu
  int N;
  int slot;
  long offset;
  double alpha;
  int tw_off;
  int dct_off;
  int plan;
  int L;
  int chirp_off;
  int bhat_off;
};
size_t batch_problem_bytes();
template <typename T>
cudaError_t launch_batch(const void* f, void* u, int nprob, int nslots, int ldb, const void* probs,
                         const int* by_slot, const void* plans, const void* pool, const long* wbase, double* S,
                         double* U, double* scratch, const long* sbase, const void* coef, const double* mass,
                         cudaStream_t s);

}  // namespace sgm

using namespace sgm;

struct sgm_batch {
  static constexpr uint32_t kMagic = 0x53474231u;
  uint32_t magic = kMagic;
  int device = 0;
  int prec = SGM_F64;
  int nprob = 0, Nmax = 0;
  int ldb = 0;                    // shared-memory buffer length of the transform kernels
  int nbluestein = 0;             // problems whose DFT runs as a Bluestein convolution
  long total = 0;                 // sum of N
  std::vector<int64_t> offsets;   // nprob + 1
  void* probs = nullptr;
  int* by_slot = nullptr;
  void* plans = nullptr;
  void* pool = nullptr;
  long* wbase = nullptr;
  long* sbase = nullptr;
  double* S = nullptr;
  double* U = nullptr;
  double* scratch = nullptr;
  double* coef = nullptr;         // (-2 pi (k+1)(k+2), -4 pi (k+1)) per row k < Nmax
  double* mass = nullptr;         // B_kk: 3 pi / 2 for k = 0, else pi
};

namespace {

void free_batch(sgm_batch* b) {
  cudaFree(b->probs);
  cudaFree(b->by_slot);
  cudaFree(b->plans);
  cudaFree(b->pool);
  cudaFree(b->wbase);
  cudaFree(b->sbase);
  cudaFree(b->S);
  cudaFree(b->U);
  cudaFree(b->scratch);
  cudaFree(b->coef);
  cudaFree(b->mass);
  b->magic = 0;
  delete b;
}

template <typename T> void push_twiddles(std::vector<cplx<T>>& pool, int N, long double denom) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < N; ++k) {
    const long double a = -pi * k / denom;
    cplx<T> w;
    w.x = (T)cosl(a);
    w.y = (T)sinl(a);
    pool.push_back(w);
  }
}

int largest_prime_factor(int n) {
  int best = 1;
  for (int p = 2; p * p <= n; ++p)
    while (n % p == 0) {
      best = p;
      n /= p;
    }
  return n > 1 ? std::max(best, n) : best;
}

// sizes with a prime factor above this run their DFT as a Bluestein convolution
constexpr int kBluesteinPrime = 32;

// in-place radix-2 DFT of a power-of-two length (exp(-2 pi i j k / L)), long double
void host_fft(std::vector<long double>& re, std::vector<long double>& im) {
  const size_t L = re.size();
  for (size_t i = 1, j = 0; i < L; ++i) {
    size_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  const long double pi = 3.141592653589793238462643383279502884L;
  for (size_t len = 2; len <= L; len <<= 1) {
    for (size_t i = 0; i < L; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const long double a = -2.0L * pi * (long double)k / (long double)len;
        const long double wr = cosl(a), wi = sinl(a);
        const size_t u = i + k, v = i + k + len / 2;
        const long double xr = re[v] * wr - im[v] * wi, xi = re[v] * wi + im[v] * wr;
        re[v] = re[u] - xr;
        im[v] = im[u] - xi;
        re[u] += xr;
        im[u] += xi;
      }
  }
}

// Bluestein tables of length N with convolution length L: chirp c_n = exp(-i pi n^2 / N)
// (n^2 reduced modulo 2N exactly), then FFT_L of b (b_n = conj c_n, b_{L-n} = b_n) divided by L
template <typename T> void push_bluestein(std::vector<cplx<T>>& pool, int N, int L, int& chirp_off, int& bhat_off) {
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> cr(N), ci(N);
  for (long n = 0; n < N; ++n) {
    const long m = (n * n) % (2L * N);
    const long double a = -pi * (long double)m / (long double)N;
    cr[n] = cosl(a);
    ci[n] = sinl(a);
  }
  chirp_off = (int)pool.size();
  for (int n = 0; n < N; ++n) pool.push_back(mk<cplx<T>>((T)cr[n], (T)ci[n]));
  std::vector<long double> br(L, 0.0L), bi(L, 0.0L);
  for (int n = 0; n < N; ++n) {
    br[n] = cr[n];
    bi[n] = -ci[n];
    if (n > 0) {
      br[L - n] = cr[n];
      bi[L - n] = -ci[n];
    }
  }
  host_fft(br, bi);
  bhat_off = (int)pool.size();
  for (int m = 0; m < L; ++m) pool.push_back(mk<cplx<T>>((T)(br[m] / L), (T)(bi[m] / L)));
}

template <typename T> int build(sgm_batch* b, const int64_t* n, const double* alpha) {
  const int P = b->nprob;
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::map<int, int> size_index;   // N -> plan index
  std::vector<FftPlan> plans;
  std::vector<cplx<T>> pool;
  std::vector<int> tw_off, dct_off, conv_len, chirp_off, bhat_off;
  std::vector<BatchProblemH> probs(P);
  b->ldb = b->Nmax + 1;
  for (int p = 0; p < P; ++p) {
    const int N = (int)n[p];
    if (!size_index.count(N)) {
      size_index[N] = (int)plans.size();
      int L = 0, co = 0, bo = 0;
      if (largest_prime_factor(N) > kBluesteinPrime) {
        L = 1;
        while (L < 2 * N - 1) L *= 2;
        b->ldb = std::max(b->ldb, L);
      }
      const int Lf = L ? L : N;
      plans.push_back(host_plan(Lf));
      tw_off.push_back((int)pool.size());
      push_twiddles<T>(pool, Lf, (long double)Lf / 2.0L);  // exp(-2 pi i k / Lf)
      dct_off.push_back((int)pool.size());
      push_twiddles<T>(pool, N, 2.0L * N);                 // exp(-i pi k / (2N))
      if (L) push_bluestein<T>(pool, N, L, co, bo);
      conv_len.push_back(L);
      chirp_off.push_back(co);
      bhat_off.push_back(bo);
    }
    const int pi = size_index[N];
    probs[p] = {N, 0, (long)b->offsets[p], alpha[p], tw_off[pi], dct_off[pi], pi, conv_len[pi], chirp_off[pi], bhat_off[pi]};
    if (conv_len[pi]) ++b->nbluestein;
  }
  std::vector<int> by_slot(P);
  for (int s = 0; s < P; ++s) {
    by_slot[s] = order[s];
    probs[order[s]].slot = s;
  }
  const int nw = (P + 31) / 32;
  std::vector<long> wbase(nw + 1), sbase(nw + 1);
  wbase[0] = sbase[0] = 0;
  for (int w = 0; w < nw; ++w) {
    const int Nw = (int)n[order[w * 32]];                  // largest N of the warp
    wbase[w + 1] = wbase[w] + (long)Nw * 32;
    sbase[w + 1] = sbase[w] + (long)(Nw / 2 + 1) * 96;
  }
  static_assert(sizeof(BatchProblemH) == 48, "BatchProblem layout");
  if (batch_problem_bytes() != sizeof(BatchProblemH)) return set_error(SGM_ERR_STATE, "problem table layout");
  cudaError_t e = cudaSuccess;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(&b->probs, probs.data(), sizeof(BatchProblemH) * P);
  up((void**)&b->by_slot, by_slot.data(), sizeof(int) * P);
  up(&b->plans, plans.data(), sizeof(FftPlan) * plans.size());
  up(&b->pool, pool.data(), sizeof(cplx<T>) * pool.size());
  up((void**)&b->wbase, wbase.data(), sizeof(long) * wbase.size());
  up((void**)&b->sbase, sbase.data(), sizeof(long) * sbase.size());
  {
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<double> coef(2 * (size_t)b->Nmax), mass(b->Nmax);
    for (int k = 0; k < b->Nmax; ++k) {
      coef[2 * k] = (double)(-2.0L * pi * (k + 1) * (k + 2));
      coef[2 * k + 1] = (double)(-4.0L * pi * (k + 1));
      mass[k] = (double)(k == 0 ? 1.5L * pi : pi);
    }
    up((void**)&b->coef, coef.data(), sizeof(double) * coef.size());
    up((void**)&b->mass, mass.data(), sizeof(double) * mass.size());
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->S, sizeof(double) * wbase[nw]);
  if (e == cudaSuccess) e = cudaMalloc(&b->U, sizeof(double) * wbase[nw]);
  if (e == cudaSuccess) e = cudaMalloc(&b->scratch, sizeof(double) * 2 * sbase[nw]);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
  return SGM_OK;
}

}  // namespace

extern "C" {

int sgm_batch_create(sgm_batch** out, int nprob, const int64_t* n, const double* alpha, int precision) {
  if (!out || !n || !alpha) return set_error(SGM_ERR_NULL, "out, n and alpha must be non-NULL");
  *out = nullptr;
  if (nprob < 1) return set_error(SGM_ERR_SIZE, "nprob must be >= 1");
  if (precision != SGM_F32 && precision != SGM_F64) return set_error(SGM_ERR_ARG, "precision must be SGM_F32 or SGM_F64");
  for (int p = 0; p < nprob; ++p) {
    if (n[p] < 4 || n[p] > 4096) return set_error(SGM_ERR_SIZE, "problem %d: N = %lld outside 4..4096", p, (long long)n[p]);
    if (!std::isfinite(alpha[p])) return set_error(SGM_ERR_ARG, "problem %d: alpha not finite", p);
  }
  sgm_batch* b = new (std::nothrow) sgm_batch;
  if (!b) return set_error(SGM_ERR_ALLOC, "host allocation failed");
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return set_error(SGM_ERR_CUDA, "no CUDA device");
  }
  b->prec = precision;
  b->nprob = nprob;
  b->offsets.resize(nprob + 1);
  b->offsets[0] = 0;
  for (int p = 0; p < nprob; ++p) {
    b->offsets[p + 1] = b->offsets[p] + n[p];
    b->Nmax = std::max(b->Nmax, (int)n[p]);
  }
  b->total = (long)b->offsets[nprob];
  const int st = precision == SGM_F32 ? build<float>(b, n, alpha) : build<double>(b, n, alpha);
  if (st != SGM_OK) {
    free_batch(b);
    return st;
  }
  *out = b;
  return SGM_OK;
}

int sgm_batch_destroy(sgm_batch* batch) {
  if (!batch) return SGM_OK;
  if (batch->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  free_batch(batch);
  return SGM_OK;
}

int sgm_batch_offsets(const sgm_batch* batch, int64_t* offsets) {
  if (!batch || !offsets) return set_error(SGM_ERR_NULL, "NULL argument");
  if (batch->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  std::memcpy(offsets, batch->offsets.data(), sizeof(int64_t) * batch->offsets.size());
  return SGM_OK;
}

int sgm_batch_helmholtz(sgm_batch* b, const void* f, void* u, void* stream) {
  if (!b) return set_error(SGM_ERR_NULL, "batch is NULL");
  if (b->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return set_error(SGM_ERR_STATE, "wrong current device");
  if (!f || !u) return set_error(SGM_ERR_NULL, "NULL data pointer");
  const size_t bytes = (b->prec == SGM_F32 ? 4 : 8) * (size_t)b->total;
  if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return set_error(SGM_ERR_ALIGN, "pointers must be 16-byte aligned");
  const char* pa = (const char*)f;
  const char* pb = (const char*)u;
  if (pa < pb + bytes && pb < pa + bytes) return set_error(SGM_ERR_ALIAS, "f and u overlap");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = b->prec == SGM_F32
                      ? launch_batch<float>(f, u, b->nprob, b->nprob, b->ldb, b->probs, b->by_slot, b->plans, b->pool,
                                            b->wbase, b->S, b->U, b->scratch, b->sbase, b->coef, b->mass, s)
                      : launch_batch<double>(f, u, b->nprob, b->nprob, b->ldb, b->probs, b->by_slot, b->plans, b->pool,
                                             b->wbase, b->S, b->U, b->scratch, b->sbase, b->coef, b->mass, s);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

}  // extern "C"
