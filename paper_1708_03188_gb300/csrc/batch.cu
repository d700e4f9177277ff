// batch.cu - host side of the batched problems (kernels in k_batch.cu): for the 1-D Helmholtz
// problems the problem table sorted by size, per-size FFT plans and twiddle pools and the
// warp-interleaved FP64 buffers; for the 2-D problems one space each; the CUDA graph that runs
// the whole batch as one launch; and the C ABI entry points sgm_batch_*.
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
  int bluestein_prime = 0;        // the autotuned threshold on the largest prime factor
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
  // 2-D problems (sgm_batch_add_2d)
  struct Prob2D {
    int N, M;
    sgm_space* sp;
    int branch;
  };
  std::vector<Prob2D> p2;
  std::vector<int64_t> off2;      // element offsets, multiples of 4
  double a2 = 0.0, b2 = 0.0;
  int nbranch = 0;                // graph branches used by the 2-D problems
  // the captured graph of sgm_batch_run and the pointers it was captured with
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> br;   // [0] 1-D problems, [1..] 2-D problems
  std::vector<cudaEvent_t> ev;    // [0] fork, [1 + i] join of branch i
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* cap[4] = {nullptr, nullptr, nullptr, nullptr};
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
  for (auto& q : b->p2) sgm_space_destroy(q.sp);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (cudaStream_t t : b->br) cudaStreamDestroy(t);
  if (b->cs) cudaStreamDestroy(b->cs);
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

// candidate thresholds of the batch autotuner: a size whose largest prime factor is above the
// threshold runs its DFT as a Bluestein convolution; kNoBluestein disables it
constexpr int kNoBluestein = 1 << 30;
// shared memory one transform CTA may use (the opt-in maximum of a CTA on sm_103a is 227 KB)
constexpr size_t kMaxBatchSmem = 227 * 1024;

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

// Size-dependent tables for one Bluestein threshold: a size N whose largest prime factor exceeds
// `prime` runs its DFT as a Bluestein convolution, every other size through its own mixed-radix
// plan.  Fills the plan fields of probs (not the slots) and returns the shared-memory buffer
// length of the transform kernels.  `blue` caches the chirp tables per size across thresholds.
template <typename T>
int plan_tables(const sgm_batch* b, const int64_t* n, const double* alpha, int prime,
                std::map<int, std::vector<cplx<T>>>& blue, std::vector<BatchProblemH>& probs,
                std::vector<FftPlan>& plans, std::vector<cplx<T>>& pool, int& nblue) {
  const int P = b->nprob;
  std::map<int, int> size_index;   // N -> plan index
  std::vector<int> tw_off, dct_off, conv_len, chirp_off, bhat_off;
  plans.clear();
  pool.clear();
  nblue = 0;
  int ldb = b->Nmax + 1;
  for (int p = 0; p < P; ++p) {
    const int N = (int)n[p];
    if (!size_index.count(N)) {
      size_index[N] = (int)plans.size();
      int L = 0, co = 0, bo = 0;
      if (largest_prime_factor(N) > prime) {
        L = 1;
        while (L < 2 * N - 1) L *= 2;
        // the two convolution buffers must fit a CTA's shared memory (227 KB); larger sizes
        // (FP64 beyond N = 2048) keep their direct plan
        if (2 * sizeof(cplx<T>) * (size_t)L > kMaxBatchSmem) L = 0;
        else ldb = std::max(ldb, L);
      }
      const int Lf = L ? L : N;
      plans.push_back(host_plan(Lf));
      tw_off.push_back((int)pool.size());
      push_twiddles<T>(pool, Lf, (long double)Lf / 2.0L);  // exp(-2 pi i k / Lf)
      dct_off.push_back((int)pool.size());
      push_twiddles<T>(pool, N, 2.0L * N);                 // exp(-i pi k / (2N))
      if (L) {
        auto it = blue.find(N);
        if (it == blue.end()) {
          std::vector<cplx<T>> tab;
          int c0 = 0, b0 = 0;
          push_bluestein<T>(tab, N, L, c0, b0);   // chirp (N values) then bhat (L values)
          it = blue.emplace(N, std::move(tab)).first;
        }
        co = (int)pool.size();
        bo = co + N;
        pool.insert(pool.end(), it->second.begin(), it->second.end());
      }
      conv_len.push_back(L);
      chirp_off.push_back(co);
      bhat_off.push_back(bo);
    }
    const int pi = size_index[N];
    const int slot = probs[p].slot;
    probs[p] = {N, slot, (long)b->offsets[p], alpha[p], tw_off[pi], dct_off[pi], pi, conv_len[pi], chirp_off[pi], bhat_off[pi]};
    if (conv_len[pi]) ++nblue;
  }
  return ldb;
}

template <typename T> int build(sgm_batch* b, const int64_t* n, const double* alpha, bool autotune) {
  const int P = b->nprob;
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::vector<BatchProblemH> probs(P);
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
  up((void**)&b->by_slot, by_slot.data(), sizeof(int) * P);
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

  // size-dependent tables; with problems present, the Bluestein threshold is autotuned: the whole
  // batch (three kernels) is timed on zero input for each candidate and the fastest is kept
  std::map<int, std::vector<cplx<T>>> blue;
  std::vector<FftPlan> plans;
  std::vector<cplx<T>> pool;
  auto install = [&](int prime) -> int {
    cudaFree(b->probs);
    cudaFree(b->plans);
    cudaFree(b->pool);
    b->probs = b->plans = b->pool = nullptr;
    int nblue = 0;
    b->ldb = plan_tables<T>(b, n, alpha, prime, blue, probs, plans, pool, nblue);
    b->nbluestein = nblue;
    b->bluestein_prime = prime;
    up(&b->probs, probs.data(), sizeof(BatchProblemH) * P);
    up(&b->plans, plans.data(), sizeof(FftPlan) * plans.size());
    up(&b->pool, pool.data(), sizeof(cplx<T>) * pool.size());
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch tables: %s", cudaGetErrorString(e));
    return SGM_OK;
  };
  const int candidates[] = {16, 32, 64, kNoBluestein};
  int best = 32;
  if (P > 0 && autotune) {
    void* f = nullptr;
    void* u = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t te = cudaMalloc(&f, sizeof(T) * (size_t)b->total);
    if (te == cudaSuccess) te = cudaMalloc(&u, sizeof(T) * (size_t)b->total);
    if (te == cudaSuccess) te = cudaMemset(f, 0, sizeof(T) * (size_t)b->total);
    if (te == cudaSuccess) te = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (te == cudaSuccess) te = cudaEventCreate(&e0);
    if (te == cudaSuccess) te = cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int prime : candidates) {
      if (te != cudaSuccess) break;
      const int st_ = install(prime);
      if (st_ != SGM_OK) {
        te = cudaErrorUnknown;
        break;
      }
      float ms_min = 1e30f;
      for (int rep = 0; rep < 4 && te == cudaSuccess; ++rep) {
        te = cudaEventRecord(e0, st);
        if (te == cudaSuccess)
          te = launch_batch<T>(f, u, b->nprob, b->nprob, b->ldb, b->probs, b->by_slot, b->plans, b->pool, b->wbase,
                               b->S, b->U, b->scratch, b->sbase, b->coef, b->mass, st);
        if (te == cudaSuccess) te = cudaEventRecord(e1, st);
        if (te == cudaSuccess) te = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (te == cudaSuccess) te = cudaEventElapsedTime(&ms, e0, e1);
        if (te == cudaSuccess && rep > 0) ms_min = std::min(ms_min, ms);   // the first run sets attributes
      }
      if (te == cudaSuccess && ms_min < best_ms) {
        best_ms = ms_min;
        best = prime;
      }
    }
    cudaFree(f);
    cudaFree(u);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (te != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(te));
  }
  return install(best);
}

constexpr int kBranches = 64;

#define SGM_BATCH_TRY(x)           \
  do {                             \
    const int st_ = (x);           \
    if (st_ != SGM_OK) return st_; \
  } while (0)

int check_batch(const sgm_batch* b) {
  if (!b) return set_error(SGM_ERR_NULL, "batch is NULL");
  if (b->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return set_error(SGM_ERR_STATE, "wrong current device");
  return SGM_OK;
}

int check_pair(const void* f, const void* u, size_t bytes) {
  if (!f || !u) return set_error(SGM_ERR_NULL, "NULL data pointer");
  if (((uintptr_t)f & 15) || ((uintptr_t)u & 15)) return set_error(SGM_ERR_ALIGN, "pointers must be 16-byte aligned");
  const char* pa = (const char*)f;
  const char* pb = (const char*)u;
  if (pa < pb + bytes && pb < pa + bytes) return set_error(SGM_ERR_ALIAS, "f and u overlap");
  return SGM_OK;
}

int launch_1d(sgm_batch* b, const void* f, void* u, cudaStream_t s) {
  cudaError_t e = b->prec == SGM_F32
                      ? launch_batch<float>(f, u, b->nprob, b->nprob, b->ldb, b->probs, b->by_slot, b->plans, b->pool,
                                            b->wbase, b->S, b->U, b->scratch, b->sbase, b->coef, b->mass, s)
                      : launch_batch<double>(f, u, b->nprob, b->nprob, b->ldb, b->probs, b->by_slot, b->plans, b->pool,
                                             b->wbase, b->S, b->U, b->scratch, b->sbase, b->coef, b->mass, s);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

int run_2d(sgm_batch* b, int q, const void* f2, void* u2, cudaStream_t s) {
  const size_t el = b->prec == SGM_F32 ? 4 : 8;
  const auto& p = b->p2[q];
  return sgm_helmholtz(p.sp, b->a2, b->b2, (const char*)f2 + el * b->off2[q], (char*)u2 + el * b->off2[q], s);
}

// (re)capture the graph of the whole batch for these pointers
int capture(sgm_batch* b, const void* f1, void* u1, const void* f2, void* u2) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  std::memset(b->cap, 0, sizeof b->cap);
  cudaError_t e = cudaSuccess;
  auto cu = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (!b->cs) {
    cu(cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking));
    for (int i = 0; i <= kBranches && e == cudaSuccess; ++i) {
      cudaStream_t t = nullptr;
      cu(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
      if (e == cudaSuccess) b->br.push_back(t);
    }
    for (int i = 0; i <= kBranches + 1 && e == cudaSuccess; ++i) {
      cudaEvent_t v = nullptr;
      cu(cudaEventCreateWithFlags(&v, cudaEventDisableTiming));
      if (e == cudaSuccess) b->ev.push_back(v);
    }
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch streams: %s", cudaGetErrorString(e));
  }
  // one eager pass: builds every lazily created table and sets kernel attributes outside capture
  if (b->nprob > 0) SGM_BATCH_TRY(launch_1d(b, f1, u1, b->cs));
  for (int q = 0; q < (int)b->p2.size(); ++q) SGM_BATCH_TRY(run_2d(b, q, f2, u2, b->cs));
  cu(cudaStreamSynchronize(b->cs));
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch warm-up: %s", cudaGetErrorString(e));

  cu(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  int st = SGM_OK;
  const int nbr = 1 + b->nbranch;
  cu(cudaEventRecord(b->ev[0], b->cs));
  for (int i = 0; i < nbr; ++i) cu(cudaStreamWaitEvent(b->br[i], b->ev[0], 0));
  if (e == cudaSuccess && b->nprob > 0) st = launch_1d(b, f1, u1, b->br[0]);
  for (int q = 0; q < (int)b->p2.size() && st == SGM_OK && e == cudaSuccess; ++q)
    st = run_2d(b, q, f2, u2, b->br[b->p2[q].branch]);
  for (int i = 0; i < nbr; ++i) {
    cu(cudaEventRecord(b->ev[1 + i], b->br[i]));
    cu(cudaStreamWaitEvent(b->cs, b->ev[1 + i], 0));
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->cs, &g);
  if (st == SGM_OK && e == cudaSuccess) e = ee;
  if (st != SGM_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != SGM_OK ? st : set_error(SGM_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    return set_error(SGM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  b->graph = g;
  b->cap[0] = f1;
  b->cap[1] = u1;
  b->cap[2] = f2;
  b->cap[3] = u2;
  return SGM_OK;
}

}  // namespace

extern "C" {

int sgm_batch_create(sgm_batch** out, int nprob, const int64_t* n, const double* alpha, int precision) {
  if (!out) return set_error(SGM_ERR_NULL, "out must be non-NULL");
  *out = nullptr;
  if (nprob < 0) return set_error(SGM_ERR_SIZE, "nprob must be >= 0");
  if (nprob > 0 && (!n || !alpha)) return set_error(SGM_ERR_NULL, "n and alpha must be non-NULL");
  const bool fixed_plan = (precision & SGM_BATCH_FIXED_PLAN) != 0;
  precision &= ~SGM_BATCH_FIXED_PLAN;
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
  const int st = precision == SGM_F32 ? build<float>(b, n, alpha, !fixed_plan) : build<double>(b, n, alpha, !fixed_plan);
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
  SGM_BATCH_TRY(check_batch(b));
  SGM_BATCH_TRY(check_pair(f, u, (b->prec == SGM_F32 ? 4 : 8) * (size_t)b->total));
  return launch_1d(b, f, u, (cudaStream_t)stream);
}

int sgm_batch_add_2d(sgm_batch* b, int nprob, const int64_t* sizes, double a, double bc) {
  SGM_BATCH_TRY(check_batch(b));
  if (!sizes) return set_error(SGM_ERR_NULL, "sizes must be non-NULL");
  if (nprob < 1) return set_error(SGM_ERR_SIZE, "nprob must be >= 1");
  if (!b->p2.empty() || b->exec) return set_error(SGM_ERR_STATE, "2-D problems were already added or the batch has run");
  if (!std::isfinite(a) || !std::isfinite(bc) || (a == 0.0 && bc == 0.0)) return set_error(SGM_ERR_ARG, "bad a, b");
  for (int q = 0; q < nprob; ++q) {
    const int64_t N = sizes[2 * q], M = sizes[2 * q + 1];
    if (N < 4 || N > 4096 || M < 2 || M > 4096)
      return set_error(SGM_ERR_SIZE, "2-D problem %d: sizes %lld x %lld outside [4, 4096] x [2, 4096]", q, (long long)N,
                       (long long)M);
  }
  const int kinds[2] = {SGM_SHEN_DIRICHLET, SGM_FOURIER_R2C};
  const int prec = b->prec == SGM_F32 ? (SGM_F32 | SGM_CHEB_AUTO) : SGM_F64;
  b->off2.assign(1, 0);
  std::vector<double> cost;
  for (int q = 0; q < nprob; ++q) {
    const int64_t n2[2] = {sizes[2 * q], sizes[2 * q + 1]};
    sgm_space* sp = nullptr;
    const int st = sgm_space_create(&sp, 2, kinds, n2, nullptr, prec);
    if (st != SGM_OK) {
      for (auto& r : b->p2) sgm_space_destroy(r.sp);
      b->p2.clear();
      b->off2.clear();
      return st;
    }
    b->p2.push_back({(int)n2[0], (int)n2[1], sp, 0});
    b->off2.push_back(b->off2.back() + (n2[0] * n2[1] + 3) / 4 * 4);
    // the serial FP64 elimination of N/2 rows dominates a problem's time
    cost.push_back((double)n2[0] * (64.0 + (double)n2[1] / 64.0));
  }
  b->a2 = a;
  b->b2 = bc;
  // longest processing time first over up to kBranches concurrent graph branches
  b->nbranch = std::min(nprob, kBranches);
  std::vector<int> order(nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> load(b->nbranch, 0.0);
  for (int q : order) {
    const int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->p2[q].branch = 1 + i;
    load[i] += cost[q];
  }
  return SGM_OK;
}

int sgm_batch_info(const sgm_batch* b, int* bluestein_prime, int* n_bluestein) {
  if (!b || !bluestein_prime || !n_bluestein) return set_error(SGM_ERR_NULL, "NULL argument");
  if (b->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  *bluestein_prime = b->bluestein_prime >= kNoBluestein ? 0 : b->bluestein_prime;
  *n_bluestein = b->nbluestein;
  return SGM_OK;
}

int sgm_batch_offsets_2d(const sgm_batch* b, int64_t* offsets) {
  if (!b || !offsets) return set_error(SGM_ERR_NULL, "NULL argument");
  if (b->magic != sgm_batch::kMagic) return set_error(SGM_ERR_STATE, "not a live sgm_batch");
  if (b->p2.empty()) return set_error(SGM_ERR_STATE, "the batch has no 2-D problems");
  std::memcpy(offsets, b->off2.data(), sizeof(int64_t) * b->off2.size());
  return SGM_OK;
}

int sgm_batch_run(sgm_batch* b, const void* f1, void* u1, const void* f2, void* u2, void* stream) {
  SGM_BATCH_TRY(check_batch(b));
  const size_t el = b->prec == SGM_F32 ? 4 : 8;
  if (b->nprob > 0) SGM_BATCH_TRY(check_pair(f1, u1, el * (size_t)b->total));
  if (!b->p2.empty()) SGM_BATCH_TRY(check_pair(f2, u2, el * (size_t)b->off2.back()));
  const void* want[4] = {f1, u1, f2, u2};
  if (!b->exec || std::memcmp(want, b->cap, sizeof want) != 0) SGM_BATCH_TRY(capture(b, f1, u1, f2, u2));
  const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

}  // extern "C"
