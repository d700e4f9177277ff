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
};
size_t batch_problem_bytes();
template <typename T>
cudaError_t launch_batch(const void* f, void* u, int nprob, int nslots, int Nmax, const void* probs,
                         const int* by_slot, const void* plans, const void* pool, const long* wbase, double* S,
                         double* U, double* scratch, const long* sbase, cudaStream_t s);

}  // namespace sgm

using namespace sgm;

struct sgm_batch {
  static constexpr uint32_t kMagic = 0x53474231u;
  uint32_t magic = kMagic;
  int device = 0;
  int prec = SGM_F64;
  int nprob = 0, Nmax = 0;
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

template <typename T> int build(sgm_batch* b, const int64_t* n, const double* alpha) {
  const int P = b->nprob;
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return n[x] > n[y]; });
  std::map<int, int> size_index;   // N -> plan index
  std::vector<FftPlan> plans;
  std::vector<cplx<T>> pool;
  std::vector<int> tw_off, dct_off;
  std::vector<BatchProblemH> probs(P);
  for (int p = 0; p < P; ++p) {
    const int N = (int)n[p];
    if (!size_index.count(N)) {
      size_index[N] = (int)plans.size();
      plans.push_back(host_plan(N));
      tw_off.push_back((int)pool.size());
      push_twiddles<T>(pool, N, (long double)N / 2.0L);    // exp(-2 pi i k / N)
      dct_off.push_back((int)pool.size());
      push_twiddles<T>(pool, N, 2.0L * N);                 // exp(-i pi k / (2N))
    }
    const int pi = size_index[N];
    probs[p] = {N, 0, (long)b->offsets[p], alpha[p], tw_off[pi], dct_off[pi], pi};
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
  static_assert(sizeof(BatchProblemH) == 40, "BatchProblem layout");
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
                      ? launch_batch<float>(f, u, b->nprob, b->nprob, b->Nmax, b->probs, b->by_slot, b->plans, b->pool,
                                            b->wbase, b->S, b->U, b->scratch, b->sbase, s)
                      : launch_batch<double>(f, u, b->nprob, b->nprob, b->Nmax, b->probs, b->by_slot, b->plans, b->pool,
                                             b->wbase, b->S, b->U, b->scratch, b->sbase, s);
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "batch launch: %s", cudaGetErrorString(e));
  return SGM_OK;
}

}  // extern "C"
