// k_cheb_tc.cu - the Chebyshev axis of a space as a dense contraction on the tensor cores, for
// N <= 128 points (the small-N form of the Chebyshev transforms).
//
// Every Chebyshev-axis operation of Sec. 3.4.2 is a fixed N x N matrix applied to each column
// of the data (each real or imaginary part of each Fourier column):
//   scalar product   S_k = sum_j (pi / N) phi_k(x_j) f_j        (Gauss-Chebyshev quadrature)
//   forward (T_k)    c_k = sum_j 2 / (N c_k) T_k(x_j) f_j         (c_0 = 2, c_k = 1)
//   backward         u_j = sum_k phi_k(x_j) u_k                   (Eq. fast_shen, evaluated)
// with phi_k the Shen basis function (T_k - T_{k+2}, or the biharmonic combination of
// Eq. chebbiharmonic), x_j = cos(pi (2j+1) / (2N)), and zero rows for k past the basis.
//
// The kernel computes Y^T = X^T P^T with tcgen05.mma: M = 128 data columns per CTA (one per TMEM
// lane), N = the padded output rows, K = the padded input rows.  Products are BF16x3 split
// products with FP32 accumulation: X = Xh + Xl and P = Ph + Pl with BF16 parts, and
// Y = Xl Ph + Xh Pl + Xh Ph (the Xl Pl term, below 2^-16 of the product, is dropped).
//   * P^T is staged by one bulk copy (cp.async.bulk) of a host-built image that is already in
//     the K-major core-matrix layout (hi part, then lo part);
//   * X is loaded coalesced (128 consecutive columns per row), split into BF16 hi/lo in
//     registers and stored transposed to the K-major layout, one 16-byte core-matrix row per
//     store (conflict-free: a warp writes 512 contiguous bytes);
//   * one thread issues 3 * Kp / 16 MMAs into a 128 x Np FP32 TMEM accumulator and commits to
//     an mbarrier; the warps then read back their TMEM lanes (32 consecutive columns per warp)
//     with tcgen05.ld and store each output row as one coalesced 128-byte (FP32) or 256-byte
//     (FP64) access;
//   * the CTAs are persistent (one to four per SM), load the matrix once, and double-buffer
//     the tiles and the TMEM accumulators so that the MMAs of one tile overlap the epilogue of
//     the previous one and the loads of the next.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "convert.cuh"
#include "tc.cuh"

namespace sgm {

__device__ int g_tc_timeouts = 0;

namespace {

constexpr int kTcCols = 128;  // data columns per CTA = MMA M = TMEM lanes

__device__ __forceinline__ float as_f32(float x) { return x; }
__device__ __forceinline__ float as_f32(double x) { return narrow_f64(x); }

// FP32 accumulator to the output type (exact widening on the integer pipe for FP64)
template <typename TO> __device__ __forceinline__ TO from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_f32<double>(float v) { return widen_f32(v); }

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) {
  return (uint32_t)a | ((uint32_t)b << 16);
}

constexpr int kTcThreads = 512;  // 4 threads per column in the load phase, 16 warps

// Persistent: each CTA loads the matrix once, then walks over column tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Tile i (local count) is staged into A[i % 2] and multiplied into
// TMEM accumulator i % 2; its epilogue runs in the next iteration, while the tensor cores work on
// tile i + 1 and the loads of tile i + 2 are in flight behind the epilogue's stores.
template <typename TI, typename TO>
__global__ void __launch_bounds__(kTcThreads) k_cheb_tc(const TI* __restrict__ in, TO* __restrict__ out,
                                                        long ncols, int nin, int nout, int Kp, int Np, int tcols,
                                                        const unsigned char* __restrict__ img) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[3];   // [0] matrix copy, [1] / [2] MMA of even / odd tiles
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t abytes = 256u * (uint32_t)Kp;              // one BF16 part of a 128-column tile
  unsigned char* Bm = smem;                                 // matrix: Np x Kp hi, then lo
  const uint32_t half_img = (uint32_t)Np * (uint32_t)Kp * 2;
  unsigned char* A0 = smem + 2 * half_img;                  // tile buffers: [buf][hi | lo]
  const uint32_t lboA = (kTcCols / 8) * 128, lboB = (uint32_t)Np * 16;
  const long ntiles = (ncols + kTcCols - 1) / kTcCols;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bar[i], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, (uint32_t)tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bar[0], 2 * half_img);
    tc::bulk_g2s(Bm, img, 2 * half_img, &bar[0]);
  }
  bool ok = true;   // thread 0: every wait so far succeeded

  // load phase: column m, K groups kq, kq + 4, ...
  const int m = tid & (kTcCols - 1), kq = tid >> 7;
  const uint32_t row_off = (uint32_t)(m >> 3) * 128 + (uint32_t)(m & 7) * 16;
  // epilogue: TMEM lane quarter warp % 4 (32 columns), output-row chunks q = warp / 4 (mod 4)
  const int lq = warp & 3, qs = warp >> 2;
  const int ngroups = Kp / 8, nchunks = Np / 16;

  auto epilogue = [&](long tile, int buf) {
    const long c = tile * kTcCols + lq * 32 + (tid & 31);
    const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * (tcols / 2));
    for (int q = qs; q < nchunks; q += 4) {
      float v[16];
      tc::tmem_ld16(base + (uint32_t)(q * 16), v);
      if (c < ncols) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = q * 16 + i;
          if (k < nout) out[(long)k * ncols + c] = from_f32<TO>(v[i]);
        }
      }
    }
  };

  long prev = -1;
  int i = 0;
  for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
    const int buf = i & 1;
    unsigned char* Ah = A0 + (uint32_t)buf * 2 * abytes;
    unsigned char* Al = Ah + abytes;
    const long c = t * kTcCols + m;
    const bool cv = c < ncols;
#pragma unroll 2
    for (int kg = kq; kg < ngroups; kg += 4) {
      TI x[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int j = kg * 8 + r;
        x[r] = (cv && j < nin) ? in[(long)j * ncols + c] : (TI)0;
      }
      uint16_t h[8], l[8];
      // FP64 input is first rounded to FP32 on the integer pipe (its residual, 2^-24, is far
      // below the 2^-16 of the split); FP64 conversions would run at 1/64 of the FP32 rate
#pragma unroll
      for (int r = 0; r < 8; ++r) tc::split_bf16(as_f32(x[r]), h[r], l[r]);
      const uint32_t off = row_off + (uint32_t)kg * lboA;
      *reinterpret_cast<uint4*>(Ah + off) =
          make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
      *reinterpret_cast<uint4*>(Al + off) =
          make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (i == 0) ok = tc::mbar_wait(&bar[0], 0);
      if (ok) {
        const uint32_t idesc = tc::idesc_bf16(kTcCols, Np);
        const uint32_t ah = tc::smem_addr(Ah), al = tc::smem_addr(Al);
        const uint32_t bh = tc::smem_addr(Bm), bl = bh + half_img;
        const uint32_t d = tmem + (uint32_t)(buf * (tcols / 2));   // accumulators tcols / 2 >= Np apart
        for (int s = 0; s < Kp / 16; ++s) {
          const uint32_t oa = (uint32_t)s * 2 * lboA, ob = (uint32_t)s * 2 * lboB;
          const uint64_t dah = tc::smem_desc(ah + oa, lboA, 128), dal = tc::smem_desc(al + oa, lboA, 128);
          const uint64_t dbh = tc::smem_desc(bh + ob, lboB, 128), dbl = tc::smem_desc(bl + ob, lboB, 128);
          tc::mma_bf16(d, dal, dbh, idesc, s > 0 ? 1u : 0u);
          tc::mma_bf16(d, dah, dbl, idesc, 1u);
          tc::mma_bf16(d, dah, dbh, idesc, 1u);
        }
      }
      tc::mma_commit(&bar[1 + buf]);   // arrives at once if nothing was issued
    }
    if (prev >= 0) {
      const int pb = (i - 1) & 1;
      bool done = tc::mbar_wait(&bar[1 + pb], (uint32_t)(((i - 1) >> 1) & 1));
      done = __all_sync(0xffffffffu, done) != 0;
      if (!done && (tid & 31) == 0) atomicAdd(&g_tc_timeouts, 1);
      tc::fence_after_sync();
      if (done) epilogue(prev, pb);
      tc::fence_before_sync();
    }
    prev = t;
  }
  if (prev >= 0) {
    const int pb = (i - 1) & 1;
    bool done = tc::mbar_wait(&bar[1 + pb], (uint32_t)(((i - 1) >> 1) & 1));
    done = __all_sync(0xffffffffu, done) != 0;
    if (!done && (tid & 31) == 0) atomicAdd(&g_tc_timeouts, 1);
    tc::fence_after_sync();
    if (done) epilogue(prev, pb);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && !ok) {
    atomicAdd(&g_tc_timeouts, 1);
    tc::mbar_wait(&bar[0], 0);   // let a late bulk copy land before exit
  }
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)tcols);
}

// ---- host: the matrix image -------------------------------------------------------------
uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // inf / nan (never produced here)
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
double bf16_to_double(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

// T_k(x_j) = cos(pi k (2j + 1) / (2N)), argument reduced exactly modulo 4N
long double cheb_T(long k, long j, long N) {
  const long m = (k * (2 * j + 1)) % (4 * N);
  return cosl(3.141592653589793238462643383279502884L * (long double)m / (long double)(2 * N));
}

long double shen_phi(int basis, long k, long j, long N) {
  if (basis == kCheb) return cheb_T(k, j, N);
  if (basis == kDirichlet) return cheb_T(k, j, N) - cheb_T(k + 2, j, N);
  if (basis == kNeumann) {
    const long double r = (long double)k / (long double)(k + 2);
    return cheb_T(k, j, N) - r * r * cheb_T(k + 2, j, N);
  }
  const long double be = -2.0L * (k + 2) / (k + 3), ga = (long double)(k + 1) / (k + 3);
  return cheb_T(k, j, N) + be * cheb_T(k + 2, j, N) + ga * cheb_T(k + 4, j, N);
}

}  // namespace

int tc_pad16(int n) { return (n + 15) / 16 * 16; }

// image of P^T (output rows n < Np, input rows kk < Kp) in the K-major core-matrix layout,
// BF16 hi part followed by the lo part; mode kChebScalar / kChebForwardT / kChebBackward
// BF16 hi and lo images of an N x N matrix P (row = output row, column = input row), zero-padded
// to tc_pad16(N) and laid out in K-major core matrices for k_cheb_tc
std::vector<uint16_t> tc_matrix_image(const std::vector<long double>& P, int N) {
  const int Kp = tc_pad16(N), Np = tc_pad16(N);
  std::vector<uint16_t> img((size_t)2 * Np * Kp, 0);
  const size_t half = (size_t)Np * Kp;
  for (int n = 0; n < Np; ++n)
    for (int kk = 0; kk < Kp; ++kk) {
      const long double v = (n < N && kk < N) ? P[(size_t)n * N + kk] : 0.0L;
      const uint16_t h = bf16_rn((float)v);
      const uint16_t l = bf16_rn((float)((double)v - bf16_to_double(h)));
      const size_t off = ((size_t)(n / 8) * 128 + (size_t)(n % 8) * 16 + (size_t)(kk % 8) * 2 +
                          (size_t)(kk / 8) * (size_t)Np * 16) / 2;
      img[off] = h;
      img[half + off] = l;
    }
  return img;
}

std::vector<uint16_t> tc_cheb_image(int mode, int basis, int N) {
  const int nb = basis_count(basis, N);
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<long double> P((size_t)N * N, 0.0L);
  for (int n = 0; n < N; ++n)
    for (int kk = 0; kk < N; ++kk) {
      long double v = 0;
      if (mode == kChebBackward) {  // output row j = n, input row k = kk
        if (kk < nb) v = shen_phi(basis, kk, n, N);
      } else if (mode == kChebForwardT) {  // output row k = n, input row j = kk
        v = cheb_T(n, kk, N) * 2.0L / ((long double)N * (n == 0 ? 2.0L : 1.0L));
      } else if (n < nb) {
        v = shen_phi(basis, n, kk, N) * pi / (long double)N;
      }
      P[(size_t)n * N + kk] = v;
    }
  return tc_matrix_image(P, N);
}

// shared memory of one CTA: the matrix and two X tiles, BF16 hi and lo parts each
size_t tc_cheb_smem(int Kp, int Np) { return (size_t)4 * Np * Kp + (size_t)2 * 512 * Kp; }

template <typename TI, typename TO>
cudaError_t launch_cheb_tc(const void* in, void* out, long ncols, int N, const void* img, cudaStream_t s) {
  if (ncols <= 0) return cudaSuccess;
  const int Kp = tc_pad16(N), Np = tc_pad16(N);
  int tcols = 32;
  while (tcols < 2 * Np) tcols *= 2;   // two accumulators of Np FP32 columns
  const size_t smem = tc_cheb_smem(Kp, Np);
  cudaError_t e = cudaFuncSetAttribute(k_cheb_tc<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb_tc<TI, TO>, kTcThreads, smem)) != cudaSuccess)
    return e;
  // TMEM: at most 512 columns per SM among the resident CTAs
  per_sm = std::max(1, std::min(per_sm, 512 / tcols));
  const long ntiles = (ncols + kTcCols - 1) / kTcCols;
  const unsigned grid = (unsigned)std::min(ntiles, (long)sms * per_sm);
  k_cheb_tc<TI, TO><<<grid, kTcThreads, smem, s>>>((const TI*)in, (TO*)out, ncols, N, N, Kp, Np, tcols,
                                                   (const unsigned char*)img);
  return cudaGetLastError();
}

template cudaError_t launch_cheb_tc<float, float>(const void*, void*, long, int, const void*, cudaStream_t);
template cudaError_t launch_cheb_tc<float, double>(const void*, void*, long, int, const void*, cudaStream_t);
template cudaError_t launch_cheb_tc<double, float>(const void*, void*, long, int, const void*, cudaStream_t);

int tc_timeouts(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof v) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_tc_timeouts, &z, sizeof z) != cudaSuccess) return -1;
  }
  return v;
}

}  // namespace sgm
