// k_stream.cu - the streaming pipeline of the physical-to-physical solves on FP32 spaces:
// persistent, TMA-fed transform kernels for the R2C/C2R last axis, the strided C2C axis and the
// Chebyshev axis, and the tensor-map encoder.
//
// The one-tile-per-CTA kernels of k_fast.cuh stage every tile through registers: a CTA waits for
// its whole tile before it computes, and the loads in flight per SM are bounded by the number of
// resident CTAs.  Here each persistent CTA owns kStages tile buffers in shared memory.  One thread
// issues the copy of a tile as one TMA operation (a 2-D or 3-D tensor box, cp.async.bulk.tensor, for
// the column tiles of the strided and Chebyshev passes; a 1-D bulk copy, cp.async.bulk, for the
// contiguous rows of the last axis), which lands without registers or load instructions and
// completes on the buffer's mbarrier.  While the CTA transforms one tile, the copy of its next tile
// is in flight.
//
// Layouts.  A column tile (16 neighbouring columns x L rows) lands as tile[e * 16 + t], and the
// column variant of the FFT engine (fft_cols) transforms it in place: its butterflies run across
// the 16 columns first, so every warp access is a run of consecutive words, with no padding and no
// copy.  The Chebyshev forward pass reads the even/odd (Makhoul) reordering of each line in its
// first FFT pass.  Row tiles land unpadded as rows[line * L + e]; they are copied into the padded
// buffer of fft_fast (the C2R pass forms the packed half-length input on the way), which frees the
// tile buffer for the next copy before the FFT starts.  The pre- and post-processing (DCT moments and Shen stencils,
// R2C/C2R twiddles, scaling) are those of the k_fast.cuh kernels.
//
// Every wait is bounded (tc::mbar_wait, ~1 s).  A CTA whose wait gives up counts the event in
// g_stream_timeouts, waits (bounded) for its other copies in flight and returns; the host reads
// the counter with sgm_tc_wait_timeouts.
#include <algorithm>
#include <mutex>

#include "k_fast.cuh"
#include "tma.cuh"

namespace sgm {

__device__ int g_stream_timeouts = 0;

namespace {

constexpr int kStages = 2;
constexpr int kTW = 16;   // columns per column tile

// barriers of a CTA's tile buffers: set-up, the bounded wait of an iteration, and the bounded
// drain of the copies still in flight after a wait gave up
struct Ring {
  uint64_t* bar;
  __device__ __forceinline__ void init() {
    if (threadIdx.x == 0) {
      for (int q = 0; q < kStages; ++q) tc::mbar_init(&bar[q], 1);
      tc::fence_mbar_init();
    }
    __syncthreads();
  }
  // true when the tile of iteration `it` has landed (all threads agree); counts a give-up
  __device__ __forceinline__ bool wait(int it) {
    const bool ok = tc::mbar_wait(&bar[it % kStages], (uint32_t)(it / kStages) & 1u);
    if (__syncthreads_and(ok)) return true;
    if (threadIdx.x == 0) atomicAdd(&g_stream_timeouts, 1);
    return false;
  }
  __device__ __forceinline__ void drain(long tile, long ntiles, int it) {
    if (tile < ntiles && threadIdx.x == 0)
      for (int k = 0; k < kStages; ++k) {
        if (tile + (long)k * gridDim.x >= ntiles) break;
        tc::mbar_wait(&bar[(it + k) % kStages], (uint32_t)((it + k) / kStages) & 1u);
      }
  }
};

template <int L>
constexpr size_t cols_smem() {
  return (size_t)kStages * L * kTW * sizeof(float2) + kStages * sizeof(uint64_t);
}
// the Chebyshev kernels add the per-row tables (DCT twiddles, two stencil coefficients)
template <int N>
constexpr size_t cheb_smem() {
  return cols_smem<N>() + (size_t)N * (sizeof(float2) + 2 * sizeof(float));
}

// Backward Chebyshev pass before the inverse FFT, in one sweep over a column tile
// (tile[e * 16 + t]): for each pair of rows (k, N - k), k = 1 .. N/2, a thread forms both Shen
// stencil outputs (Eq. fast_shen) from the coefficient rows and writes their DCT-III pre-twiddled
// values; every read precedes the one synchronisation before the writes.  Row 0 keeps its
// coefficient (no stencil term, no twiddle).  Rows past the basis hold zero.
template <int N>
__device__ __forceinline__ void cheb_backward_prepare_tile(float2* buf, int basis, const ChebTables<float>& tb) {
  using C = float2;
  constexpr int HALF = N / 2;
  static_assert((HALF * kTW) % kFastThreads == 0, "whole pairs per thread");
  constexpr int PH = HALF * kTW / kFastThreads;
  auto at = [](int t, int e) { return e * kTW + t; };
  auto stencil = [&](int t, int k) -> C {
    C v = buf[at(t, k)];
    if (basis == kDirichlet) {
      if (k >= 2) v = csub(v, buf[at(t, k - 2)]);
    } else if (basis == kNeumann) {
      if (k >= 2) {
        const float q = tb.c1[k - 2];
        const C u = buf[at(t, k - 2)];
        v.x -= q * u.x;
        v.y -= q * u.y;
      }
    } else if (basis == kBiharmonic) {
      if (k >= 2) {
        const float be = tb.c1[k - 2];
        const C u = buf[at(t, k - 2)];
        v.x += be * u.x;
        v.y += be * u.y;
      }
      if (k >= 4) {
        const float ga = tb.c2[k - 4];
        const C u = buf[at(t, k - 4)];
        v.x += ga * u.x;
        v.y += ga * u.y;
      }
    }
    return v;
  };
  C o1[PH], o2[PH];
#pragma unroll
  for (int q = 0; q < PH; ++q) {
    const int idx = threadIdx.x + q * kFastThreads;
    const int t = idx % kTW, k = 1 + idx / kTW;
    const C x = stencil(t, k);
    const C y = k < HALF ? stencil(t, N - k) : x;
    o1[q] = cscale(cmulc(mk<C>(x.x + y.y, x.y - y.x), tb.dctw[k]), 0.5f);
    o2[q] = cscale(cmulc(mk<C>(y.x + x.y, y.y - x.x), tb.dctw[N - k]), 0.5f);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PH; ++q) {
    const int idx = threadIdx.x + q * kFastThreads;
    const int t = idx % kTW, k = 1 + idx / kTW;
    buf[at(t, k)] = o1[q];
    if (k < HALF) buf[at(t, N - k)] = o2[q];
  }
  __syncthreads();
}

// ---- Chebyshev axis, column tiles of [N][inner] ------------------------------------------------
// MODE kChebScalar: tiles of the complex64 Fourier intermediate -> complex64 spectral array (scalar
// product: DCT moments + Shen stencil, both FP32; the elimination widens them exactly).  MODE kChebBackward: tiles of the complex64 spectral
// solution -> the same array in place (Shen stencil + DCT-III); rows past the basis read as zero.
template <int MODE, int N>
__global__ void __launch_bounds__(kFastThreads, 2) k_cheb_stream(const __grid_constant__ CUtensorMap map,
                                                                 void* __restrict__ out, long inner, int basis,
                                                                 const float2* __restrict__ twf,
                                                                 const float2* __restrict__ dctw) {
  using C = float2;
  constexpr uint32_t TILE_BYTES = (uint32_t)N * kTW * sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* tiles = reinterpret_cast<C*>(smem_raw);
  Ring ring{reinterpret_cast<uint64_t*>(smem_raw + (size_t)kStages * TILE_BYTES)};
  C* tw_s = reinterpret_cast<C*>(smem_raw + (size_t)kStages * TILE_BYTES + kStages * sizeof(uint64_t));
  float* c1_s = reinterpret_cast<float*>(tw_s + N);
  float* c2_s = c1_s + N;
  const long ntiles = (inner + kTW - 1) / kTW;
  const int nb = basis_count(basis, N);
  if (threadIdx.x == 0) tma::prefetch_map(&map);
  fill_cheb_tables<float>(tw_s, c1_s, c2_s, N, basis, dctw);
  const ChebTables<float> tabs{tw_s, c1_s, c2_s};
  ring.init();   // its synchronisation also publishes the tables
  auto issue = [&](long tile, int q) {
    tc::mbar_arrive_expect_tx(&ring.bar[q], TILE_BYTES);
    tma::load_2d(tiles + (size_t)q * N * kTW, &map, (int)(tile * kTW * 2), 0, &ring.bar[q]);
  };
  if (threadIdx.x == 0)
    for (int q = 0; q < kStages; ++q)
      if (blockIdx.x + (long)q * gridDim.x < ntiles) issue(blockIdx.x + (long)q * gridDim.x, q);
  int it = 0;
  long tile = blockIdx.x;
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    if (!ring.wait(it)) break;
    C* buf = tiles + (size_t)(it % kStages) * N * kTW;
    const long t0 = tile * kTW;
    const int nt = (int)min((long)kTW, inner - t0);
    if (MODE == kChebScalar) {
      // v_e = x_{2e} (e < N/2), x_{2(N-1-e)+1} (e >= N/2): the even/odd reordering, read by the
      // first FFT pass in place
      fft_cols<N, kTW, kFastThreads, false>(buf, twf, [](int e) { return e < N / 2 ? 2 * e : 2 * (N - 1 - e) + 1; });
      cheb_forward_finish<float, kChebScalar, float, N, true>(buf, nt, t0, inner, basis, 0, out, dctw, &tabs);
    } else {
      for (int idx = threadIdx.x + nb * kTW; idx < N * kTW; idx += kFastThreads) buf[idx] = make_float2(0.f, 0.f);
      __syncthreads();
      cheb_backward_prepare_tile<N>(buf, basis, tabs);
      fft_cols<N, kTW, kFastThreads, true>(buf, twf, [](int e) { return e; });
      for (int idx = threadIdx.x; idx < N * kTW; idx += kFastThreads) {
        const int j = idx / kTW, t = idx % kTW;
        if (t < nt) reinterpret_cast<C*>(out)[(long)j * inner + t0 + t] = buf[cheb_reord<N>(j) * kTW + t];
      }
    }
    __syncthreads();   // tile buffer free: load the CTA's tile kStages iterations ahead into it
    if (threadIdx.x == 0) {
      const long nx = tile + (long)kStages * gridDim.x;
      if (nx < ntiles) {
        tc::fence_proxy_async();
        issue(nx, it % kStages);
      }
    }
  }
  ring.drain(tile, ntiles, it);
}

// ---- strided axis of the padded intermediate [outer][L][hp], in place ---------------------------
// A tile is 16 neighbouring columns (last-axis indices t0 .. t0 + 15) of one plane o: the box
// {32 floats, L rows, 1 plane} of the tensor map over (2 hp floats, L, outer).  Boxes reaching past
// hp read zeros there, and only columns below hp are stored.
template <bool INV, int L>
__global__ void __launch_bounds__(kFastThreads, 2) k_strided_stream(const __grid_constant__ CUtensorMap map,
                                                                    float2* __restrict__ data, long outer, int hp,
                                                                    const float2* __restrict__ twf) {
  using C = float2;
  constexpr uint32_t TILE_BYTES = (uint32_t)L * kTW * sizeof(C);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* tiles = reinterpret_cast<C*>(smem_raw);
  Ring ring{reinterpret_cast<uint64_t*>(smem_raw + (size_t)kStages * TILE_BYTES)};
  const int tpp = (hp + kTW - 1) / kTW;   // tiles per plane
  const long ntiles = outer * tpp;
  if (threadIdx.x == 0) tma::prefetch_map(&map);
  ring.init();
  auto issue = [&](long tile, int q) {
    const int o = (int)(tile / tpp), kt = (int)(tile - (long)o * tpp);
    tc::mbar_arrive_expect_tx(&ring.bar[q], TILE_BYTES);
    tma::load_3d(tiles + (size_t)q * L * kTW, &map, kt * kTW * 2, 0, o, &ring.bar[q]);
  };
  if (threadIdx.x == 0)
    for (int q = 0; q < kStages; ++q)
      if (blockIdx.x + (long)q * gridDim.x < ntiles) issue(blockIdx.x + (long)q * gridDim.x, q);
  int it = 0;
  long tile = blockIdx.x;
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    if (!ring.wait(it)) break;
    C* buf = tiles + (size_t)(it % kStages) * L * kTW;
    const long o = tile / tpp;
    const int t0 = (int)(tile - o * tpp) * kTW;
    const int nt = min(kTW, hp - t0);
    fft_cols<L, kTW, kFastThreads, INV>(buf, twf, [](int e) { return e; });
    const float sc = INV ? 1.f : 1.f / (float)L;
    C* dst = data + o * L * hp + t0;
    for (int idx = threadIdx.x; idx < L * kTW; idx += kFastThreads) {
      const int i = idx / kTW, t = idx % kTW;
      if (t < nt) dst[(long)i * hp + t] = INV ? buf[idx] : cscale(buf[idx], sc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const long nx = tile + (long)kStages * gridDim.x;
      if (nx < ntiles) {
        tc::fence_proxy_async();
        issue(nx, it % kStages);
      }
    }
  }
  ring.drain(tile, ntiles, it);
}

// ---- rows of the contiguous last axis (R2C forward, C2R backward) --------------------------------
// A tile is LINES = 4096 / LF consecutive rows, copied by one 1-D bulk copy.  R2C: the input rows
// (L = 2 LF reals) are contiguous; the output rows hold H + 1 = LF + 1 coefficients at a row stride
// of hp complex values (hp >= H + 1, even, so that every row starts on a 16-byte boundary for the
// tensor maps of the next passes), the columns past H written as zero.  C2R: the input rows of
// stride hp are contiguous; the output rows are contiguous.
template <int MODE, int LF>
__global__ void __launch_bounds__(kFastThreads, 2) k_rows_stream(const void* __restrict__ in, void* __restrict__ out,
                                                                 long nrows, int hp, const float2* __restrict__ twf,
                                                                 const float2* __restrict__ tw_L) {
  using C = float2;
  constexpr int LINES = 4096 / LF;
  constexpr int LDP = row_ld(LF);
  constexpr int H = LF;
  constexpr int L = 2 * LF;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int row_elems = MODE == kRowR2C ? LF : hp;               // complex values per input row
  const int stage_elems = LINES * row_elems;
  C* stage = reinterpret_cast<C*>(smem_raw);
  C* buf = stage + (size_t)kStages * stage_elems;
  Ring ring{reinterpret_cast<uint64_t*>(buf + (size_t)LINES * LDP)};
  const long ntiles = (nrows + LINES - 1) / LINES;
  ring.init();
  auto issue = [&](long tile, int q) {
    const long row0 = tile * LINES;
    const int nl = (int)min((long)LINES, nrows - row0);
    const uint32_t bytes = (uint32_t)nl * row_elems * sizeof(C);
    tc::mbar_arrive_expect_tx(&ring.bar[q], bytes);
    tc::bulk_g2s(stage + (size_t)q * stage_elems, reinterpret_cast<const C*>(in) + row0 * row_elems, bytes,
                 &ring.bar[q]);
  };
  if (threadIdx.x == 0)
    for (int q = 0; q < kStages; ++q)
      if (blockIdx.x + (long)q * gridDim.x < ntiles) issue(blockIdx.x + (long)q * gridDim.x, q);
  int it = 0;
  long tile = blockIdx.x;
  for (; tile < ntiles; tile += gridDim.x, ++it) {
    if (!ring.wait(it)) break;
    const int q = it % kStages;
    const long row0 = tile * LINES;
    const int nl = (int)min((long)LINES, nrows - row0);
    const C* st = stage + (size_t)q * stage_elems;
    if (MODE == kRowR2C) {
      // into the padded buffer (reading the unpadded rows directly in the first FFT pass would
      // put lanes of neighbouring lines, 1 KB apart, on the same banks)
      for (int idx = threadIdx.x; idx < nl * LF; idx += kFastThreads) buf[(idx / LF) * LDP + padi(idx % LF)] = st[idx];
      __syncthreads();
    } else {
      for (int idx = threadIdx.x; idx < nl * H; idx += kFastThreads) {
        const int line = idx / H, k = idx - line * H;
        C x = st[line * hp + k], y = st[line * hp + (H - k)];
        if (k == 0) { x.y = 0; y.y = 0; }
        const C yc = cconj(y);
        const C e = cadd(x, yc);
        const C o = cmulc(csub(x, yc), __ldg(&tw_L[k]));
        buf[line * LDP + padi(k)] = mk<C>(e.x - o.y, e.y + o.x);
      }
      __syncthreads();
    }
    // stage q consumed
    if (threadIdx.x == 0) {
      const long nx = tile + (long)kStages * gridDim.x;
      if (nx < ntiles) {
        tc::fence_proxy_async();
        issue(nx, q);
      }
    }
    fft_fast<LF, LINES, kFastThreads, MODE == kRowC2R, LDP>(buf, nl, twf);
    if (MODE == kRowR2C) {
      // X_k from Z_k and Z_{H-k} (indices mod H): one thread forms the pair k, H - k from the same
      // two values, k < H/2 running over aligned blocks of 16 (conflict-free loads of Z_k)
      C* dst = reinterpret_cast<C*>(out) + row0 * hp;
      const float sc = 0.5f / (float)L;
      auto coef = [&](const C z, const C zp, int k) {
        const C zc = cconj(zp);
        const C e = cadd(z, zc);
        const C o = rot90<false>(cmul(__ldg(&tw_L[k]), csub(z, zc)));
        return cscale(cadd(e, o), sc);
      };
      constexpr int HH = H / 2;
      for (int idx = threadIdx.x; idx < nl * HH; idx += kFastThreads) {
        const int line = idx / HH, k = idx - line * HH;
        const C z = buf[line * LDP + padi(k)], zp = buf[line * LDP + padi(k == 0 ? 0 : H - k)];
        dst[(long)line * hp + k] = coef(z, zp, k);
        dst[(long)line * hp + H - k] = coef(zp, z, H - k);
      }
      // k = H/2, its own partner, and the padding columns H + 1 .. hp - 1
      for (int idx = threadIdx.x; idx < nl * (hp - H); idx += kFastThreads) {
        const int line = idx / (hp - H), c = idx - line * (hp - H);
        if (c == 0) {
          const C z = buf[line * LDP + padi(HH)];
          dst[(long)line * hp + HH] = coef(z, z, HH);
        } else {
          dst[(long)line * hp + H + c] = mk<C>(0.f, 0.f);
        }
      }
    } else {
      C* dst = reinterpret_cast<C*>(out) + row0 * LF;
      for (int idx = threadIdx.x; idx < nl * LF; idx += kFastThreads) dst[idx] = buf[(idx / LF) * LDP + padi(idx % LF)];
    }
    __syncthreads();   // work buffer free for the next tile
  }
  ring.drain(tile, ntiles, it);
}

// grid of a persistent kernel: the resident CTAs of all SMs, at most one per tile
template <typename K>
cudaError_t persistent_launch_params(K kernel, size_t smem, long ntiles, unsigned* grid) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFastThreads, smem);
  *grid = (unsigned)std::max(1L, std::min(ntiles, (long)std::max(1, per_sm) * std::max(1, sms)));
  return e;
}

template <int MODE, int N>
cudaError_t launch_cheb_n(const CUtensorMap& map, void* out, long inner, int basis, const float2* twf,
                          const float2* dctw, cudaStream_t s) {
  const size_t smem = cheb_smem<N>();
  unsigned grid = 1;
  cudaError_t e = persistent_launch_params(k_cheb_stream<MODE, N>, smem, (inner + kTW - 1) / kTW, &grid);
  if (e != cudaSuccess) return e;
  k_cheb_stream<MODE, N><<<grid, kFastThreads, smem, s>>>(map, out, inner, basis, twf, dctw);
  return cudaGetLastError();
}

template <bool INV, int L>
cudaError_t launch_strided_l(const CUtensorMap& map, float2* data, long outer, int hp, const float2* twf,
                             cudaStream_t s) {
  const size_t smem = cols_smem<L>();
  unsigned grid = 1;
  cudaError_t e = persistent_launch_params(k_strided_stream<INV, L>, smem, outer * ((hp + kTW - 1) / kTW), &grid);
  if (e != cudaSuccess) return e;
  k_strided_stream<INV, L><<<grid, kFastThreads, smem, s>>>(map, data, outer, hp, twf);
  return cudaGetLastError();
}

template <int MODE, int LF>
cudaError_t launch_rows_lf(const void* in, void* out, long nrows, int hp, const float2* twf, const float2* tw_L,
                           cudaStream_t s) {
  constexpr int LINES = 4096 / LF;
  const size_t stage = (size_t)LINES * (MODE == kRowR2C ? LF : hp) * sizeof(float2);
  const size_t smem = kStages * stage + (size_t)LINES * row_ld(LF) * sizeof(float2) + kStages * sizeof(uint64_t);
  unsigned grid = 1;
  cudaError_t e = persistent_launch_params(k_rows_stream<MODE, LF>, smem, (nrows + LINES - 1) / LINES, &grid);
  if (e != cudaSuccess) return e;
  k_rows_stream<MODE, LF><<<grid, kFastThreads, smem, s>>>(in, out, nrows, hp, twf, tw_L);
  return cudaGetLastError();
}

}  // namespace

// Lengths with a streaming kernel: a column tile is one TMA box of at most 256 rows; a row tile
// holds 4096 / LF rows of the packed half length LF.
bool cheb_stream_length(int N) { return N == 64 || N == 128 || N == 256; }
bool strided_stream_length(int L) { return L == 32 || L == 64 || L == 128 || L == 256; }
bool rows_stream_length(int LF) { return LF == 32 || LF == 64 || LF == 128 || LF == 256 || LF == 512; }

// mode kChebScalar: map over the complex64 Fourier intermediate (floats), out complex64 spectral;
// mode kChebBackward: map over the complex64 spectral solution (floats), out the same array.
cudaError_t launch_cheb_stream(int mode, int N, const CUtensorMap& map, void* out, long inner, int basis,
                               const float2* twf, const float2* dctw, cudaStream_t s) {
  if (inner <= 0) return cudaSuccess;
#define SGM_CS(n)                                                                                  \
  case n:                                                                                          \
    return mode == kChebScalar ? launch_cheb_n<kChebScalar, n>(map, out, inner, basis, twf, dctw, s) \
                               : launch_cheb_n<kChebBackward, n>(map, out, inner, basis, twf, dctw, s);
  switch (N) {
    SGM_CS(64) SGM_CS(128) SGM_CS(256)
    default: return cudaErrorInvalidValue;
  }
#undef SGM_CS
}

cudaError_t launch_strided_stream(bool inverse, int L, const CUtensorMap& map, float2* data, long outer, int hp,
                                  const float2* twf, cudaStream_t s) {
  if (outer <= 0) return cudaSuccess;
#define SGM_SS(n)                                                            \
  case n:                                                                    \
    return inverse ? launch_strided_l<true, n>(map, data, outer, hp, twf, s) \
                   : launch_strided_l<false, n>(map, data, outer, hp, twf, s);
  switch (L) {
    SGM_SS(32) SGM_SS(64) SGM_SS(128) SGM_SS(256)
    default: return cudaErrorInvalidValue;
  }
#undef SGM_SS
}

cudaError_t launch_rows_stream(int mode, int LF, const void* in, void* out, long nrows, int hp, const float2* twf,
                               const float2* tw_L, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
#define SGM_RS(n)                                                                       \
  case n:                                                                               \
    return mode == kRowR2C ? launch_rows_lf<kRowR2C, n>(in, out, nrows, hp, twf, tw_L, s) \
                           : launch_rows_lf<kRowC2R, n>(in, out, nrows, hp, twf, tw_L, s);
  switch (LF) {
    SGM_RS(32) SGM_RS(64) SGM_RS(128) SGM_RS(256) SGM_RS(512)
    default: return cudaErrorInvalidValue;
  }
#undef SGM_RS
}

int stream_timeouts(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_stream_timeouts, sizeof v) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_stream_timeouts, &z, sizeof z) != cudaSuccess) return -1;
  }
  return v;
}

cudaError_t encode_tiled_map(CUtensorMap* map, CUtensorMapDataType dtype, int rank, const void* base,
                             const uint64_t* dims, const uint64_t* strides, const uint32_t* box) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static cudaError_t look = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    look = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (look == cudaSuccess && q != cudaDriverEntryPointSuccess) look = cudaErrorSymbolNotFound;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (look != cudaSuccess || !fn) return look != cudaSuccess ? look : cudaErrorSymbolNotFound;
  cuuint64_t d[5];
  cuuint64_t st[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  const CUresult r = fn(map, dtype, (cuuint32_t)rank, const_cast<void*>(base), d, st, bx, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace sgm
