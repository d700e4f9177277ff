// k_cnn_tc.cu - the 32 -> 32 channel layers of the learned closure on the tcgen05 tensor cores.
//
// A periodic 3x3 layer with 32 input and 32 output channels is a GEMM over the im2col patches:
//   forward          y[p, o]  = bias[o] + sum_k A[p, k] Wf[o, k],  A[p, (c,t)] = x[c, p + d_t]
//   input gradient   gx[p, c] = sum_k A[p, k] Wb[c, k],             A[p, (o,t)] = gy[o, p + d_t]
//                    with Wb[c, (o,t)] = W[o, c, 8 - t] (the flipped kernel), times the ReLU mask
//   weight gradient  gW[o, (c,t)] = sum_p gy[o, p] x[c, p + d_t]   (sum over every pixel p)
// where k = 9 c + t, t = 3 p + q is the tap and d_t = (p - 1, q - 1) its periodic offset.
// Activations and weights are BF16, so the forward products are exact; the FP32 gradients are
// split into BF16 hi + lo parts (two MMAs, relative error of hi + lo below 2^-16).  Every sum is
// accumulated in FP32 in tensor memory.
//
// Forward / input gradient (k_conv_tc): one CTA per 128 consecutive pixels of one sample
// (M = 128), N = 32 channels, K = 288 in 18 MMAs of K = 16.  The weights are staged as the B
// operand in the K-major core-matrix layout, the CTA's im2col tile as the A operand (gathered
// from the L2-resident activations), and the epilogue reads one TMEM lane per pixel, so each
// output channel is stored as a coalesced row of 32 pixels per warp.
// Weight gradient (k_conv_tc_wgrad): M = 128 of the 288 (c, t) rows (three tiles, the last one
// padded), N = 32 output channels, the pixels are the reduction dimension in chunks of 64; each
// CTA reduces a range of pixels and adds its 128 x 32 partial sums to gW with FP32 atomics.
#include <cuda_bf16.h>

#include "../../include/sgm.h"
#include "common.cuh"
#include "tc.cuh"

namespace sgm {

__device__ int g_cnn_tc_timeouts = 0;

namespace {

constexpr int kC = 32;          // channels of the hidden layers
constexpr int kK = 9 * kC;      // 288 = (channel, tap)
constexpr int kKG = kK / 8;     // 36 core-matrix columns of 8 BF16
constexpr int kPix = 128;       // pixels per CTA (MMA M)
constexpr uint32_t kLboM128 = (kPix / 8) * 128;  // K-direction stride of a 128-row operand
constexpr uint32_t kLboN32 = (kC / 8) * 128;     // K-direction stride of a 32-row operand
constexpr uint32_t kBBytes = kC * kK * 2;        // 18432: weights, one BF16 part
constexpr uint32_t kABytes = kPix * kK * 2;      // 73728: im2col tile, one BF16 part

__device__ __forceinline__ uint16_t bits(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
__device__ __forceinline__ uint32_t pk(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }
// byte offset of element (row r, k) in a K-major core-matrix operand with K-direction stride lbo
__device__ __forceinline__ uint32_t cm_off(int r, int k, uint32_t lbo) {
  return (uint32_t)(r >> 3) * 128 + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2 + (uint32_t)(k >> 3) * lbo;
}

// bounded wait for an MMA commit; false (and a recorded timeout) if it gave up, warp-uniform
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t parity) {
  bool done = tc::mbar_wait(bar, parity);
  done = __all_sync(0xffffffffu, done) != 0;
  if (!done && (threadIdx.x & 31) == 0) atomicAdd(&g_cnn_tc_timeouts, 1);
  tc::fence_after_sync();
  return done;
}

// MODE 0: forward (in = x BF16, out = y TO, bias, ReLU); MODE 1: input gradient (in = gy FP32,
// out = gx FP32, optional BF16 mask: gx = 0 where mask <= 0)
template <int MODE, typename TO>
__global__ void __launch_bounds__(256) k_conv_tc(const void* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                 const float* __restrict__ bias, const __nv_bfloat16* __restrict__ mask,
                                                 TO* __restrict__ out, int H, int W, int relu) {
  constexpr int NPART = MODE == 0 ? 1 : 2;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  unsigned char* Bs = smem;
  unsigned char* As = smem + kBBytes;   // [part][128 x 288]
  const int tid = threadIdx.x, warp = tid >> 5;
  const long plane = (long)H * W;
  const long p0 = (long)blockIdx.x * kPix;
  const long b = p0 / plane;
  const long r0 = p0 - b * plane;

  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 32);

  // B operand: row n (output channel of the GEMM), k = 9 c' + t
  for (int e = tid; e < kC * kKG; e += 256) {
    const int n = e / kKG, kg = e - n * kKG;
    uint16_t v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int k = kg * 8 + r, c = k / 9, t = k - 9 * c;
      v[r] = MODE == 0 ? bits(w[(n * kC + c) * 9 + t]) : bits(w[(c * kC + n) * 9 + (8 - t)]);
    }
    *reinterpret_cast<uint4*>(Bs + cm_off(n, kg * 8, kLboN32)) =
        make_uint4(pk(v[0], v[1]), pk(v[2], v[3]), pk(v[4], v[5]), pk(v[6], v[7]));
  }
  // A operand: row m = pixel, k = 9 c + t: the input channel c at the pixel shifted by tap t.
  // One item = 8 consecutive k of one pixel (a 16-byte core-matrix row); a warp takes 32
  // consecutive pixels, so its gathers are coalesced and its stores fill 512 contiguous bytes.
  // The input gradient stages K in two halves through the same buffer (hi and lo parts of 144
  // columns each), which keeps the CTA at 92 KB of shared memory, two CTAs per SM.
  constexpr int NHALF = MODE == 0 ? 1 : 2, KGH = kKG / NHALF;
  const uint32_t part_bytes = (uint32_t)kPix * KGH * 16;
  bool ok = true;
  uint32_t tmem = 0;
  for (int hf = 0; hf < NHALF; ++hf) {
    for (int e = tid; e < kPix * KGH; e += 256) {
      const int m = e & (kPix - 1), kgl = e >> 7, kg = hf * KGH + kgl;
      const long rem = r0 + m;
      const int i = (int)(rem / W), j = (int)(rem - (long)i * W);
      // wrapped neighbour rows (as element offsets) and columns of the pixel
      const int im = i == 0 ? H - 1 : i - 1, ip = i == H - 1 ? 0 : i + 1;
      const int jm = j == 0 ? W - 1 : j - 1, jp = j == W - 1 ? 0 : j + 1;
      const long row0 = (long)im * W, row1 = (long)i * W, row2 = (long)ip * W;
      int c = (kg * 8) / 9, t = kg * 8 - 9 * c;
      uint16_t h[8], l[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int p = t >= 6 ? 2 : (t >= 3 ? 1 : 0), q = t - 3 * p;
        const long g = (b * kC + c) * plane + (p == 0 ? row0 : (p == 1 ? row1 : row2)) + (q == 0 ? jm : (q == 1 ? j : jp));
        if constexpr (MODE == 0) {
          h[r] = bits(reinterpret_cast<const __nv_bfloat16*>(in)[g]);
        } else {
          tc::split_bf16(reinterpret_cast<const float*>(in)[g], h[r], l[r]);
        }
        if (++t == 9) {
          t = 0;
          ++c;
        }
      }
      const uint32_t off = cm_off(m, kgl * 8, kLboM128);
      *reinterpret_cast<uint4*>(As + off) = make_uint4(pk(h[0], h[1]), pk(h[2], h[3]), pk(h[4], h[5]), pk(h[6], h[7]));
      if constexpr (MODE == 1)
        *reinterpret_cast<uint4*>(As + part_bytes + off) =
            make_uint4(pk(l[0], l[1]), pk(l[2], l[3]), pk(l[4], l[5]), pk(l[6], l[7]));
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem = tmem_slot;
    if (tid == 0) {
      const uint32_t idesc = tc::idesc_bf16(kPix, kC);
      const uint32_t a0 = tc::smem_addr(As), bb = tc::smem_addr(Bs);
      for (int s = 0; s < KGH / 2; ++s) {
        const int sg = hf * (KGH / 2) + s;   // K step within the full 288
        const uint64_t db = tc::smem_desc(bb + (uint32_t)sg * 2 * kLboN32, kLboN32, 128);
#pragma unroll
        for (int part = 0; part < (MODE == 0 ? 1 : 2); ++part) {
          const uint64_t da = tc::smem_desc(a0 + (uint32_t)part * part_bytes + (uint32_t)s * 2 * kLboM128, kLboM128, 128);
          tc::mma_bf16(tmem, da, db, idesc, (sg > 0 || part > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&bar);
    }
    // the next half overwrites the A operand: wait for these MMAs first
    ok = wait_mma(&bar, (uint32_t)hf) && ok;
    tc::fence_before_sync();
  }
  if (ok) {
    const int lq = warp & 3, n0 = (warp >> 2) * 16;
    const int m = lq * 32 + (tid & 31);
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)n0, v);
    const long pix = r0 + m;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int n = n0 + r;
      const long g = (b * kC + n) * plane + pix;
      float val = v[r];
      if constexpr (MODE == 0) {
        val += bias[n];
        if (relu) val = fmaxf(val, 0.0f);
        if constexpr (sizeof(TO) == 2) out[g] = __float2bfloat16_rn(val);
        else out[g] = val;
      } else {
        if (mask && !(__bfloat162float(mask[g]) > 0.0f)) val = 0.0f;
        out[g] = val;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

constexpr int kWChunk = 64;            // pixels per MMA chunk of the weight gradient
constexpr int kWChunksPerCta = 2;      // 128 pixels per CTA: enough CTAs to fill the SMs
constexpr uint32_t kWA = kPix * kWChunk * 2;   // 16 KB: 128 (c, t) rows x 64 pixels
constexpr uint32_t kWB = kC * kWChunk * 2;     // 4 KB: 32 channels x 64 pixels, one part

__global__ void __launch_bounds__(256) k_conv_tc_wgrad(const float* __restrict__ gy, const __nv_bfloat16* __restrict__ x,
                                                       float* __restrict__ gw, float* __restrict__ gb, int H, int W,
                                                       long nchunks) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  unsigned char* As = smem;
  unsigned char* Bh = smem + kWA;
  unsigned char* Bl = Bh + kWB;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = blockIdx.x;                         // rows m = 128 mt + 0..127 of the 288
  const long plane = (long)H * W;
  const long c0 = (long)blockIdx.y * kWChunksPerCta;
  const long c1 = c0 + kWChunksPerCta < nchunks ? c0 + kWChunksPerCta : nchunks;

  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc::idesc_bf16(kPix, kC);
  float bsum = 0.0f;          // bias gradient of channel tid & 31 (CTAs of the first row tile)
  bool ok = true;
  uint32_t phase = 0;
  for (long ch = c0; ch < c1; ++ch) {
    const long q0 = ch * kWChunk;                  // first pixel of the chunk (one sample)
    const long b = q0 / plane;
    const long r0 = q0 - b * plane;
    // A: row m = (c, t), 8 consecutive pixels per core-matrix row
    for (int e = tid; e < kPix * (kWChunk / 8); e += 256) {
      const int m = e & (kPix - 1), kg = e >> 7;
      const int mm = mt * kPix + m;
      uint16_t v[8];
      if (mm < kK) {
        // 8 consecutive pixels of one row (W is a multiple of 16), shifted by tap t
        const int c = mm / 9, t = mm - 9 * c, p = t / 3, q = t - 3 * p;
        const long rem = r0 + kg * 8;
        const int i = (int)(rem / W), j0 = (int)(rem - (long)i * W);
        int ii = i + p - 1;
        ii = ii < 0 ? ii + H : (ii >= H ? ii - H : ii);
        const __nv_bfloat16* row = x + (b * kC + c) * plane + (long)ii * W;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          int jj = j0 + r + q - 1;
          jj = jj < 0 ? jj + W : (jj >= W ? jj - W : jj);
          v[r] = bits(row[jj]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = 0;
      }
      *reinterpret_cast<uint4*>(As + cm_off(m, kg * 8, kLboM128)) =
          make_uint4(pk(v[0], v[1]), pk(v[2], v[3]), pk(v[4], v[5]), pk(v[6], v[7]));
    }
    // B: row n = output channel, gy split into BF16 hi and lo parts
    {
      const int n = tid & 31, kg = tid >> 5;
      const float* src = gy + (b * kC + n) * plane + r0 + kg * 8;
      uint16_t h[8], l[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float g = src[r];
        if (mt == 0) bsum += g;
        tc::split_bf16(g, h[r], l[r]);
      }
      const uint32_t off = cm_off(n, kg * 8, kLboN32);
      *reinterpret_cast<uint4*>(Bh + off) = make_uint4(pk(h[0], h[1]), pk(h[2], h[3]), pk(h[4], h[5]), pk(h[6], h[7]));
      *reinterpret_cast<uint4*>(Bl + off) = make_uint4(pk(l[0], l[1]), pk(l[2], l[3]), pk(l[4], l[5]), pk(l[6], l[7]));
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(As), bh = tc::smem_addr(Bh), bl = tc::smem_addr(Bl);
      for (int s = 0; s < kWChunk / 16; ++s) {
        const uint64_t da = tc::smem_desc(a0 + (uint32_t)s * 2 * kLboM128, kLboM128, 128);
        const uint64_t dh = tc::smem_desc(bh + (uint32_t)s * 2 * kLboN32, kLboN32, 128);
        const uint64_t dl = tc::smem_desc(bl + (uint32_t)s * 2 * kLboN32, kLboN32, 128);
        tc::mma_bf16(tmem, da, dl, idesc, (ch > c0 || s > 0) ? 1u : 0u);
        tc::mma_bf16(tmem, da, dh, idesc, 1u);
      }
      tc::mma_commit(&bar);
    }
    // the next chunk overwrites the operands: wait for these MMAs first
    ok = wait_mma(&bar, phase) && ok;
    phase ^= 1u;
    tc::fence_before_sync();
  }
  if (ok && c1 > c0) {
    const int lq = warp & 3, n0 = (warp >> 2) * 16;
    const int mm = mt * kPix + lq * 32 + (tid & 31);
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)n0, v);
    if (mm < kK) {
#pragma unroll
      for (int r = 0; r < 16; ++r) atomicAdd(&gw[(n0 + r) * kK + mm], v[r]);
    }
  }
  if (mt == 0) atomicAdd(&gb[tid & 31], bsum);   // 8 threads hold partial sums of each channel
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

}  // namespace

size_t conv_tc_smem(int /*mode*/) { return kBBytes + kABytes; }   // 92 KB: the A buffer holds 288 (or 2 x 144) columns

// forward of a 32 -> 32 layer; H * W must be a multiple of 128
template <typename TO>
cudaError_t launch_conv_tc_fwd(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, TO* y, int B, int H,
                               int W, bool relu, cudaStream_t s) {
  const size_t smem = conv_tc_smem(0);
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<0, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((long)B * H * W / kPix);
  k_conv_tc<0, TO><<<grid, 256, smem, s>>>(x, w, bias, nullptr, y, H, W, relu ? 1 : 0);
  return cudaGetLastError();
}
template cudaError_t launch_conv_tc_fwd<float>(const __nv_bfloat16*, const __nv_bfloat16*, const float*, float*, int,
                                               int, int, bool, cudaStream_t);
template cudaError_t launch_conv_tc_fwd<__nv_bfloat16>(const __nv_bfloat16*, const __nv_bfloat16*, const float*,
                                                       __nv_bfloat16*, int, int, int, bool, cudaStream_t);

cudaError_t launch_conv_tc_bwd_data(const float* gy, const __nv_bfloat16* w, const __nv_bfloat16* mask, float* gx,
                                    int B, int H, int W, cudaStream_t s) {
  const size_t smem = conv_tc_smem(1);
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((long)B * H * W / kPix);
  k_conv_tc<1, float><<<grid, 256, smem, s>>>(gy, w, nullptr, mask, gx, H, W, 0);
  return cudaGetLastError();
}

// adds the weight and bias gradients of a 32 -> 32 layer into gw, gb; H * W a multiple of 64
cudaError_t launch_conv_tc_wgrad(const float* gy, const __nv_bfloat16* x, float* gw, float* gb, int B, int H, int W,
                                 cudaStream_t s) {
  const long nchunks = (long)B * H * W / kWChunk;
  const dim3 grid(3, (unsigned)((nchunks + kWChunksPerCta - 1) / kWChunksPerCta));
  const size_t smem = kWA + 2 * kWB;
  k_conv_tc_wgrad<<<grid, 256, smem, s>>>(gy, x, gw, gb, H, W, nchunks);
  return cudaGetLastError();
}

int cnn_tc_timeouts(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_cnn_tc_timeouts, sizeof v) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_cnn_tc_timeouts, &z, sizeof z) != cudaSuccess) return -1;
  }
  return v;
}

}  // namespace sgm
