// k_cnn.cu - the learned closure's kernels: periodic 3x3 convolutions (forward, backward with
// respect to the input and to the weights), AdamW, the MSE loss gradient, and the glue between
// Ginzburg-Landau states and network channels (spectral truncation, complex <-> 2 channels).
// The closure has no counterpart in the paper.
//
// One layer is the circular cross-correlation
//     y[b, o, i, j] = bias[o] + sum_{c, p, q} W[o, c, p, q] x[b, c, (i + p - 1) mod H, (j + q - 1) mod W]
// (p, q in 0..2), optionally followed by ReLU.  Activations and weights are stored in BF16,
// every product is accumulated in FP32; gradients are FP32.  The 32 -> 32 layers run as
// implicit GEMMs on the tensor cores (k_cnn_tc.cu); the 2 -> 32 and 32 -> 2 layers, whose GEMM
// has 2 rows or a K of 18, use the kernels below on the CUDA cores.  A CTA owns a 16 x 16 pixel
// tile of one sample: it stages the tile plus a one-pixel periodic halo of every input channel
// and the layer's weights in shared memory (FP32), and each thread accumulates all output
// channels of one pixel (forward and input gradient) or a few (output, input) channel pairs over
// the tile (weight gradient, partial sums added to the FP32 gradient with atomics).
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "../../include/sgm.h"
#include "common.cuh"

namespace sgm {

// the 32 -> 32 layers on the tensor cores (k_cnn_tc.cu)
template <typename TO>
cudaError_t launch_conv_tc_fwd(const __nv_bfloat16* x, const __nv_bfloat16* w, const float* bias, TO* y, int B, int H,
                               int W, bool relu, cudaStream_t s);
cudaError_t launch_conv_tc_bwd_data(const float* gy, const __nv_bfloat16* w, const __nv_bfloat16* mask, float* gx,
                                    int B, int H, int W, cudaStream_t s);
cudaError_t launch_conv_tc_wgrad(const float* gy, const __nv_bfloat16* x, float* gw, float* gb, int B, int H, int W,
                                 cudaStream_t s);

constexpr int kTile = 16;
constexpr int kHalo = kTile + 2;

__device__ __forceinline__ float ldf(const __nv_bfloat16* p, long i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldf(const float* p, long i) { return p[i]; }
// the network input (layer 0) may be FP32: the physical field itself, without a BF16 rounding

// ---- forward ---------------------------------------------------------------------------------
template <int CIN, int COUT, bool RELU, typename TO, typename TI>
__global__ void __launch_bounds__(256) k_conv_fwd(const TI* __restrict__ x, const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, TO* __restrict__ y, int H, int W) {
  extern __shared__ float sm[];
  float(*xs)[kHalo][kHalo] = reinterpret_cast<float(*)[kHalo][kHalo]>(sm);
  float* ws = sm + CIN * kHalo * kHalo;
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const long plane = (long)H * W;
  for (int t = threadIdx.x; t < COUT * CIN * 9; t += 256) ws[t] = __bfloat162float(w[t]);
  for (int t = threadIdx.x; t < CIN * kHalo * kHalo; t += 256) {
    const int c = t / (kHalo * kHalo), r = t % (kHalo * kHalo);
    const int hi = r / kHalo, hj = r % kHalo;
    const int gi = (i0 + hi - 1 + H) % H, gj = (j0 + hj - 1 + W) % W;
    xs[c][hi][hj] = ldf(x, ((long)b * CIN + c) * plane + (long)gi * W + gj);
  }
  __syncthreads();
  const int ty = threadIdx.x / kTile, tx = threadIdx.x % kTile;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
  for (int c = 0; c < CIN; ++c)
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float xv = xs[c][ty + p][tx + q];
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = fmaf(ws[(o * CIN + c) * 9 + p * 3 + q], xv, acc[o]);
      }
  const long pix = (long)(i0 + ty) * W + (j0 + tx);
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    const float v = RELU ? fmaxf(acc[o], 0.0f) : acc[o];
    if constexpr (sizeof(TO) == 2) y[((long)b * COUT + o) * plane + pix] = __float2bfloat16_rn(v);
    else y[((long)b * COUT + o) * plane + pix] = v;
  }
}

// ---- gradient with respect to the input ---------------------------------------------------------
// gx[b, c, i, j] = sum_{o, p, q} W[o, c, p, q] gy[b, o, i - p + 1, j - q + 1], times 1[x_in > 0]
// when the layer input is a ReLU output (mask != nullptr).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float* __restrict__ gy, const __nv_bfloat16* __restrict__ w,
                                                       const __nv_bfloat16* __restrict__ mask, float* __restrict__ gx,
                                                       int H, int W) {
  extern __shared__ float sm[];
  float(*gs)[kHalo][kHalo] = reinterpret_cast<float(*)[kHalo][kHalo]>(sm);
  float* ws = sm + COUT * kHalo * kHalo;
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const long plane = (long)H * W;
  for (int t = threadIdx.x; t < COUT * CIN * 9; t += 256) ws[t] = __bfloat162float(w[t]);
  for (int t = threadIdx.x; t < COUT * kHalo * kHalo; t += 256) {
    const int o = t / (kHalo * kHalo), r = t % (kHalo * kHalo);
    const int hi = r / kHalo, hj = r % kHalo;
    const int gi = (i0 + hi - 1 + H) % H, gj = (j0 + hj - 1 + W) % W;
    gs[o][hi][hj] = gy[((long)b * COUT + o) * plane + (long)gi * W + gj];
  }
  __syncthreads();
  const int ty = threadIdx.x / kTile, tx = threadIdx.x % kTile;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.0f;
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float gv = gs[o][ty + 2 - p][tx + 2 - q];   // gy at (i - p + 1, j - q + 1)
#pragma unroll
        for (int c = 0; c < CIN; ++c) acc[c] = fmaf(ws[(o * CIN + c) * 9 + p * 3 + q], gv, acc[c]);
      }
  const long pix = (long)(i0 + ty) * W + (j0 + tx);
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const long g = ((long)b * CIN + c) * plane + pix;
    float v = acc[c];
    if (mask && !(__bfloat162float(mask[g]) > 0.0f)) v = 0.0f;
    gx[g] = v;
  }
}

// ---- gradient with respect to the weights and the bias (accumulated) ------------------------------
template <int CIN, int COUT, typename TI>
__global__ void __launch_bounds__(256) k_conv_bwd_weights(const float* __restrict__ gy, const TI* __restrict__ x,
                                                          float* __restrict__ gw, float* __restrict__ gb, int H, int W) {
  extern __shared__ float sm[];
  float(*xs)[kHalo][kHalo] = reinterpret_cast<float(*)[kHalo][kHalo]>(sm);
  float(*gs)[kTile * kTile] = reinterpret_cast<float(*)[kTile * kTile]>(sm + CIN * kHalo * kHalo);
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const long plane = (long)H * W;
  for (int t = threadIdx.x; t < CIN * kHalo * kHalo; t += 256) {
    const int c = t / (kHalo * kHalo), r = t % (kHalo * kHalo);
    const int hi = r / kHalo, hj = r % kHalo;
    const int gi = (i0 + hi - 1 + H) % H, gj = (j0 + hj - 1 + W) % W;
    xs[c][hi][hj] = ldf(x, ((long)b * CIN + c) * plane + (long)gi * W + gj);
  }
  for (int t = threadIdx.x; t < COUT * kTile * kTile; t += 256) {
    const int o = t / (kTile * kTile), r = t % (kTile * kTile);
    gs[o][r] = gy[((long)b * COUT + o) * plane + (long)(i0 + r / kTile) * W + (j0 + r % kTile)];
  }
  __syncthreads();
  for (int item = threadIdx.x; item < COUT * CIN; item += 256) {
    const int o = item / CIN, c = item % CIN;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    float accb = 0.0f;
    for (int r = 0; r < kTile * kTile; ++r) {
      const float g = gs[o][r];
      const int ty = r / kTile, tx = r % kTile;
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[p * 3 + q] = fmaf(g, xs[c][ty + p][tx + q], acc[p * 3 + q]);
      accb += g;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(&gw[(o * CIN + c) * 9 + k], acc[k]);
    if (c == 0) atomicAdd(&gb[o], accb);
  }
}

// ---- AdamW on FP32 master weights, BF16 copy refreshed -------------------------------------------
__global__ void k_adamw(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                        float* __restrict__ m, float* __restrict__ v, long n, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1 / (sqrtf(vi / c2) + eps) + wd * w[i]);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

// ---- MSE: grad = 2 (out - target) / n, loss += sum (out - target)^2 / n ----------------------------
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, float* __restrict__ grad,
                      float* __restrict__ loss, long n) {
  float acc = 0.0f;
  const float inv = 1.0f / (float)n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float d = out[i] - target[i];
    grad[i] = 2.0f * d * inv;
    acc = fmaf(d * d, inv, acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// ---- spectral truncation of M_f x M_f coefficients to M_c x M_c (same wavenumbers) ----------------
__global__ void k_truncate(const float2* __restrict__ src, int Mf, float2* __restrict__ dst, int Mc, int B) {
  const long n = (long)B * Mc * Mc;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ((long)Mc * Mc));
    const int r = (int)((t / Mc) % Mc), j = (int)(t % Mc);
    const int lr = signed_wavenumber(r, Mc, 0), lj = signed_wavenumber(j, Mc, 0);
    const int fr = (lr + Mf) % Mf, fj = (lj + Mf) % Mf;
    dst[t] = src[((long)b * Mf + fr) * Mf + fj];
  }
}

// ---- complex field <-> (Re, Im) channels -------------------------------------------------------------
__global__ void k_pack(const float2* __restrict__ u, __nv_bfloat16* __restrict__ x, long plane, int B, float scale) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)B * plane; t += (long)gridDim.x * blockDim.x) {
    const long b = t / plane, p = t % plane;
    const float2 v = u[t];
    x[(b * 2) * plane + p] = __float2bfloat16_rn(v.x * scale);
    x[(b * 2 + 1) * plane + p] = __float2bfloat16_rn(v.y * scale);
  }
}
// ---- training batch: pool gather + symmetry transform + (Re, Im) channels -------------------------
// Output pixel (i, j) of sample b comes from the pool field idx[b] at the position the transform
// sends there: undo the reflections (i -> (M - i) mod M on a reflected axis), then the
// transposition, then the translation by (sx, sy); the value is multiplied by phase[b].
__global__ void k_augment_pack(const float2* __restrict__ u, const float2* __restrict__ d, int n, int M,
                               const int* __restrict__ idx, const float2* __restrict__ phase, int B, int sx, int sy,
                               int flags, float su, float sd, float* __restrict__ xu, float* __restrict__ xd) {
  const long plane = (long)M * M;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)B * plane; t += (long)gridDim.x * blockDim.x) {
    const int b = (int)(t / plane);
    const int p = (int)(t - (long)b * plane);
    int i = p / M, j = p - (p / M) * M;
    if (flags & SGM_AUG_FLIP0) i = (M - i) % M;
    if (flags & SGM_AUG_FLIP1) j = (M - j) % M;
    if (flags & SGM_AUG_TRANSPOSE) {
      const int k = i;
      i = j;
      j = k;
    }
    i = (i - sx % M + M) % M;
    j = (j - sy % M + M) % M;
    const int k = idx[b];
    float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    if (k >= 0 && k < n) {
      const float2 w = phase[b];
      const long src = (long)k * plane + (long)i * M + j;
      const float2 uv = u[src], dv = d[src];
      a = make_float2(uv.x * w.x - uv.y * w.y, uv.x * w.y + uv.y * w.x);
      c = make_float2(dv.x * w.x - dv.y * w.y, dv.x * w.y + dv.y * w.x);
    }
    xu[((long)b * 2) * plane + p] = su * a.x;
    xu[((long)b * 2 + 1) * plane + p] = su * a.y;
    xd[((long)b * 2) * plane + p] = sd * c.x;
    xd[((long)b * 2 + 1) * plane + p] = sd * c.y;
  }
}

__global__ void k_unpack_add(const float* __restrict__ d, float2* __restrict__ u, long plane, int B, float scale) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)B * plane; t += (long)gridDim.x * blockDim.x) {
    const long b = t / plane, p = t % plane;
    float2 v = u[t];
    v.x += scale * d[(b * 2) * plane + p];
    v.y += scale * d[(b * 2 + 1) * plane + p];
    u[t] = v;
  }
}

}  // namespace sgm

using namespace sgm;

namespace {
int shape_ok(int B, int Cin, int Cout, int H, int W) {
  if (B < 1 || H < kTile || W < kTile || H % kTile || W % kTile)
    return set_error(SGM_ERR_SIZE, "B >= 1 and H, W multiples of %d are required", kTile);
  const bool ok = (Cin == 2 && Cout == 32) || (Cin == 32 && Cout == 32) || (Cin == 32 && Cout == 2);
  if (!ok) return set_error(SGM_ERR_SIZE, "channel pair (%d, %d) not built (2->32, 32->32, 32->2)", Cin, Cout);
  return SGM_OK;
}
int launched(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return SGM_OK;
}
int grid_for(long n) { return (int)std::min<long>((n + 255) / 256, 152 * 16); }

template <typename K> int launch_smem(K kernel, size_t bytes, dim3 grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e == cudaSuccess ? SGM_OK : set_error(SGM_ERR_CUDA, "smem attribute: %s", cudaGetErrorString(e));
}
size_t fwd_smem(int ci, int co) { return sizeof(float) * (ci * kHalo * kHalo + co * ci * 9); }
size_t bwd_data_smem(int ci, int co) { return sizeof(float) * (co * kHalo * kHalo + co * ci * 9); }
size_t bwd_w_smem(int ci, int co) { return sizeof(float) * (ci * kHalo * kHalo + co * kTile * kTile); }
}  // namespace

extern "C" {

int sgm_conv3x3_forward(const void* x, const void* w, const float* bias, void* y, int B, int Cin, int Cout, int H,
                        int W, int flags, void* stream) {
  if (!x || !w || !bias || !y) return set_error(SGM_ERR_NULL, "NULL pointer");
  int st = shape_ok(B, Cin, Cout, H, W);
  if (st != SGM_OK) return st;
  const bool relu = flags & SGM_CONV_RELU, out_f32 = flags & SGM_CONV_OUT_F32, in_f32 = flags & SGM_CONV_IN_F32;
  if (in_f32 && Cin != 2) return set_error(SGM_ERR_SIZE, "FP32 input is built for the 2-channel input layer only");
  const dim3 grid(W / kTile, H / kTile, B);
  cudaStream_t s = (cudaStream_t)stream;
  const auto* wb = (const __nv_bfloat16*)w;
  const size_t sb = fwd_smem(Cin, Cout);
  auto go = [&](auto kernel, const auto* in, auto* out) {
    if (launch_smem(kernel, sb, grid, s) != SGM_OK) return;
    kernel<<<grid, 256, sb, s>>>(in, wb, bias, out, H, W);
  };
  using bf = __nv_bfloat16;
  // every (input type, output type, ReLU) combination of one channel pair
  auto pick = [&](auto ci, auto co) {
    constexpr int CI = decltype(ci)::value, CO = decltype(co)::value;
    auto with_out = [&](const auto* in) {
      using TI = std::remove_const_t<std::remove_pointer_t<decltype(in)>>;
      if (out_f32) {
        if (relu) go(k_conv_fwd<CI, CO, true, float, TI>, in, (float*)y);
        else go(k_conv_fwd<CI, CO, false, float, TI>, in, (float*)y);
      } else {
        if (relu) go(k_conv_fwd<CI, CO, true, bf, TI>, in, (bf*)y);
        else go(k_conv_fwd<CI, CO, false, bf, TI>, in, (bf*)y);
      }
    };
    if constexpr (CI == 2) {
      if (in_f32) with_out((const float*)x);
      else with_out((const bf*)x);
    } else {
      with_out((const bf*)x);
    }
  };
  if (Cin == 32 && Cout == 32) {
    const cudaError_t e = out_f32 ? launch_conv_tc_fwd<float>((const bf*)x, wb, bias, (float*)y, B, H, W, relu, s)
                                  : launch_conv_tc_fwd<bf>((const bf*)x, wb, bias, (bf*)y, B, H, W, relu, s);
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "conv forward: %s", cudaGetErrorString(e));
    return SGM_OK;
  }
  if (Cin == 2) pick(std::integral_constant<int, 2>{}, std::integral_constant<int, 32>{});
  else pick(std::integral_constant<int, 32>{}, std::integral_constant<int, 2>{});
  return launched("conv forward");
}

int sgm_conv3x3_backward_data(const float* gy, const void* w, const void* mask, float* gx, int B, int Cin, int Cout,
                              int H, int W, void* stream) {
  if (!gy || !w || !gx) return set_error(SGM_ERR_NULL, "NULL pointer");
  int st = shape_ok(B, Cin, Cout, H, W);
  if (st != SGM_OK) return st;
  const dim3 grid(W / kTile, H / kTile, B);
  cudaStream_t s = (cudaStream_t)stream;
  const auto* wb = (const __nv_bfloat16*)w;
  const auto* mb = (const __nv_bfloat16*)mask;
  const size_t sb = bwd_data_smem(Cin, Cout);
  auto go = [&](auto kernel) {
    if (launch_smem(kernel, sb, grid, s) != SGM_OK) return;
    kernel<<<grid, 256, sb, s>>>(gy, wb, mb, gx, H, W);
  };
  if (Cin == 32 && Cout == 32) {
    const cudaError_t e = launch_conv_tc_bwd_data(gy, wb, mb, gx, B, H, W, s);
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "conv backward data: %s", cudaGetErrorString(e));
    return SGM_OK;
  }
  if (Cin == 2) go(k_conv_bwd_data<2, 32>);
  else go(k_conv_bwd_data<32, 2>);
  return launched("conv backward data");
}

int sgm_conv3x3_backward_weights(const float* gy, const void* x, float* gw, float* gb, int B, int Cin, int Cout, int H,
                                 int W, int flags, void* stream) {
  if (!gy || !x || !gw || !gb) return set_error(SGM_ERR_NULL, "NULL pointer");
  int st = shape_ok(B, Cin, Cout, H, W);
  if (st != SGM_OK) return st;
  const bool in_f32 = flags & SGM_CONV_IN_F32;
  if (in_f32 && Cin != 2) return set_error(SGM_ERR_SIZE, "FP32 input is built for the 2-channel input layer only");
  const dim3 grid(W / kTile, H / kTile, B);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sb = bwd_w_smem(Cin, Cout);
  auto go = [&](auto kernel, const auto* in) {
    if (launch_smem(kernel, sb, grid, s) != SGM_OK) return;
    kernel<<<grid, 256, sb, s>>>(gy, in, gw, gb, H, W);
  };
  using bf = __nv_bfloat16;
  if (Cin == 2) {
    if (in_f32) go(k_conv_bwd_weights<2, 32, float>, (const float*)x);
    else go(k_conv_bwd_weights<2, 32, bf>, (const bf*)x);
  } else if (Cout == 32) {
    const cudaError_t e = launch_conv_tc_wgrad(gy, (const bf*)x, gw, gb, B, H, W, s);
    if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "conv backward weights: %s", cudaGetErrorString(e));
    return SGM_OK;
  } else {
    go(k_conv_bwd_weights<32, 2, bf>, (const bf*)x);
  }
  return launched("conv backward weights");
}

int sgm_adamw_step(float* w, void* w_bf16, const float* g, float* m, float* v, int64_t n, float lr, float beta1,
                   float beta2, float eps, float weight_decay, int step, void* stream) {
  if (!w || !g || !m || !v) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (n < 0 || step < 1) return set_error(SGM_ERR_ARG, "n >= 0 and step >= 1 required");
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  k_adamw<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16*)w_bf16, g, m, v, n, lr, beta1, beta2, eps,
                                                        weight_decay, c1, c2);
  return launched("adamw");
}

int sgm_mse_grad(const float* out, const float* target, float* grad, float* loss, int64_t n, void* stream) {
  if (!out || !target || !grad || !loss) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (n < 1) return set_error(SGM_ERR_ARG, "n >= 1 required");
  k_mse<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, target, grad, loss, n);
  return launched("mse");
}

int sgm_spectral_truncate(const void* src, int Mf, void* dst, int Mc, int B, void* stream) {
  if (!src || !dst) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (Mc < 1 || Mf < Mc || B < 1) return set_error(SGM_ERR_SIZE, "need 1 <= Mc <= Mf and B >= 1");
  const long n = (long)B * Mc * Mc;
  k_truncate<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>((const float2*)src, Mf, (float2*)dst, Mc, B);
  return launched("spectral truncate");
}

int sgm_pack_channels(const void* u, void* x, int B, int H, int W, float scale, void* stream) {
  if (!u || !x) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (B < 1 || H < 1 || W < 1) return set_error(SGM_ERR_SIZE, "bad shape");
  const long plane = (long)H * W;
  k_pack<<<grid_for(B * plane), 256, 0, (cudaStream_t)stream>>>((const float2*)u, (__nv_bfloat16*)x, plane, B, scale);
  return launched("pack channels");
}

int sgm_augment_pack(const void* u, const void* d, int n, int M, const int* idx, const void* phase, int B, int sx,
                     int sy, int flags, float su, float sd, float* xu, float* xd, void* stream) {
  if (!u || !d || !idx || !phase || !xu || !xd) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (n < 1 || M < 1 || B < 1) return set_error(SGM_ERR_SIZE, "n, M and B must be positive");
  if (sx < 0 || sy < 0 || (flags & ~(SGM_AUG_TRANSPOSE | SGM_AUG_FLIP0 | SGM_AUG_FLIP1)))
    return set_error(SGM_ERR_ARG, "shifts must be >= 0 and flags a combination of SGM_AUG_*");
  const long total = (long)B * M * M;
  k_augment_pack<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>((const float2*)u, (const float2*)d, n, M, idx,
                                                                    (const float2*)phase, B, sx, sy, flags, su, sd,
                                                                    xu, xd);
  return launched("augment pack");
}

int sgm_unpack_add(const float* d, void* u, int B, int H, int W, float scale, void* stream) {
  if (!d || !u) return set_error(SGM_ERR_NULL, "NULL pointer");
  if (B < 1 || H < 1 || W < 1) return set_error(SGM_ERR_SIZE, "bad shape");
  const long plane = (long)H * W;
  k_unpack_add<<<grid_for(B * plane), 256, 0, (cudaStream_t)stream>>>(d, (float2*)u, plane, B, scale);
  return launched("unpack add");
}

}  // extern "C"
