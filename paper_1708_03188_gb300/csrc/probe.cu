// probe.cu - sgm_alu_probe: a fused multiply-add throughput probe, so that the FP64 and FP32
// ALU peaks the eliminations and the Ginzburg-Landau passes are measured against come from
// the GPU that runs them, not from a datasheet.
//
// Every thread runs CH independent chains a_q <- fma(a_q, x, y) for `iters` rounds (2 flops
// per FMA).  x and y are kernel arguments and the chains' sum is written to `sink`, so the
// compiler can neither fold nor drop the work.  With CH = 8 independent chains per thread
// and several warps per SM sub-partition, the dependent-FMA latency is hidden and the pipe
// itself is the limit.  The host times a launch with CUDA events; flops per launch are
// 2 * CH * iters * threads.
#include "../../include/sgm.h"
#include "common.cuh"

namespace sgm {
namespace {

constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* __restrict__ sink, long iters, T x, T y) {
  T a[kProbeChains];
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (long i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = fma(a[q], x, y);
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += a[q];
  sink[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sgm

using namespace sgm;

extern "C" int sgm_alu_probe(int precision, int blocks, int threads, int64_t iters, void* sink, double* flops,
                             void* stream) {
  if (!sink || !flops) return set_error(SGM_ERR_NULL, "sink and flops must be non-NULL");
  if (precision != SGM_F32 && precision != SGM_F64) return set_error(SGM_ERR_ARG, "precision must be SGM_F32 or SGM_F64");
  if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 1)
    return set_error(SGM_ERR_SIZE, "blocks >= 1, threads a multiple of 32 in 32..256, iters >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == SGM_F64)
    k_fma_probe<double><<<blocks, threads, 0, s>>>((double*)sink, (long)iters, 0.999999, 1e-7);
  else
    k_fma_probe<float><<<blocks, threads, 0, s>>>((float*)sink, (long)iters, 0.999999f, 1e-7f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(SGM_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  *flops = 2.0 * kProbeChains * (double)iters * (double)blocks * (double)threads;
  return SGM_OK;
}
