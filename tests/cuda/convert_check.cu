// Checks the integer-pipe conversions of csrc/convert.cuh bitwise against the hardware
// conversions: widen_f32 on all 2^32 FP32 bit patterns, narrow_f64 on random doubles and on
// constructed ties, near-ties, carries and range edges, including ties of results in the FP32
// subnormal range.  Prints "mismatches <n>"; exit 0.
#include <cstdio>
#include <cstdint>
#include "../../paper_1708_03188_gb300/csrc/convert.cuh"

__global__ void widen_all(unsigned long long* bad) {
  const unsigned long long n = 1ull << 32;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float f = __uint_as_float((unsigned)i);
    const double a = sgm::widen_f32(f), b = (double)f;
    if (__double_as_longlong(a) != __double_as_longlong(b) && !(a != a && b != b)) atomicAdd(bad, 1ull);
  }
}

__device__ unsigned long long mix(unsigned long long x) {  // splitmix64
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__global__ void narrow_many(unsigned long long* bad, unsigned long long n) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long r = mix(i);
    unsigned long long bits;
    const unsigned kind = (unsigned)(r & 7);
    const unsigned long long sign = (r >> 63) << 63;
    const unsigned long long ex = 870 + (mix(r) % 310);             // around the FP32 range
    unsigned long long mant = mix(r + 1) & 0xfffffffffffffull;
    if (kind == 1) mant = (mant & ~0x1fffffffull) | 0x10000000ull;   // exact tie
    if (kind == 2) mant = (mant & ~0x1fffffffull) | 0x0fffffffull;   // just below a tie
    if (kind == 3) mant = (mant & ~0x1fffffffull) | 0x10000001ull;   // just above a tie
    if (kind == 4) mant = 0xfffffffffffffull;                        // carry into the exponent
    bits = sign | (ex << 52) | mant;
    if (kind == 5) bits = mix(r + 7);                                // any pattern
    if (kind == 6 || kind == 7) {   // FP32-subnormal results: an exact tie (6), one unit above it (7)
      const unsigned long long es = 873 + (mix(r + 3) % 24);      // 873..896
      const unsigned sh = (unsigned)(926 - es);
      unsigned long long M = (1ull << 52) | mant;
      M = ((M >> sh) << sh) | (1ull << (sh - 1));
      if (kind == 7) M += 1;
      bits = sign | (es << 52) | (M & 0xfffffffffffffull);
    }
    const double d = __longlong_as_double((long long)bits);
    const float a = sgm::narrow_f64(d), b = __double2float_rn(d);
    if (__float_as_uint(a) != __float_as_uint(b) && !(a != a && b != b)) atomicAdd(bad, 1ull);
  }
}

int main() {
  unsigned long long* bad;
  cudaMalloc(&bad, 2 * sizeof(unsigned long long));
  cudaMemset(bad, 0, 2 * sizeof(unsigned long long));
  widen_all<<<4096, 256>>>(bad);
  narrow_many<<<4096, 256>>>(bad + 1, 1ull << 30);
  unsigned long long h[2] = {~0ull, ~0ull};
  cudaError_t e = cudaMemcpy(h, bad, sizeof h, cudaMemcpyDeviceToHost);
  printf("status %s\nwiden_mismatches %llu\nnarrow_mismatches %llu\n", cudaGetErrorString(e), h[0], h[1]);
  cudaFree(bad);
  return e == cudaSuccess ? 0 : 1;
}
