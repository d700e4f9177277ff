// convert.cuh - FP32 <-> FP64 conversions on the integer pipe.
//
// On GB300 the FP64 pipe executes 2 operations per clock per SM and the hardware
// float<->double conversions issue on it, so the FP64 eliminations of k_solve.cu do these
// conversions with integer bit operations (IEEE 754 binary32/binary64 layouts).  Widening
// never uses the hardware conversion; narrowing falls back to it for results outside the
// normal FP32 range (zeros, subnormals, overflow) and for non-finite inputs.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace sgm {

// Exact widening: binary32 exponent e (bias 127) -> e + 896 (bias 1023); the 23-bit
// significand moves to the top of the 52-bit field.  Every class stays on the integer pipe: zero
// keeps exponent 0; a subnormal significand m is normalised (the shift sh = clz(m) - 8 brings its
// leading one to bit 23, and the value m 2^-149 has binary64 exponent 897 - sh); infinities and NaNs
// keep the all-ones exponent.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x7fffffu;
  const unsigned sh = __clz(m) - 8u;
  unsigned E = e + 896u, M = m;
  if (e == 0u) {
    E = m == 0u ? 0u : 897u - sh;
    M = m == 0u ? 0u : (m << sh) & 0x7fffffu;
  } else if (e == 0xffu) {
    E = 0x7ffu;
  }
  const unsigned hi = (b & 0x80000000u) | (E << 20) | (M >> 3);
  return __hiloint2double((int)hi, (int)(M << 29));
}

// Round to nearest, ties to even: keep the top 23 of the 52 significand bits and add one
// unit when the dropped 29 bits exceed half a unit, or equal it with an odd kept part; a
// carry out of the significand correctly increments the exponent (and reaches the
// infinity encoding on overflow).  Results that would be subnormal or zero, and
// non-finite inputs, use the hardware conversion.
__device__ __forceinline__ float narrow_f64(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return __double2float_rn(d);
  unsigned r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  r += (rem > 0x10000000u) || (rem == 0x10000000u && (r & 1u));
  return __uint_as_float((hi & 0x80000000u) | r);
}

template <typename T> __device__ __forceinline__ double widen(T v);
template <> __device__ __forceinline__ double widen<float>(float v) { return widen_f32(v); }
template <> __device__ __forceinline__ double widen<double>(double v) { return v; }
template <typename T> __device__ __forceinline__ T narrow(double v);
template <> __device__ __forceinline__ float narrow<float>(double v) { return narrow_f64(v); }
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }

// Spectral-side element access with storage type TS (T, or double when computing in FP32).
template <typename TS, typename C> __device__ __forceinline__ C from_spec(const TS* p, long g, bool real) {
  using T = decltype(C::x);
  if constexpr (sizeof(TS) == sizeof(T)) {
    return real ? mk<C>(((const T*)p)[g], (T)0) : ((const C*)p)[g];
  } else {
    if (real) return mk<C>(narrow<T>(p[g]), (T)0);
    const double2 v = ((const double2*)p)[g];
    return mk<C>(narrow<T>(v.x), narrow<T>(v.y));
  }
}
template <typename TS, typename C> __device__ __forceinline__ void to_spec(TS* p, long g, bool real, C v) {
  using T = decltype(C::x);
  if constexpr (sizeof(TS) == sizeof(T)) {
    if (real) ((T*)p)[g] = v.x;
    else ((C*)p)[g] = v;
  } else {
    if (real) { p[g] = widen<T>(v.x); return; }
    ((double2*)p)[g] = make_double2(widen<T>(v.x), widen<T>(v.y));
  }
}

}  // namespace sgm
