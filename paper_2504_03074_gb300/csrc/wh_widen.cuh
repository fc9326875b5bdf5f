// wh_widen.cuh -- FP32 -> FP64 widening with integer operations, shared by the two- and
// three-dimensional kernels (and exported for testing as wh_widen_f32).
//
// The filter accumulation of the FP32 march (Algorithm 1's time filter, kept in FP64) widens
// every FP32 state value.  On this part the hardware float -> double conversion runs on the
// narrow FP64 pipe and occupies it several times longer than a DFMA (in the FP32 march it
// kept that pipe ~70% busy while the DFMAs used a tenth of its rate).  IEEE 754 fixes the
// binary64 value of a normal binary32 number: the same sign, the exponent rebiased by
// 1023 - 127 = 896 and the 23 fraction bits followed by 29 zeros, which integer operations
// assemble exactly; signed zeros keep their sign with a zero exponent and fraction.
// Subnormals, infinities and NaNs (never produced by a stable march) use the hardware
// conversion.
#pragma once
#include <cuda_runtime.h>

namespace wh {

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)x;
}

}  // namespace wh
