// pft_narrow.cuh -- double -> float narrowing on the integer pipe (GB300 runs F2F on its
// 1/64-rate FP64 pipe).
#pragma once
#include "pft_fft.cuh"

namespace pft {
// double -> float rounded to nearest (ties to even) by integer operations, the inverse
// companion of widen: exact IEEE-754 rounding for results in the normal float range;
// results below the smallest normal float become a signed zero, overflow gives infinity,
// NaN stays NaN.
__device__ __forceinline__ float narrow_rn(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ffu);
  const unsigned long long m = u & 0xfffffffffffffull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  const int ef = e - 1023 + 127;
  if (ef <= 0) return __uint_as_float(sign);
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);
  unsigned keep = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1fffffffull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) keep += 1u;
  unsigned bits = ((unsigned)ef << 23) + keep;  // a mantissa carry moves into the exponent
  if ((bits >> 23) >= 255u) bits = 0x7f800000u;
  return __uint_as_float(sign | bits);
}
__device__ __forceinline__ double narrow_rn_as(double d, double) { return d; }
__device__ __forceinline__ float narrow_rn_as(double d, float) { return narrow_rn(d); }

}  // namespace pft
