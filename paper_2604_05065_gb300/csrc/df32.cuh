// Compensated FP32 arithmetic: a value is carried as an unevaluated sum s + c of two
// floats, products are made exact with an FMA (a*h = p + e) and sums with Knuth's
// TwoSum, which keeps about 44 significant bits.
#pragma once
#include <cuda_runtime.h>

namespace apl {

struct DF {
  float s, c;
};

// FP32 -> FP64 by moving the bits (exact for normal numbers; zero, subnormals, infinities
// and NaN take the conversion instruction): GB300 runs conversions to FP64 at its FP64
// rate, integer operations at full rate.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)f;
  const uint64_t bits = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(ex + 896u) << 52) |
                        ((uint64_t)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }


// s + c += a * (h + l).  Explicit round-to-nearest intrinsics keep the compiler from
// contracting the error terms.
__device__ __forceinline__ void df_fma(DF& acc, float a, float h, float l) {
  const float p = __fmul_rn(a, h);
  const float e = __fmaf_rn(a, h, -p);
  const float t = __fadd_rn(acc.s, p);
  const float bv = __fsub_rn(t, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  acc.s = t;
  acc.c = __fmaf_rn(a, l, __fadd_rn(acc.c, __fadd_rn(err, e)));
}

__device__ __forceinline__ double df_val(const DF& a) { return (double)a.s + (double)a.c; }

// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

}  // namespace apl
