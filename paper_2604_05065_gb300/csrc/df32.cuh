// Compensated FP32 arithmetic: a value is carried as an unevaluated sum s + c of two
// floats, products are made exact with an FMA (a*h = p + e) and sums with Knuth's
// TwoSum, which keeps about 44 significant bits.
#pragma once
#include <cuda_runtime.h>

namespace apl {

struct DF {
  float s, c;
};

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
