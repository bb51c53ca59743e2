// Double-float arithmetic shared by the PCG's reductions and the rigid
// pre-alignment's sums.
#pragma once
#include <cuda_runtime.h>

namespace sw {

// Double-float accumulation: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  Products
// come from the error-free TwoProduct (one FMA recovers the rounding error of
// a*b, Dekker 1971); sums use Knuth's TwoSum on the high and the low parts
// followed by two renormalisations (the "accurate" pair addition analysed by
// Joldes, Muller and Popescu, ACM TOMS 2017: relative error below 3 * 2^-48).
// Only FP32 operations are involved: an FP64 instruction occupies this part's
// FP64 pipe for tens of cycles, and the reductions sit on the critical path.
// The _rn intrinsics are never contracted or reassociated by the compiler.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b| or a == 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return DF{s, e};
}

// the pair's value, exactly (hi + lo fits an FP64 mantissa)
__device__ __forceinline__ double df_value(DF v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ DF df_from(float x) { return DF{x, 0.f}; }

__device__ __forceinline__ DF df_shfl_xor(DF v, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

}  // namespace sw
