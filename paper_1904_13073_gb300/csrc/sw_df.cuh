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

// a * b for pairs: the high parts' exact product (TwoProduct) plus the two
// cross terms, renormalised (the lo * lo term is below the pair's precision)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return DF{s, t};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// c - a * b
__device__ __forceinline__ DF df_fnma(DF a, DF b, DF c) { return df_add(c, df_neg(df_mul(a, b))); }

// 1 / x for a positive pair of normal magnitude: the FP32 reciprocal of the
// high part, refined by one Newton-Raphson step r + r (1 - x r) evaluated in
// pairs (about 24 -> 48 correct bits)
__device__ __forceinline__ DF df_recip(DF x) {
  const DF r = DF{__frcp_rn(x.hi), 0.f};
  const DF q = df_add(DF{1.f, 0.f}, df_neg(df_mul(x, r)));
  return df_add(r, df_mul(r, q));
}

// the pair's value, exactly (hi + lo fits an FP64 mantissa)
__device__ __forceinline__ double df_value(DF v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ DF df_from(float x) { return DF{x, 0.f}; }

__device__ __forceinline__ DF df_shfl_xor(DF v, int o) {
  return DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

}  // namespace sw
