// Pieces shared by the two persistent PCG kernels (k_pcg.cu: the
// cooperative one over global memory; k_pcg_cluster.cu: the thread-block
// cluster one over distributed shared memory): the inner-product
// accumulators, packed 6x6 indexing and the scalar step of the
// Chronopoulos-Gear recurrences (Sec. 7's block-Jacobi PCG).
#pragma once
#include <type_traits>

#include "sw_df.cuh"

namespace sw {

// ------------------------------------------------------------------ accumulators

// Operations the PCG needs from an accumulator type.  TwoSum's error term is
// exact, so df_add(a, b) == df_add(b, a) bit for bit and every lane of a
// butterfly ends with the same value; the same holds for FP64 addition.
template <typename Acc>
struct AccOps;

template <>
struct AccOps<DF> {
  static __device__ __forceinline__ DF zero() { return DF{0.f, 0.f}; }
  static __device__ __forceinline__ DF prod(float a, float b) { return df_prod(a, b); }
  static __device__ __forceinline__ DF add(DF a, DF b) { return df_add(a, b); }
  static __device__ __forceinline__ DF shfl_xor(DF v, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
  }
  static __device__ __forceinline__ unsigned long long bits(DF v) {
    return (unsigned long long)__float_as_uint(v.hi) | ((unsigned long long)__float_as_uint(v.lo) << 32);
  }
  static __device__ __forceinline__ DF from_bits(unsigned long long b) {
    return DF{__uint_as_float((unsigned)(b & 0xffffffffu)), __uint_as_float((unsigned)(b >> 32))};
  }
  static __device__ __forceinline__ bool nonzero(DF v) { return v.hi != 0.f; }
  static __device__ __forceinline__ double value(DF v) { return (double)v.hi + (double)v.lo; }
};

template <>
struct AccOps<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double prod(float a, float b) { return (double)a * (double)b; }   // exact
  static __device__ __forceinline__ double prod(double a, double b) { return a * b; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ unsigned long long bits(double v) { return (unsigned long long)__double_as_longlong(v); }
  static __device__ __forceinline__ double from_bits(unsigned long long b) { return __longlong_as_double((long long)b); }
  static __device__ __forceinline__ bool nonzero(double v) { return v != 0.0; }
  static __device__ __forceinline__ double value(double v) { return v; }
};

// Cheaper addition for long reduction trees of double-float values
// (cascaded summation, Ogita, Rump & Oishi 2005, "Sum2"): the high parts
// are added by an error-free TwoSum and all low parts and errors by plain
// FP32 additions, with no renormalisation on the way; the result, once
// renormalised by acc_norm, is as accurate as a sum evaluated in twice the
// working precision and then rounded.  For FP64 accumulators a plain add.
__device__ __forceinline__ DF df_add_cascaded(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return DF{s, __fadd_rn(__fadd_rn(a.lo, b.lo), e)};
}
template <typename Acc>
__device__ __forceinline__ Acc acc_add_cascaded(Acc a, Acc b) {
  if constexpr (std::is_same<Acc, DF>::value) return df_add_cascaded(a, b);
  else return a + b;
}
// an FP32 value as an accumulator (exact)
template <typename Acc>
__device__ __forceinline__ Acc acc_from(float x) {
  if constexpr (std::is_same<Acc, DF>::value) return DF{x, 0.f};
  else return (double)x;
}
template <typename Acc>
__device__ __forceinline__ Acc acc_norm(Acc a) {
  if constexpr (std::is_same<Acc, DF>::value) {
    float s, e;
    two_sum(a.hi, a.lo, s, e);
    return DF{s, e};
  } else {
    return a;
  }
}
template <typename Acc>
__device__ __forceinline__ Acc warp_sum_cascaded(Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = acc_add_cascaded(v, AccOps<Acc>::shfl_xor(v, o));
  return v;
}

template <typename Acc>
__device__ __forceinline__ Acc warp_sum_acc(Acc v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = AccOps<Acc>::add(v, AccOps<Acc>::shfl_xor(v, o));
  return v;
}

// a / b for positive FP64 values, rounded to FP32: the exponents are split
// off exactly (frexp) and only the mantissa ratio is divided, in FP32 (an
// FP64 division is several hundred cycles on this part).
__device__ __forceinline__ float ratio_f32(double a, double b) {
  int ea, eb;
  const double ma = frexp(a, &ea), mb = frexp(b, &eb);
  return ldexpf(__fdiv_rn((float)ma, (float)mb), ea - eb);
}

// ------------------------------------------------------------------ packed 6x6 and NaN markers

__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }   // packed, r >= c
__device__ __forceinline__ int sym(int r, int c) { return r >= c ? tri(r, c) : tri(c, r); }
// the packed-lower offsets of row r (0..5) of a symmetric 6x6 block, 5 bits
// each: computed once for a lane-dependent row, then read by sym_at with a
// constant column in an unrolled loop (no per-column index arithmetic; one
// register, which the 64-register cooperative kernels cannot spare)
__device__ __forceinline__ unsigned sym_offsets(int r) {
  unsigned o = 0;
#pragma unroll
  for (int c = 0; c < 6; ++c) o |= (unsigned)sym(r, c) << (5 * c);
  return o;
}
__device__ __forceinline__ int sym_at(unsigned offsets, int c) { return (int)((offsets >> (5 * c)) & 31u); }

template <typename Acc>
__device__ __forceinline__ Acc acc_nan() {
  if constexpr (std::is_same<Acc, DF>::value) return DF{__int_as_float(0x7fffffff), 0.f};
  else return __longlong_as_double(0x7ff8000000000000ll);
}

template <typename Acc>
__device__ __forceinline__ bool acc_is_nan(Acc a) {
  if constexpr (std::is_same<Acc, DF>::value) return a.hi != a.hi;
  else return a != a;
}

// ------------------------------------------------------------------ Chronopoulos-Gear scalars

// One step's scalars from the reduction's totals γ = (r, u) and δ = (w, u):
//   first step  β = 0, α = γ / δ;
//   later       β = γ / γ_prev, α = γ / (δ − β γ / α_prev).
// The denominator is pᵀAp in exact arithmetic; a value <= 0 (or a NaN from a
// broken diagonal block) is a breakdown.  γ = 0 is exact convergence.
// kGearLate is the caller's: a CTA's wait for a neighbour's vector ran out.
enum { kGearOk = 0, kGearBreakdown = 1, kGearConverged = 2, kGearLate = 3 };

template <typename Acc>
__device__ __forceinline__ int gear_step(int k, Acc g, Acc dl, Acc g_prev, float a_prev, float* alpha_out,
                                         float* beta_out) {
  using O = AccOps<Acc>;
  *alpha_out = 0.f;
  *beta_out = 0.f;
  if (acc_is_nan(g) || acc_is_nan(dl)) return kGearBreakdown;
  if (!O::nonzero(g)) return kGearConverged;
  float beta = 0.f, alpha;
  bool pos;
  if constexpr (std::is_same<Acc, DF>::value) {
    float den = dl.hi;
    if (k > 0) {
      beta = __fdiv_rn(g.hi, g_prev.hi);
      const float tt = __fmul_rn(beta, __fdiv_rn(g.hi, a_prev));
      den = df_add(dl, DF{-tt, 0.f}).hi;
    }
    pos = den > 0.f;
    alpha = pos ? __fdiv_rn(g.hi, den) : 0.f;
  } else {
    double den = dl;
    if (k > 0) {
      beta = ratio_f32(g, g_prev);
      den = dl - (double)beta * (double)ratio_f32(g, (double)a_prev);
    }
    pos = den > 0.0;
    alpha = pos ? ratio_f32(g, den) : 0.f;
  }
  if (!pos) return kGearBreakdown;
  *alpha_out = alpha;
  *beta_out = beta;
  return kGearOk;
}

}  // namespace sw
