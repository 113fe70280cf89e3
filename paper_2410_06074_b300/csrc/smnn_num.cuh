// smnn_num.cuh -- number types of the refinement residual and the gradient kernel.
//
// The residual r = beta - M y of iterative refinement (and the gradient formulas, whose
// terms d_t - c_t.y_t and c_t.g_t cancel) need more than FP32.  Two arithmetics serve:
//   double  FP64 on the FP64 pipe (~2 FMA/clock/SM on B300);
//   ff      "float-float": a value is an unevaluated sum hi + lo of two FP32 numbers
//           (|lo| <= ulp(hi)/2, ~48-bit significand), computed on the FP32 pipe with
//           error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and the
//           FMA form of TwoProduct (the product a*b and its exact rounding error
//           fma(a, b, -a*b)).  Additions and products carry ~2^-47 relative error of
//           the operands, i.e. the role FP64 rounding plays in the FP64 variant.
//   ffl     float-float without renormalisation (below), for the refinement residual.
// The kernels are written once over a number type N with +, -, * and the conversions
// of Num<N>; the round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the error-free steps.
#pragma once
#include <cstdint>

namespace smnn {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator+(ff a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator-(ff a, float b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator*(ff a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { a = a - b; return a; }

// "Lazy" float-float for the refinement residual: the same unevaluated sum hi + lo, but no
// operation renormalises it.  A sum adds the high parts with TwoSum (exact: hi + err equals
// a.hi + b.hi) and the low parts and err in FP32; a product by a float or a pair splits
// hi * b exactly (FMA TwoProduct) and adds the cross terms into the low part.  After a
// cancellation |lo| may exceed ulp(hi), but every rounding still acts on a low part, whose
// size is ~2^-24 times the operands that formed it, so the absolute error of a short
// expression stays ~2^-47 times the size of its operands -- what the residual needs -- at
// 8 FP32 operations per pair sum instead of 11, and 3-4 per product instead of 6-7.
struct ffl {
  float hi, lo;
};
__device__ __forceinline__ ffl operator+(ffl a, ffl b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ffl{s.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo)};
}
__device__ __forceinline__ ffl operator+(ffl a, float b) {
  const ff s = ff_two_sum(a.hi, b);
  return ffl{s.hi, __fadd_rn(a.lo, s.lo)};
}
__device__ __forceinline__ ffl operator-(ffl a) { return ffl{-a.hi, -a.lo}; }
__device__ __forceinline__ ffl operator-(ffl a, ffl b) { return a + (-b); }
__device__ __forceinline__ ffl operator-(ffl a, float b) { return a + (-b); }
__device__ __forceinline__ ffl operator*(ffl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  return ffl{p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p))};
}
__device__ __forceinline__ ffl operator*(ffl a, ffl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  return ffl{p, __fmaf_rn(a.lo, b.hi, e)};
}
__device__ __forceinline__ ffl& operator+=(ffl& a, ffl b) { a = a + b; return a; }
__device__ __forceinline__ ffl& operator-=(ffl& a, ffl b) { a = a - b; return a; }

// Conversions and constants of a number type.
template <class N> struct Num;

template <> struct Num<double> {
  __device__ static double from_f(float v) { return double(v); }
  __device__ static double from_d(double v) { return v; }
  __device__ static double pair(float hi, float lo) { return double(hi) + double(lo); }
  __device__ static double pair(double hi, double lo) { return hi + lo; }
  __device__ static float to_f(double v) { return float(v); }
  __device__ static double to_d(double v) { return v; }
  __device__ static double zero() { return 0.0; }
};

template <> struct Num<ff> {
  __device__ static ff from_f(float v) { return ff{v, 0.f}; }
  __device__ static ff from_d(double v) {
    const float h = float(v);
    return ff{h, float(v - double(h))};
  }
  __device__ static ff pair(float hi, float lo) { return ff{hi, lo}; }
  __device__ static float to_f(ff v) { return __fadd_rn(v.hi, v.lo); }
  __device__ static double to_d(ff v) { return double(v.hi) + double(v.lo); }
  __device__ static ff zero() { return ff{0.f, 0.f}; }
};

template <> struct Num<ffl> {
  __device__ static ffl from_f(float v) { return ffl{v, 0.f}; }
  __device__ static ffl from_d(double v) {
    const float h = float(v);
    return ffl{h, float(v - double(h))};
  }
  __device__ static ffl pair(float hi, float lo) { return ffl{hi, lo}; }
  __device__ static float to_f(ffl v) { return __fadd_rn(v.hi, v.lo); }
  __device__ static double to_d(ffl v) { return double(v.hi) + double(v.lo); }
  __device__ static ffl zero() { return ffl{0.f, 0.f}; }
};

// 1/k! as a number of type N (hi/lo split done at compile time for ff).
template <class N> __device__ __forceinline__ N inv_fact_n(int k);
template <> __device__ __forceinline__ double inv_fact_n<double>(int k) {
  return k <= 1 ? 1.0 : (k == 2 ? 0.5 : 1.0 / 6.0);
}
template <> __device__ __forceinline__ ffl inv_fact_n<ffl>(int k) {
  switch (k) {
    case 0: case 1: return ffl{1.f, 0.f};
    case 2: return ffl{0.5f, 0.f};
    default: {
      constexpr double v = 1.0 / 6.0;
      constexpr float h = float(v);
      constexpr float l = float(v - double(h));
      return ffl{h, l};
    }
  }
}
template <> __device__ __forceinline__ ff inv_fact_n<ff>(int k) {
  // exact for k <= 2; for k = 3 (1/6) the split of the double value
  switch (k) {
    case 0: case 1: return ff{1.f, 0.f};
    case 2: return ff{0.5f, 0.f};
    default: {
      constexpr double v = 1.0 / 6.0;
      constexpr float h = float(v);
      constexpr float l = float(v - double(h));
      return ff{h, l};
    }
  }
}

}  // namespace smnn
