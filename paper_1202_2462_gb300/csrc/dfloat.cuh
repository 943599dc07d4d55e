// Double-float arithmetic: a real number held as the unevaluated sum hi + lo
// of two FP32 numbers (Dekker, "A floating-point technique for extending the
// available precision", Numer. Math. 18, 1971; Knuth, TAOCP vol. 2, 4.2.2),
// with the error-free product taken from the fused multiply-add.  About 48
// significand bits, i.e. a relative rounding error of a few 1e-15, on the
// FP32 units.  Each double-float multiply-add costs about 18 FP32
// instructions in dependent chains; for the Dirac stencil it measured slower
// than the FP64 units (an opt-in of dirac_apply, MG_FP64_ON_FP32).  Every
// operation uses the explicitly rounded intrinsics, so the compiler can
// neither fuse nor reorder the error-free transformations.
#pragma once
#include "common.cuh"

namespace sapmg {

struct DF {
  float hi, lo;
  DF() = default;
  __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ DF(int i) : hi((float)i), lo(0.f) {}
  // the FP64 value split into its leading 24 bits and the next 24 (d - hi is
  // exact in FP64; the hi + lo sum below is exact as well)
  __device__ __forceinline__ explicit DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly, |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// s + e = a + b exactly, any order
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
// p + e = a.hi b.hi exactly (the FMA's single rounding), plus the cross terms
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF fma(DF a, DF b, DF c) { return a * b + c; }
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { a = a + b; return a; }

}  // namespace sapmg
