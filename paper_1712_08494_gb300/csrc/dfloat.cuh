// Double-float arithmetic and per-thread running sums, shared by the
// Poisson solvers and the observables.
#pragma once

namespace lbeh {

// Double-float numbers (hi + lo, two FP32 words, ~48-bit significand) with
// error-free transformations: the FP32 modes keep the potential and form the
// defect-correction residual in this form, on the FP32 pipes (the FP64 rate
// of the target is a small fraction of its FP32 rate).  Intrinsics keep the
// compiler from contracting the compensated sums.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  const DF t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, DF{-b.hi, -b.lo}); }
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_add_f(DF a, float b) {
  DF s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

// Per-thread running sum: double-float words in the FP32 modes (site values
// are FP32 and the FP64 pipe is slow), plain FP64 in the FP64 mode; the block
// and grid reductions that follow run in FP64.
template <bool DFM> struct SumAcc;
template <> struct SumAcc<true> {
  DF v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = df_add_f(v, x); }
  __device__ __forceinline__ double get() const { return double(v.hi) + double(v.lo); }
};
template <> struct SumAcc<false> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double get() const { return v; }
};

// u w and u w^2 added to a running sum, the products formed exactly in the
// double-float case
__device__ __forceinline__ void acc_prod(SumAcc<true> &a, float u, float w) {
  const float p = __fmul_rn(u, w);
  a.v = df_add(a.v, DF{p, __fmaf_rn(u, w, -p)});
}
__device__ __forceinline__ void acc_prod(SumAcc<false> &a, double u, double w) { a.v += u * w; }
__device__ __forceinline__ void acc_prod2(SumAcc<true> &a, float u, float w) {
  const float p = __fmul_rn(u, w);
  a.v = df_add(a.v, df_mul_f(DF{p, __fmaf_rn(u, w, -p)}, w));
}
__device__ __forceinline__ void acc_prod2(SumAcc<false> &a, double u, double w) { a.v += u * w * w; }

}  // namespace lbeh
