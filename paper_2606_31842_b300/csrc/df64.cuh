// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, a ~48-bit significand computed on the FP32 pipes (on B300 FP64 runs at 1/64
// of the FP32 rate).  Built from the error-free transformations
//   two-sum (Knuth, TAOCP vol. 2):      s = a + b exactly as s + e, any a, b
//   fast two-sum (Dekker 1971):         the same when |a| >= |b|
//   exact product with an FMA:          a b = p + e, e = fma(a, b, -p)
// The sum is Dekker's double-word addition (add2, 1971): a two-sum of the high parts, the low
// parts added to its error term, one fast two-sum to renormalise (11 FP32 operations instead of
// the 20 of the form that two-sums the low parts as well).  Its error is bounded relative to
// |a| + |b| rather than to |a + b| -- about 2^-46 (|a| + |b|) -- so under cancellation it keeps
// an absolute, not a relative, accuracy: enough for the wave solves, where every sum has
// operands of the size of the field (W^n, W^{n-1}, the neighbours, the filter sum) and what
// matters is the error against that size.  No expression here has a multiply next to an add
// that the compiler could contract into an FMA and change.
#pragma once

#include <cuda_runtime.h>

namespace whv {

struct dfl {
  float hi, lo;
};

__host__ __device__ __forceinline__ dfl df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfl df_zero() { return {0.0f, 0.0f}; }
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// coefficients of the double-float step (from FP64 host values)
struct DfCoef {
  dfl ih2[3], dt2, hdt2, fph, w0, w1;
  dfl a[3], b;   // 2nd order, c = 1: W^{n+1} = sum_m a_m (W_{+m} + W_{-m}) + b W^n - W^{n-1}
};

}  // namespace whv
