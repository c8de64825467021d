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

// The leapfrog update and the filter sum in one pass each, renormalised once at the end: every
// product and sum of the HIGH parts is made exact (exact product with an FMA, two-sum), the
// first-order low-order terms (a.hi b.lo, a.lo b.hi, the error terms) are summed in FP32 and
// the pair is renormalised by one fast two-sum.  The terms dropped (products of two low parts)
// and the FP32 rounding of the low-order sum are each below ~u^2 |operand| (u = 2^-24), so the
// error of an update is below ~16 u^2 sum |operands| -- the same order as the chain of
// double-word additions and products it replaces (each ~2^-46 (|a| + |b|)), in about 70 % of
// its FP32 operations (forced 5-point update with its neighbour sums: 67 against 94; filter
// sum: 15 against 18).
struct dfs {             // unnormalised double-float: value h + l, |l| a few ulp(h)
  float h, l;
};
__device__ __forceinline__ dfs df_pair_sum(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return {s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo)};
}

// b c - prv + sum_{m < D} a_m s_m  (- fph f when F): the second-order leapfrog update with c = 1
// in the order of the double-word form df_sub(df_mul(b, c), prv), df_add(., df_mul(a_m, s_m)), ...
template <int D, bool F>
__device__ __forceinline__ dfl df_leapfrog(dfl b, dfl c, dfl prv, const dfl* a, const dfs* sm, dfl fph, dfl f) {
  float p = __fmul_rn(b.hi, c.hi);
  float lo = __fmaf_rn(b.hi, c.hi, -p);
  dfl t = two_sum(p, -prv.hi);
  lo = __fadd_rn(lo, t.lo);
  float th = t.hi;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    const float q = __fmul_rn(a[m].hi, sm[m].h);
    lo = __fadd_rn(lo, __fmaf_rn(a[m].hi, sm[m].h, -q));
    t = two_sum(th, q);
    th = t.hi;
    lo = __fadd_rn(lo, t.lo);
  }
  if (F) {
    const float q = __fmul_rn(fph.hi, f.hi);
    lo = __fsub_rn(lo, __fmaf_rn(fph.hi, f.hi, -q));
    t = two_sum(th, -q);
    th = t.hi;
    lo = __fadd_rn(lo, t.lo);
  }
  lo = __fmaf_rn(b.hi, c.lo, lo);
  lo = __fmaf_rn(b.lo, c.hi, lo);
  lo = __fsub_rn(lo, prv.lo);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    lo = __fmaf_rn(a[m].hi, sm[m].l, lo);
    lo = __fmaf_rn(a[m].lo, sm[m].h, lo);
  }
  if (F) {
    lo = __fmaf_rn(-fph.hi, f.lo, lo);
    lo = __fmaf_rn(-fph.lo, f.hi, lo);
  }
  return fast_two_sum(th, lo);
}

// acc + w x (the trapezoid filter sum)
__device__ __forceinline__ dfl df_fma_acc(dfl acc, dfl w, dfl x) {
  const float p = __fmul_rn(w.hi, x.hi);
  float lo = __fmaf_rn(w.hi, x.hi, -p);
  const dfl s = two_sum(acc.hi, p);
  lo = __fadd_rn(lo, s.lo);
  lo = __fadd_rn(lo, acc.lo);
  lo = __fmaf_rn(w.hi, x.lo, lo);
  lo = __fmaf_rn(w.lo, x.hi, lo);
  return fast_two_sum(s.hi, lo);
}

// coefficients of the double-float step (from FP64 host values)
struct DfCoef {
  dfl ih2[3], dt2, hdt2, fph, w0, w1;
  dfl a[3], b;   // 2nd order, c = 1: W^{n+1} = sum_m a_m (W_{+m} + W_{-m}) + b W^n - W^{n-1}
};

}  // namespace whv
