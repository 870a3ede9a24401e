// Double-float arithmetic for the FP32 pipes.  A value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2: about 48
// significant bits, with FP32's exponent range.  GB300 issues FP32 FMAs at
// 64 times its FP64 rate, so element passes that need more than FP32 but
// not all of FP64 run several times faster this way.
//
// Built on error-free transformations: TwoSum (Knuth, TAOCP vol. 2,
// Sec. 4.2.2) and FastTwoSum (Dekker 1971) give s + e = a + b exactly;
// TwoProduct with a fused multiply-add gives p + e = a * b exactly.  The
// product is Dekker's double-length multiplication with its cross terms
// folded in by FMA, the quotient long division with two correction steps;
// sums come in Dekker's form (operator+) and an accurate form (both parts
// added separately, renormalised twice) for cancelling totals.
// Requires IEEE FP32 without flush-to-zero and without reassociation (the
// library is built without fast-math).
#pragma once
#include <cuda_runtime.h>

namespace pf {

struct df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  // exact small integers and compile-time constants; a runtime double in
  // device code would cost FP64 instructions (use df_from)
  __host__ __device__ constexpr df(int i) : hi(float(i)), lo(0.f) {}
  __host__ __device__ constexpr df(double d)
      : hi(float(d)), lo(float(d - double(float(d)))) {}
};

__device__ __forceinline__ df df_from(double d) {
  const float h = __double2float_rn(d);
  return df(h, __double2float_rn(d - double(h)));
}
__device__ __forceinline__ double df_to_double(df x) { return double(x.hi) + double(x.lo); }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// Accurate double-length sum: error about 2^-47 |x + y| even under
// cancellation.  Used where sums of many elements cancel (nodal sums of
// element contributions, energy totals).
__device__ __forceinline__ df add_accurate(df x, df y) {
  float s, e, t, f;
  two_sum(x.hi, y.hi, s, e);
  two_sum(x.lo, y.lo, t, f);
  e += t;
  fast_two_sum(s, e, s, e);
  e += f;
  fast_two_sum(s, e, s, e);
  return df(s, e);
}

// Dekker's double-length sum: error about 2^-46 (|x| + |y|), half the
// instructions of add_accurate.  The operator form, used inside the element
// algebra, whose intermediate sums do not cancel to far below their terms.
__device__ __forceinline__ df operator+(df x, df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e += x.lo + y.lo;
  fast_two_sum(s, e, s, e);
  return df(s, e);
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s;
  fast_two_sum(p, e, s, e);
  return df(s, e);
}
__device__ __forceinline__ df operator/(df x, df y) {
  const float q1 = x.hi / y.hi;
  df r = x - y * df(q1, 0.f);
  const float q2 = r.hi / y.hi;
  r = r - y * df(q2, 0.f);
  const float q3 = r.hi / y.hi;
  float s, e;
  fast_two_sum(q1, q2, s, e);
  return df(s, e) + df(q3, 0.f);
}
__device__ __forceinline__ df& operator+=(df& x, df y) { return x = x + y; }
__device__ __forceinline__ df& operator-=(df& x, df y) { return x = x - y; }
__device__ __forceinline__ df& operator*=(df& x, df y) { return x = x * y; }

}  // namespace pf
