// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi) / 2, about 48 significant bits computed on the
// FP32 pipes.  GB300 executes FP32 at 64x its FP64 rate per SM, so a
// factorisation in double-float (about 15 FP32 operations per multiply-add)
// runs several times faster than in native FP64 at nearly FP64 accuracy.
// The operations are the classical error-free transformations: TwoSum
// (Knuth) for sums, TwoProd through the fused multiply-add for products
// (Dekker; Hida, Li & Bailey's double-double algorithms).
#pragma once

namespace bipm {

struct df {
  float hi, lo;
  df() = default;
  __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ df(float h) : hi(h), lo(0.0f) {}
  __device__ __forceinline__ df(int v) : hi((float)v), lo(0.0f) {}
  __device__ __forceinline__ df(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return df(s, e);
}
__device__ __forceinline__ df operator+(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  df t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df operator/(df a, df b) {
  float q1 = a.hi / b.hi;
  df r = a - b * df(q1);
  float q2 = r.hi / b.hi;
  r = r - b * df(q2);
  float q3 = r.hi / b.hi;
  df q = df_fast_two_sum(q1, q2);
  return q + df(q3);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

// precision traits of the factorisation type
template <class T> struct HighPrecision { static constexpr bool value = false; };
template <> struct HighPrecision<double> { static constexpr bool value = true; };
template <> struct HighPrecision<df> { static constexpr bool value = true; };

}  // namespace bipm
