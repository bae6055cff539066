// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  On this GPU FP64 instructions have long
// latency and low throughput, so the small sequential factorizations of the FP32 paths (a
// Cholesky step is a chain of dependent operations) run in double-float on the FP32 pipes.
//
// Building blocks (published error-free transformations):
//   two_sum       Knuth, TAOCP vol. 2, 4.2.2: s + e = a + b exactly (6 operations).
//   fast_two_sum  Dekker 1971 ("A floating-point technique for extending the available
//                 precision"): s + e = a + b exactly when |a| >= |b| (3 operations).
//   two_prod      p + e = a b exactly with one fused multiply-add (e = fma(a, b, -p)).
// Products and sums of double-floats follow Dekker's mul2 / add2 with the FMA-based product.
// The exponent range is FP32's: callers scale their data by a power of two first.
#pragma once

namespace rh {
namespace dfl {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ F2 add(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  const F2 t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ F2 neg(F2 x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ F2 mul(F2 x, F2 y) {
  F2 p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
// x - a b
__device__ __forceinline__ F2 fms(F2 x, F2 a, F2 b) { return add(x, neg(mul(a, b))); }
__device__ __forceinline__ F2 from_double(double d) {
  const float h = (float)d;
  return {h, (float)(d - (double)h)};
}
__device__ __forceinline__ double to_double(F2 x) { return (double)x.hi + (double)x.lo; }
// 1 / sqrt(x) for x > 0: FP32 estimate, then one Newton step y + y (1 - x y^2) / 2 evaluated in
// double-float (the estimate's ~2^-22 relative error becomes ~2^-43).
__device__ __forceinline__ F2 rsqrt(F2 x) {
  const float y0 = rsqrtf(x.hi);
  const F2 r = add(F2{1.0f, 0.0f}, neg(mul(x, two_prod(y0, y0))));
  const F2 c = mul(F2{0.5f * y0, 0.0f}, r);
  return add(F2{y0, 0.0f}, c);
}

}  // namespace dfl
}  // namespace rh
