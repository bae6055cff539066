// Device-side Gaussian stream for Omega_n (Sec. 2.4: i.i.d. N(0,1) entries; Sec. 3.1:
// entries generated on the fly, never stored).
//
// Specification (the paper fixes only the distribution):
//   Philox4x32-10 (Salmon et al., SC'11) with key (lo32 seed, hi32 seed) and counter
//   (col/4, lo32 row, hi32 row, (tensor_id << 4) | mode);
//   u = ((w >> 8) | 1) * 2^-24;  Box-Muller on (w0,w1) and (w2,w3):
//   rho = sqrt(-2 log u_a), (rho cos 2 pi u_b, rho sin 2 pi u_b).
// Every FP32 operation is an explicitly rounded intrinsic (no contraction into FMA),
// so the values are reproducible bit for bit by any IEEE implementation that follows
// the same operation order.  log and sin/cos are this library's own:
//   log u:   u = m 2^e, m in (sqrt(1/2), sqrt(2)], log m = 2 atanh(s), s = (m-1)/(m+1),
//            atanh by its Taylor series through s^9, e ln2 with a 15-bit head of ln2.
//   2 pi u:  q = round(4u), r = u - q/4 (exact), Taylor series of sin(2 pi r) through r^9
//            and cos(2 pi r) through r^10, then the quadrant rotation by q.
#pragma once

#include <stdint.h>

namespace rh {
namespace rng {

constexpr double kTau = 6.283185307179586476925286766559;

__host__ __device__ constexpr double tau_pow(int k) { return k == 0 ? 1.0 : kTau * tau_pow(k - 1); }

// log constants
constexpr float kSqrt2 = (float)1.4142135623730950488;
constexpr float kLn2Hi = 0.693145751953125f;  // 0x3F317200
constexpr float kLn2Lo = (float)(0.6931471805599453094 - 0.693145751953125);
constexpr float kL3 = (float)(2.0 / 3.0);
constexpr float kL5 = (float)(2.0 / 5.0);
constexpr float kL7 = (float)(2.0 / 7.0);
constexpr float kL9 = (float)(2.0 / 9.0);
constexpr float kL11 = (float)(2.0 / 11.0);
// sin / cos (2 pi r) Taylor coefficients
constexpr float kS1 = (float)kTau;
constexpr float kS3 = (float)(-tau_pow(3) / 6.0);
constexpr float kS5 = (float)(tau_pow(5) / 120.0);
constexpr float kS7 = (float)(-tau_pow(7) / 5040.0);
constexpr float kS9 = (float)(tau_pow(9) / 362880.0);
constexpr float kC2 = (float)(-tau_pow(2) / 2.0);
constexpr float kC4 = (float)(tau_pow(4) / 24.0);
constexpr float kC6 = (float)(-tau_pow(6) / 720.0);
constexpr float kC8 = (float)(tau_pow(8) / 40320.0);
constexpr float kC10 = (float)(-tau_pow(10) / 3628800.0);

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ float uniform24(uint32_t w) {
  return __fmul_rn((float)((w >> 8) | 1u), 5.9604644775390625e-8f);  // * 2^-24, exact
}

__device__ __forceinline__ float log_f32(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > kSqrt2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(m, 1.0f));
  const float z = __fmul_rn(s, s);
  float p = kL11;
  p = __fadd_rn(__fmul_rn(p, z), kL9);
  p = __fadd_rn(__fmul_rn(p, z), kL7);
  p = __fadd_rn(__fmul_rn(p, z), kL5);
  p = __fadd_rn(__fmul_rn(p, z), kL3);
  float t = __fmul_rn(s, z);
  t = __fmul_rn(t, p);
  const float logm = __fadd_rn(__fadd_rn(s, s), t);
  const float ef = (float)e;
  return __fadd_rn(__fmul_rn(ef, kLn2Hi), __fadd_rn(__fmul_rn(ef, kLn2Lo), logm));
}

__device__ __forceinline__ void cossin_2pi_f32(float u, float& co, float& si) {
  const float q = rintf(__fmul_rn(u, 4.0f));
  const float r = __fsub_rn(u, __fmul_rn(q, 0.25f));
  const float z = __fmul_rn(r, r);
  float ps = kS9;
  ps = __fadd_rn(__fmul_rn(ps, z), kS7);
  ps = __fadd_rn(__fmul_rn(ps, z), kS5);
  ps = __fadd_rn(__fmul_rn(ps, z), kS3);
  ps = __fadd_rn(__fmul_rn(ps, z), kS1);
  const float s = __fmul_rn(r, ps);
  float pc = kC10;
  pc = __fadd_rn(__fmul_rn(pc, z), kC8);
  pc = __fadd_rn(__fmul_rn(pc, z), kC6);
  pc = __fadd_rn(__fmul_rn(pc, z), kC4);
  pc = __fadd_rn(__fmul_rn(pc, z), kC2);
  const float c = __fadd_rn(__fmul_rn(pc, z), 1.0f);
  switch (((int)q) & 3) {
    case 0: co = c; si = s; break;
    case 1: co = -s; si = c; break;
    case 2: co = -c; si = -s; break;
    default: co = s; si = -c; break;
  }
}

__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const float rho = __fsqrt_rn(__fmul_rn(log_f32(uniform24(wa)), -2.0f));
  float co, si;
  cossin_2pi_f32(uniform24(wb), co, si);
  n0 = __fmul_rn(rho, co);
  n1 = __fmul_rn(rho, si);
}

// Four consecutive entries Omega(row, 4q .. 4q+3).
__device__ __forceinline__ float4 omega4(uint32_t k0, uint32_t k1, uint32_t sid, int64_t row, uint32_t q) {
  const uint4 w = philox4x32_10(make_uint4(q, (uint32_t)((uint64_t)row & 0xFFFFFFFFu),
                                           (uint32_t)((uint64_t)row >> 32), sid),
                                k0, k1);
  float4 r;
  box_muller(w.x, w.y, r.x, r.y);
  box_muller(w.z, w.w, r.z, r.w);
  return r;
}

}  // namespace rng
}  // namespace rh
