// Inline-PTX wrappers for the sm_103a tensor-core path: mbarriers, TMA tile loads, tcgen05
// (TMEM allocation, MMA, commit, TMEM loads) and the shared-memory / instruction descriptors.
//
// Every wait on an mbarrier is bounded: after kSpinLimit polls it records an error in
// *err and gives up, so a kernel can always finish (the caller reads the flag).
#pragma once

#include "f32x2.cuh"
#include <cuda.h>
#include <stdint.h>

namespace rh {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- mbarrier ----------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; returns false (and sets *err) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* err, int32_t code,
                                          uint32_t limit = kSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, code);
  return false;
}

// Wait-timeout probe (test support).  A launch that the host marks as probed has thread 0 wait,
// with a short limit, on an mbarrier that nothing arrives at, right after the barriers are
// initialised -- before any TMEM allocation, TMA copy or MMA -- so the wait gives up with
// nothing in flight, records kProbeCode in *err and the whole CTA returns.  This exercises the
// reporting path of a bounded wait that gave up (info bit 16, the wait status words) without
// stalling a pipeline.
constexpr int32_t kProbeCode = 64;
constexpr uint32_t kProbeSpin = 1u << 12;

// ---- proxies -------------------------------------------------------------------------
// Generic-proxy writes to shared memory that the async proxy (TMA, tensor cores) will read.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- TMA -----------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, int32_t c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// ---- tcgen05 ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (BF16 inputs, FP32 accumulation), one CTA.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on *bar once all previously issued MMAs of this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor, 128-byte swizzle (atoms of 8 rows x 128 B, 1024-B aligned):
// start address, leading-dimension byte offset, stride byte offset, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator, M x N tile;
// a_mn / b_mn select MN-major (1) or K-major (0) operands.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4)                     // D format: F32
         | (1u << 7)                   // A format: BF16
         | (1u << 10)                  // B format: BF16
         | ((uint32_t)a_mn << 15)      // A major
         | ((uint32_t)b_mn << 16)      // B major
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// Round an FP32 value to the nearest BF16 (ties to even); finite inputs only.
__device__ __forceinline__ uint16_t bf16_rne(float x) {
  uint32_t b = __float_as_uint(x);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
__device__ __forceinline__ float bf16_to_f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// Two FP32 values rounded to BF16 (nearest, ties to even) and packed: lo in bits 0-15.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

__device__ __forceinline__ float2 bf16x2_unpack(uint32_t h) {
  return make_float2(__uint_as_float(h << 16), __uint_as_float(h & 0xFFFF0000u));
}

// The exact head / tail split of four FP32 values: h = bf16(v), t = bf16(v - h), packed two per
// word (h01 = values 0, 1); s01 / s23 accumulate (h + t)^2 lane-wise.  The subtractions and sums
// run on packed pairs.
__device__ __forceinline__ void split4_bf16x2(const float4 v, uint2& h, uint2& t, float2& s01, float2& s23) {
  h.x = pack_bf16x2(v.x, v.y);
  h.y = pack_bf16x2(v.z, v.w);
  const float2 f01 = bf16x2_unpack(h.x), f23 = bf16x2_unpack(h.y);
  const float2 d01 = f2_sub(make_float2(v.x, v.y), f01), d23 = f2_sub(make_float2(v.z, v.w), f23);
  t.x = pack_bf16x2(d01.x, d01.y);
  t.y = pack_bf16x2(d23.x, d23.y);
  const float2 g01 = f2_add(f01, bf16x2_unpack(t.x)), g23 = f2_add(f23, bf16x2_unpack(t.y));
  s01 = f2_fma(g01, g01, s01);
  s23 = f2_fma(g23, g23, s23);
}

// The exact three-piece split of four FP32 values: h = bf16(v), m = bf16(v - h), t = bf16(v - h - m)
// with both differences exact (each operand lies within a factor of two of the other) and t exact
// in BF16 (v has 24 significant bits, h and m take the leading 8 each), so v = h + m + t.  s01 /
// s23 accumulate v^2 lane-wise (the pieces add up to v exactly).
__device__ __forceinline__ void split4_bf16x3(const float4 v, uint2& h, uint2& m, uint2& t, float2& s01,
                                              float2& s23) {
  const float2 v01 = make_float2(v.x, v.y), v23 = make_float2(v.z, v.w);
  h.x = pack_bf16x2(v.x, v.y);
  h.y = pack_bf16x2(v.z, v.w);
  const float2 r01 = f2_sub(v01, bf16x2_unpack(h.x)), r23 = f2_sub(v23, bf16x2_unpack(h.y));
  m.x = pack_bf16x2(r01.x, r01.y);
  m.y = pack_bf16x2(r23.x, r23.y);
  const float2 q01 = f2_sub(r01, bf16x2_unpack(m.x)), q23 = f2_sub(r23, bf16x2_unpack(m.y));
  t.x = pack_bf16x2(q01.x, q01.y);
  t.y = pack_bf16x2(q23.x, q23.y);
  s01 = f2_fma(v01, v01, s01);
  s23 = f2_fma(v23, v23, s23);
}

// Split of one float4 into NP = 2 pieces (head, tail: 16 significant bits; s accumulates
// (head + tail)^2) or NP = 3 (exact; s accumulates v^2), stored at byte offset off of each piece.
template <int NP>
__device__ __forceinline__ void split_store(const float4 v, uint8_t* __restrict__ p0, uint8_t* __restrict__ p1,
                                            uint8_t* __restrict__ p2, int off, float2& s01, float2& s23) {
  static_assert(NP == 2 || NP == 3, "two or three pieces");
  if constexpr (NP == 2) {
    uint2 h, tl;
    split4_bf16x2(v, h, tl, s01, s23);
    *reinterpret_cast<uint2*>(p0 + off) = h;
    *reinterpret_cast<uint2*>(p1 + off) = tl;
  } else {
    uint2 h, md, tl;
    split4_bf16x3(v, h, md, tl, s01, s23);
    *reinterpret_cast<uint2*>(p0 + off) = h;
    *reinterpret_cast<uint2*>(p1 + off) = md;
    *reinterpret_cast<uint2*>(p2 + off) = tl;
  }
}

// Split a 32 KB tile of FP32 values staged by TMA (boxes of 32 values x kRowsPerBox rows, 128-byte
// rows, 128-byte swizzle) into its BF16 head and tail, written as 128 rows of 64 values (128-byte
// rows, 128-byte swizzle): box b, row r holds the values 32 (b & 1) .. 32 (b & 1) + 31 of output
// row (b >> 1) kRowsPerBox + r.  Eight consecutive threads read one 128-byte FP32 row (4 values
// each); the four rows of a warp are boxes b, b ^ 1 of two consecutive rows, so its 8-byte stores
// fill whole 128-byte output rows (no bank conflicts).  Returns the FP32 sum of (head + tail)^2
// over the values this thread handled.  NP = 3: three pieces (hi, lo, lo2: exact, split_store) and
// the sum of the values' squares.
template <int kRowsPerBox, int kThreadsConv, int NP = 2>
__device__ __forceinline__ float convert_tile(const uint8_t* __restrict__ f32, uint8_t* __restrict__ hi,
                                              uint8_t* __restrict__ lo, int t, uint8_t* __restrict__ lo2 = nullptr) {
  static_assert(kThreadsConv == 256 && kRowsPerBox >= 128, "unit j of a thread is row 16 j + (t / 16) of box (t / 8) % 2");
  constexpr int kUnits = 2048 / kThreadsConv;
  // unit j of thread t: 16-byte piece k = t % 8 of row r = 16 j + t / 16 of box b = (t / 8) % 2;
  // r % 8 does not depend on j, so both offsets advance by 16 rows (2048 bytes) per unit
  const int k = t & 7, b = (t >> 3) & 1, r0 = t >> 4;
  const uint8_t* src = f32 + b * (kRowsPerBox * 128) + r0 * 128 + ((k ^ (r0 & 7)) << 4);
  const int ci = 4 * b + (k >> 1);
  const int off0 = r0 * 128 + ((ci ^ (r0 & 7)) << 4) + (k & 1) * 8;
  float4 v[kUnits];
#pragma unroll
  for (int j = 0; j < kUnits; ++j) v[j] = *reinterpret_cast<const float4*>(src + j * 2048);   // all loads first
  float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < kUnits; ++j) split_store<NP>(v[j], hi, lo, lo2, off0 + j * 2048, s01, s23);
  return (s01.x + s01.y) + (s23.x + s23.y);
}

// As convert_tile, for a tile staged unswizzled: kPRows columns of 128 consecutive FP32 rows each
// (value (i, p) at byte 512 p + 4 i, one TMA box of 512-byte rows); the output pieces are the same
// (value (p, i) at (i / 64) kPRows 128 + 128 p + ((i % 64 / 8) ^ (p % 8)) 16 + 2 (i % 8)).  A warp
// reads one 512-byte column (conflict-free) and writes two 128-byte output rows.
template <int kPRows, int kThreadsConv, int NP = 2>
__device__ __forceinline__ float convert_tile_plain(const uint8_t* __restrict__ f32, uint8_t* __restrict__ hi,
                                                    uint8_t* __restrict__ lo, int t, uint8_t* __restrict__ lo2 = nullptr) {
  static_assert(kThreadsConv % 256 == 0, "unit j of a thread is column 8 j + (t / 32) of its first one");
  constexpr int kUnits = kPRows * 32 / kThreadsConv;
  constexpr int kColStep = kThreadsConv / 32;   // columns between a thread's consecutive units
  // unit j of thread t: column p = kColStep j + t / 32, rows i = 4 (t % 32) .. + 3; p % 8 does not
  // depend on j, so the swizzled output offset is off0 + 128 kColStep j
  const int p0 = t >> 5, i = (t & 31) * 4;
  const uint8_t* src = f32 + p0 * 512 + (t & 31) * 16;
  const int off0 = (i >> 6) * (kPRows * 128) + p0 * 128 + ((((i & 63) >> 3) ^ (p0 & 7)) << 4) + ((i >> 2) & 1) * 8;
  float4 v[kUnits];
#pragma unroll
  for (int j = 0; j < kUnits; ++j) v[j] = *reinterpret_cast<const float4*>(src + j * kColStep * 512);
  float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < kUnits; ++j) split_store<NP>(v[j], hi, lo, lo2, off0 + j * kColStep * 128, s01, s23);
  return (s01.x + s01.y) + (s23.x + s23.y);
}

// Input kinds of the tensor-core sketch and mode product: BF16 pieces loaded by TMA as they are,
// FP32 values or E4M3 bytes (with per-128-element scales) converted in shared memory; kInF32S, FP32
// values of a mode with L > 1 (its unfolding's rows strided by L, the L-index contiguous), read by
// 3-D boxes over (l, i, r) and converted like kInF32.
constexpr int kInPieces = 0, kInF32 = 1, kInFp8 = 2, kInF32S = 3;

// As convert_tile, for a 128-row x 64-value FP32 tile staged unswizzled with the 64 values of a row
// consecutive (value (row, k) at byte 256 row + 4 k: a 3-D box of 64 l x 128 i): head and tail as
// 128 rows of 64 values in the K-major 128-byte-swizzled layout (value (row, k) at
// (row / 8) 1024 + (row % 8) 128 + ((k / 8) ^ (row % 8)) 16 + 2 (k % 8)).  A warp reads two 256-byte
// rows and writes two 128-byte output rows.
template <int kThreadsConv, int NP = 2>
__device__ __forceinline__ float convert_tile_kmajor(const uint8_t* __restrict__ f32, uint8_t* __restrict__ hi,
                                                     uint8_t* __restrict__ lo, int t, uint8_t* __restrict__ lo2 = nullptr) {
  static_assert(kThreadsConv % 128 == 0, "unit j of a thread is row 16 j + (t / 16) of its first one");
  constexpr int kUnits = 2048 / kThreadsConv;
  constexpr int kRowStep = kThreadsConv / 16;   // rows between a thread's consecutive units
  // unit j of thread t: row 16 j' + t / 16 (kRowStep = 16 j'), values 4 (t % 16) .. + 3; row % 8
  // does not depend on j, so the swizzled output offset is off0 + 128 kRowStep j
  const int r0 = t >> 4, q = t & 15;
  const uint8_t* src = f32 + r0 * 256 + q * 16;
  const int off0 = (r0 >> 3) * 1024 + (r0 & 7) * 128 + (((q >> 1) ^ (r0 & 7)) << 4) + (q & 1) * 8;
  float4 v[kUnits];
#pragma unroll
  for (int j = 0; j < kUnits; ++j) v[j] = *reinterpret_cast<const float4*>(src + j * kRowStep * 256);
  float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < kUnits; ++j) split_store<NP>(v[j], hi, lo, lo2, off0 + j * kRowStep * 128, s01, s23);
  return (s01.x + s01.y) + (s23.x + s23.y);
}

// Value of an E4M3 byte (OCP FP8: 1 sign, 4 exponent bits with bias 7, 3 mantissa bits, no
// infinities, S.1111.111 = NaN) as an FP32 number, exactly: a normal code has value
// 2^(e - 7) (1 + m / 8), i.e. FP32 exponent field e + 120 and the 3 mantissa bits on top of the
// FP32 mantissa; a subnormal code (e = 0) has value m 2^-9.
// The E4M3 values in bits 0-7 (e0) and 8-15 (e1) of w, by the hardware conversion to a pair of
// FP16 values (every E4M3 value, subnormals included, is an FP16 value) and then to FP32: exact,
// and equal to e4m3_to_f32 of each byte for every finite value.
__device__ __forceinline__ void e4m3x2_to_f32(uint32_t w, float& e0, float& e1) {
  const uint16_t b = (uint16_t)(w & 0xFFFFu);
  asm("{\n.reg .b32 h2;\n.reg .b16 lo, hi;\ncvt.rn.f16x2.e4m3x2 h2, %2;\nmov.b32 {lo, hi}, h2;\n"
      "cvt.f32.f16 %0, lo;\ncvt.f32.f16 %1, hi;\n}"
      : "=f"(e0), "=f"(e1)
      : "h"(b));
}

__device__ __forceinline__ float e4m3_to_f32(uint32_t b) {
  const uint32_t e = (b >> 3) & 15u, m = b & 7u;
  float v = e ? __uint_as_float(((e + 120u) << 23) | (m << 20)) : __fmul_rn((float)m, 0x1p-9f);
  if ((b & 0x7Fu) == 0x7Fu) v = __uint_as_float(0x7FC00000u);
  return (b & 0x80u) ? -v : v;
}

// Dequantize a tile of E4M3 values staged by TMA (kPRows rows of kRowBytes bytes, no swizzle; a
// row is one column p of the unfolding, its bytes consecutive rows i) and round it to one BF16
// piece, bf16(x) (ties to even), written in the layout of convert_tile (or, with kTwoPieces, split
// into head and tail exactly as convert_tile does for FP32 input).  The value of storage element
// (i, p) of the tensor (leading dimension ld) is x = fl32(e4m3 * s) with s = scales[(i + ld p) /
// 128]; elements outside the tensor (i >= I or p >= M, zero-filled by TMA) take s = 0.  Output:
// value (p, i) at byte (i / 64) kPRows 128 + 128 p + ((i % 64 / 8) ^ (p % 8)) 16 + 2 (i % 8).  Each
// unit is 16 consecutive bytes of one row; ld % 16 == 0 puts its 16 elements in one scale block.
// Returns the FP32 sum of the squares of the values written (bf16(x), or head + tail).
template <int kRowBytes, int kPRows, int kThreadsConv, bool kTwoPieces = false>
__device__ __forceinline__ float convert_fp8_tile(const uint8_t* __restrict__ src, uint8_t* __restrict__ hi,
                                                  uint8_t* __restrict__ lo, int t, const float* __restrict__ scales,
                                                  int64_t ld, int64_t i0, int64_t p0, int64_t I, int64_t M) {
  constexpr int kUnitsPerRow = kRowBytes / 16;
  constexpr int kUnits = kPRows * kUnitsPerRow / kThreadsConv;
  static_assert(kPRows * kUnitsPerRow % kThreadsConv == 0, "whole units per thread");
  uint4 raw[kUnits];
  float sc[kUnits];
#pragma unroll
  for (int j = 0; j < kUnits; ++j) {
    const int u = j * kThreadsConv + t;
    const int p = u / kUnitsPerRow, il = (u % kUnitsPerRow) * 16;
    raw[j] = *reinterpret_cast<const uint4*>(src + p * kRowBytes + il);
    const int64_t gi = i0 + il, gp = p0 + p;
    sc[j] = (gi < I && gp < M) ? __ldg(scales + ((gi + ld * gp) >> 7)) : 0.0f;
  }
  float ss = 0.0f;
#pragma unroll
  for (int j = 0; j < kUnits; ++j) {
    const int u = j * kThreadsConv + t;
    const int p = u / kUnitsPerRow, il = (u % kUnitsPerRow) * 16;
    const uint32_t w[4] = {raw[j].x, raw[j].y, raw[j].z, raw[j].w};
    uint32_t h[8], tl[8];
    (void)tl;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t word = w[q >> 1] >> (16 * (q & 1));
      float e0, e1;   // the two E4M3 values of the low 16 bits, decoded exactly
      e4m3x2_to_f32(word, e0, e1);
      const float x0 = __fmul_rn(e0, sc[j]);
      const float x1 = __fmul_rn(e1, sc[j]);
      h[q] = pack_bf16x2(x0, x1);
      const float f0 = __uint_as_float(h[q] << 16), f1 = __uint_as_float(h[q] & 0xFFFF0000u);
      if constexpr (kTwoPieces) {
        tl[q] = pack_bf16x2(x0 - f0, x1 - f1);
        const float g0 = f0 + __uint_as_float(tl[q] << 16), g1 = f1 + __uint_as_float(tl[q] & 0xFFFF0000u);
        ss = fmaf(g0, g0, ss);
        ss = fmaf(g1, g1, ss);
      } else {
        ss = fmaf(f0, f0, ss);
        ss = fmaf(f1, f1, ss);
      }
    }
    const int base = (il >> 6) * (kPRows * 128) + p * 128;
    const int c0 = (il & 63) >> 3;
    const int o0 = base + ((c0 ^ (p & 7)) << 4), o1 = base + (((c0 + 1) ^ (p & 7)) << 4);
    *reinterpret_cast<uint4*>(hi + o0) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(hi + o1) = make_uint4(h[4], h[5], h[6], h[7]);
    if constexpr (kTwoPieces) {
      *reinterpret_cast<uint4*>(lo + o0) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
      *reinterpret_cast<uint4*>(lo + o1) = make_uint4(tl[4], tl[5], tl[6], tl[7]);
    }
  }
  return ss;
}

}  // namespace tc
}  // namespace rh
