// Tensor-core (tcgen05) mode product for the first mode of a tensor held as BF16 pieces:
// B = Q^T X_(1) (Alg. 1 step 3), with X_(1) of size I x M, rows contiguous, and Q of size
// I x ell (ell <= 64) given in FP64.
//
// Q is split exactly into two BF16 pieces, Q = Q_h + Q_t (16 significant bits), stacked as the
// 128 x I operand A = [Q_h^T; Q_t^T] (rows >= ell are zero).  For every BF16 piece X_k of X the
// tensor cores accumulate D = A X_k (FP32, in TMEM), so rows c and 64 + c of D hold
// Q_h^T X and Q_t^T X; the epilogue adds them.  All four products Q_a^T X_b are formed, each
// exact, with FP32 accumulation.
//
// Persistent CTAs walk tiles of 128 columns of X_(1).  Per 64-row K-stage, TMA brings the
// 128 x 64 slice of A and the 128 x 64 slices of the X pieces (K-major, 128-byte swizzle);
// MMAs are M = 128, N = 128, K = 16.  The accumulator is double-buffered in TMEM so the
// epilogue of one tile overlaps the MMAs of the next.  Warp roles (192 threads): warp 0 TMA,
// warp 1 TMEM + MMA, warps 2-5 epilogue (warps 2, 3 read the tail rows and hand them to
// warps 4, 5 through shared memory, which add the head rows and store B[c + ell p]).
// FP32 input (448 threads): TMA brings FP32 slices (two 32 x 128 boxes per stage) and warps
// 6-13 split them in shared memory into the head / tail pieces, so B is bit-identical to the
// two-piece form.
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace rh {

rh_status make_bf16_map_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_cols);
rh_status make_map_2d(CUtensorMap* map, const void* base, int esize, int64_t rows, int64_t cols, int box_cols);
rh_status make_u8_map_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t ld, int64_t cols, int box_rows,
                         int box_cols);

namespace {

constexpr int kNTile = 128;   // columns of X_(1) per tile
constexpr int kKStage = 64;   // rows of X_(1) per stage
constexpr uint32_t kATile = 128 * 64 * 2;      // A slice: 128 rows x 64 (BF16)
constexpr uint32_t kXTile = kNTile * 64 * 2;   // X slice: 128 columns x 64 rows (BF16)
constexpr uint32_t kF32Box = kNTile * 32 * 4;  // FP32 TMA box: 32 rows x 128 columns

constexpr uint32_t kFp8Box = kNTile * 64;      // E4M3 TMA box: 64 rows (bytes) x 128 columns

// BF16 pieces in: 3 stages (A slice + pieces) filled by TMA.  FP32 in: 3 stages of FP32 slices
// filled by TMA, split by eight converter warps into 2 stages of pieces; the converters also
// request the A slice of their stage.  E4M3 in: 8 stages of byte slices, dequantized and split
// the same way.
// NP = 3 (FP32 input split exactly into three pieces): one FP32 stage fewer, for the third piece.
template <int IN, int NP = 2>
struct TtmCfg {
  static constexpr bool kConvIn = IN != tc::kInPieces;
  static constexpr int kPStages = kConvIn ? 2 : 3;
  static constexpr bool kF32Like = IN == tc::kInF32 || IN == tc::kInF32S;
  static constexpr int kF32Stages = kF32Like ? (NP == 3 ? 2 : 3) : (IN == tc::kInFp8 ? 8 : 1);
  static constexpr uint32_t kStageBytes = kF32Like ? 2 * kF32Box : (IN == tc::kInFp8 ? kFp8Box : 1024);
  static constexpr int kConv = 256;   // converter threads (warps 6..13)
  static constexpr int kThreads = kConvIn ? 192 + kConv : 192;
};

template <int IN, int NP = 2>
struct alignas(1024) TtmSmem {
  uint8_t xf[TtmCfg<IN, NP>::kF32Stages][TtmCfg<IN, NP>::kStageBytes];
  uint8_t a[TtmCfg<IN, NP>::kPStages][kATile];
  uint8_t x[TtmCfg<IN, NP>::kPStages][NP][kXTile];
  float xchg[64][kNTile + 2];   // rows of 130 floats: pairs of columns 8-byte aligned, lanes c on distinct banks
  uint64_t f32full[TtmCfg<IN, NP>::kF32Stages], f32empty[TtmCfg<IN, NP>::kF32Stages];
  uint64_t full[TtmCfg<IN, NP>::kPStages], empty[TtmCfg<IN, NP>::kPStages], afull[TtmCfg<IN, NP>::kPStages];
  uint64_t tfull[2], tempty[2];
  uint32_t tmem_slot;
};

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// IN = kInPieces: mapX0 / mapX1 are the BF16 pieces (box 64 x 128).  IN = kInF32: mapX0 is the
// FP32 tensor (box 32 x 128), split on the fly into the same two pieces.  IN = kInF32S: a mode with
// L > 1 (L a multiple of 128): mapX0 is the 3-D view (l, i, r), each stage one box of 128 l x 64 i at
// one r, split into MN-major pieces (K = i, N = l), B written through ``co`` in the (L, ell, R)
// layout of the mode product.  IN = kInFp8: mapX0 is
// the E4M3 tensor (box 64 x 128 bytes, leading dimension ld), dequantized with ``scales`` and split.
// One 128-column tile's contribution to the 4 x 4 block (bi, bj) of W = B B^T, B's tile held as
// xc[c][p]: the products of the even and of the odd columns each summed in FP32 in column order
// (the two lanes of packed pairs), their sum added to the FP32 pair (gh, gl) that keeps every
// rounding error (TwoSum).
__device__ __forceinline__ void gram_tile(const float (*xc)[kNTile + 2], int bi, int bj, float (&gh)[4][4],
                                          float (&gl)[4][4]) {
  // even and odd columns in the two lanes of packed FP32 pairs, added at the end of the tile
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.0f, 0.0f);
#pragma unroll 2
  for (int pp = 0; pp < kNTile; pp += 2) {
    float2 xa[4], yb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xa[a] = *reinterpret_cast<const float2*>(&xc[4 * bi + a][pp]);
#pragma unroll
    for (int b = 0; b < 4; ++b) yb[b] = *reinterpret_cast<const float2*>(&xc[4 * bj + b][pp]);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = f2_fma(xa[a], yb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float v = acc[a][b].x + acc[a][b].y;
      const float t = __fadd_rn(gh[a][b], v);
      const float bp = __fsub_rn(t, gh[a][b]);
      gl[a][b] = __fadd_rn(gl[a][b], __fadd_rn(__fsub_rn(gh[a][b], __fsub_rn(t, bp)), __fsub_rn(v, bp)));
      gh[a][b] = t;
    }
}

// kT (FP32 input only; the truncated-core product): the accumulator is transposed, D(p, n) =
// X_k(p, :) A(n, :)^T with the X pieces as operand A (rows p) and [Q_h^T; Q_t^T] as operand B, so
// TMEM lane p holds column p's head sums in columns c and its tail sums in columns 64 + c.  Each
// epilogue warp then finishes its own 32 columns p (no exchange between warps) and writes
// B[co.base(p) + c co.cstride()] with the lanes along p.
// kG (ell <= 60): the epilogue warps also form W = B B^T of the B they write, as the FP32 Gram
// route of the truncation does (each 128-column tile's products summed in FP32 in column order, the
// tile sums accumulated in FP32 pairs), thread t of the four warps owning the t-th 4 x 4 block of
// the upper triangle; gram_part[blockIdx.x] receives the CTA's partial (upper triangle, FP64), so
// the truncation only reduces the partials instead of reading B again.
template <int IN, bool kT = false, int NP = 2, bool kG = false>
__global__ void __launch_bounds__(TtmCfg<IN, NP>::kThreads, 1)
    ttm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX0,
                  const __grid_constant__ CUtensorMap mapX1, int npieces, int64_t I, int64_t M, int ell,
                  float* __restrict__ B, int32_t* __restrict__ err, const float* __restrict__ scales, int64_t ld,
                  CoreOut co, int probe, int64_t L, double* __restrict__ gram_part) {
  using Cfg = TtmCfg<IN, NP>;
  constexpr bool F32IN = Cfg::kConvIn;   // any converted input (FP32 or E4M3)
  constexpr int NS = Cfg::kPStages;
  constexpr int NF = Cfg::kF32Stages;
  extern __shared__ uint8_t smem_raw[];
  TtmSmem<IN, NP>& S =
      *reinterpret_cast<TtmSmem<IN, NP>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (M + kNTile - 1) / kNTile;
  const int kstages = (int)((I + kKStage - 1) / kKStage);
  const uint32_t tmem_cols = 256;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&S.full[s], F32IN ? Cfg::kConv : 1);
      tc::mbar_init(&S.empty[s], 1);
      tc::mbar_init(&S.afull[s], 1);
    }
    if (F32IN) {
      for (int s = 0; s < NF; ++s) {
        tc::mbar_init(&S.f32full[s], 1);
        tc::mbar_init(&S.f32empty[s], Cfg::kConv);
      }
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&S.tfull[b], 1);
      tc::mbar_init(&S.tempty[b], 128);
    }
    tc::fence_mbar_init();
  }
  if (probe) {   // wait-timeout probe: nothing allocated or issued yet
    if (threadIdx.x == 0) tc::mbar_wait(&S.tfull[0], 0, err, tc::kProbeCode, tc::kProbeSpin);
    return;
  }
  if (warp == 1) {
    tc::tmem_alloc(&S.tmem_slot, tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = S.tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      tc::prefetch_tmap(&mapX0);
      if (!F32IN) {
        tc::prefetch_tmap(&mapA);
        if (npieces > 1) tc::prefetch_tmap(&mapX1);
      }
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int32_t p0 = (int32_t)(t * kNTile);
        for (int ks = 0; ks < kstages; ++ks, ++it) {
          if constexpr (F32IN) {
            const uint32_t s = it % NF;
            if (it >= NF && !tc::mbar_wait(&S.f32empty[s], ((it / NF) - 1) & 1, err, 11)) {
              ok = false;
              break;
            }
            if constexpr (IN == tc::kInFp8) {
              tc::mbar_arrive_expect_tx(&S.f32full[s], kFp8Box);
              tc::tma_load_2d(&S.xf[s][0], &mapX0, ks * kKStage, p0, &S.f32full[s]);
            } else if constexpr (IN == tc::kInF32S) {
              tc::mbar_arrive_expect_tx(&S.f32full[s], 2 * kF32Box);
              tc::tma_load_3d(&S.xf[s][0], &mapX0, (int32_t)((int64_t)p0 % L), ks * kKStage,
                              (int32_t)((int64_t)p0 / L), &S.f32full[s]);   // 128 l x 64 i at one r
            } else {
              tc::mbar_arrive_expect_tx(&S.f32full[s], 2 * kF32Box);
              tc::tma_load_2d(&S.xf[s][0], &mapX0, ks * kKStage, p0, &S.f32full[s]);
              tc::tma_load_2d(&S.xf[s][kF32Box], &mapX0, ks * kKStage + 32, p0, &S.f32full[s]);
            }
          } else {
            const uint32_t s = it % NS;
            if (it >= NS && !tc::mbar_wait(&S.empty[s], ((it / NS) - 1) & 1, err, 11)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&S.full[s], kATile + kXTile * (uint32_t)npieces);
            tc::tma_load_2d(&S.a[s][0], &mapA, ks * kKStage, 0, &S.full[s]);
            tc::tma_load_2d(&S.x[s][0][0], &mapX0, ks * kKStage, p0, &S.full[s]);
            if (npieces > 1) tc::tma_load_2d(&S.x[s][1][0], &mapX1, ks * kKStage, p0, &S.full[s]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // A = [Q_h^T; Q_t^T] K-major; B (the X pieces) K-major, or MN-major for a strided mode
      constexpr uint32_t idesc = tc::idesc_bf16(128, kNTile, 0, IN == tc::kInF32S ? 1 : 0);
      uint32_t it = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const uint32_t b = tl & 1;
        if (tl >= 2 && !tc::mbar_wait(&S.tempty[b], ((tl >> 1) - 1) & 1, err, 12)) break;
        tc::tc_fence_after();
        const uint32_t d = tmem + b * kNTile;
        for (int ks = 0; ks < kstages; ++ks, ++it) {
          const uint32_t s = it % NS;
          if (!tc::mbar_wait(&S.full[s], (it / NS) & 1, err, 13) ||
              (F32IN && !tc::mbar_wait(&S.afull[s], (it / NS) & 1, err, 15))) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a_addr = tc::smem_u32(&S.a[s][0]);
          for (int kk = 0; kk < kKStage / 16; ++kk) {
            const uint64_t adesc = tc::sdesc_sw128(a_addr + kk * 32, 16, 1024);
            for (int pc = 0; pc < npieces; ++pc) {
              const uint64_t bdesc = IN == tc::kInF32S
                                         ? tc::sdesc_sw128(tc::smem_u32(&S.x[s][pc][0]) + kk * 2048, 8192, 1024)
                                         : tc::sdesc_sw128(tc::smem_u32(&S.x[s][pc][0]) + kk * 32, 16, 1024);
              if constexpr (kT)
                tc::mma_bf16(d, bdesc, adesc, idesc, (ks == 0 && kk == 0 && pc == 0) ? 0u : 1u);
              else
                tc::mma_bf16(d, adesc, bdesc, idesc, (ks == 0 && kk == 0 && pc == 0) ? 0u : 1u);
            }
          }
          tc::mma_commit(&S.empty[s]);
        }
        tc::mma_commit(&S.tfull[b]);
      }
    }
  } else if (warp < 6) {
    // epilogue: warps 2..5 -> TMEM lane quadrants 2, 3, 0, 1
    const int quad = warp & 3;
    const bool tail = quad >= 2;        // rows 64..127: Q_t^T X
    const int crow = (quad & 1) * 32 + lane;   // output row c (0..63)
    // kG: this thread's 4 x 4 block (gbi, gbj) of the upper triangle of W
    const int et = threadIdx.x - 64;   // 0..127
    int gbi = 0, gbj = et;
    const int gnb = (ell + 3) / 4;
    while (gbi < gnb && gbj >= gnb - gbi) {
      gbj -= gnb - gbi;
      ++gbi;
    }
    gbj += gbi;
    const bool gact = kG && et < gnb * (gnb + 1) / 2;
    float gh[4][4], gl[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) gh[a][b2] = gl[a][b2] = 0.0f;
    uint32_t tl = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const uint32_t b = tl & 1;
      if (!tc::mbar_wait(&S.tfull[b], (tl >> 1) & 1, err, 14)) break;
      tc::tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + b * kNTile;
      if constexpr (kT) {
        const int64_t p = t * kNTile + quad * 32 + lane;
        const int64_t ob = p < M ? co.base(p, ell) : 0;
        const int64_t cs = co.cstride();
        for (int cc = 0; cc < (ell + 15) / 16; ++cc) {
          float h[16], tv[16];
          tc::tmem_ld16(base + (uint32_t)(cc * 16), h);
          tc::tmem_ld16(base + (uint32_t)(64 + cc * 16), tv);
          if (p < M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = cc * 16 + j;
              if (c < ell) B[ob + cs * c] = h[j] + tv[j];
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&S.tempty[b]);
        continue;
      }
      if (tail) {
        for (int cc = 0; cc < kNTile / 16; ++cc) {
          float v[16];
          tc::tmem_ld16(base + cc * 16, v);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float2*>(&S.xchg[crow][cc * 16 + 2 * j]) = make_float2(v[2 * j], v[2 * j + 1]);
        }
      }
      named_sync(1, 128);
      const int64_t p0 = t * kNTile;
      if (co.plain()) {
        // B[c + ell p]: the threads of a warp hold consecutive rows c, so the stores are coalesced
        if (!tail) {
          for (int cc = 0; cc < kNTile / 16; ++cc) {
            float v[16];
            tc::tmem_ld16(base + cc * 16, v);
            if (crow < ell) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float2* xp = reinterpret_cast<float2*>(&S.xchg[crow][cc * 16 + 2 * j]);
                const float2 tv = *xp;
                const float f0 = v[2 * j] + tv.x, f1 = v[2 * j + 1] + tv.y;
                if constexpr (kG) *xp = make_float2(f0, f1);   // this lane's own row
                const int64_t p = p0 + cc * 16 + 2 * j;
                if (p < M) B[crow + (int64_t)ell * p] = f0;
                if (p + 1 < M) B[crow + (int64_t)ell * (p + 1)] = f1;
              }
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&S.tempty[b]);
        if constexpr (kG) {
          named_sync(1, 128);   // the tile's final values are in xchg
          if (gact) gram_tile(S.xchg, gbi, gbj, gh, gl);
        }
      } else {
        // B[co.base(p) + c co.cstride()] (CoreOut): sum the halves in shared memory, then each
        // warp writes whole rows c with its lanes along p
        if (!tail) {
          for (int cc = 0; cc < kNTile / 16; ++cc) {
            float v[16];
            tc::tmem_ld16(base + cc * 16, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float2* xp = reinterpret_cast<float2*>(&S.xchg[crow][cc * 16 + 2 * j]);
              const float2 tv = *xp;
              *xp = make_float2(tv.x + v[2 * j], tv.y + v[2 * j + 1]);
            }
          }
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&S.tempty[b]);
        named_sync(1, 128);
        const int wq = warp - 2;   // 0..3
        const int64_t cs = co.cstride();
        for (int jj = lane; jj < kNTile; jj += 32) {
          const int64_t p = p0 + jj;
          if (p < M) {
            const int64_t base = co.base(p, ell);
            for (int c = wq; c < ell; c += 4) B[base + cs * c] = S.xchg[c][jj];
          }
        }
        if constexpr (kG) {
          if (gact) gram_tile(S.xchg, gbi, gbj, gh, gl);
        }
      }
      named_sync(1, 128);   // xchg is free again
    }
    if constexpr (kG) {
      if (gact) {
        double* o = gram_part + (int64_t)blockIdx.x * ell * ell;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) {
            const int r = 4 * gbi + a, c = 4 * gbj + b2;
            if (r <= c && c < ell) o[r + (int64_t)ell * c] = (double)gh[a][b2] + (double)gl[a][b2];
          }
      }
    }
  } else if constexpr (F32IN) {
    // converters (warps 6..13): FP32 / E4M3 slice -> BF16 head + tail; thread 0 also requests the A slice
    const int t = threadIdx.x - 192;   // 0..kConv-1
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tt = blockIdx.x; tt < ntiles && ok; tt += gridDim.x) {
      for (int ks = 0; ks < kstages; ++ks, ++it) {
        const uint32_t s = it % NF, ps = it % NS;
        if (it >= NS && !tc::mbar_wait(&S.empty[ps], ((it / NS) - 1) & 1, err, 16)) {
          ok = false;
          break;
        }
        if (t == 0) {
          tc::mbar_arrive_expect_tx(&S.afull[ps], kATile);
          tc::tma_load_2d(&S.a[ps][0], &mapA, ks * kKStage, 0, &S.afull[ps]);
        }
        if (!tc::mbar_wait(&S.f32full[s], (it / NF) & 1, err, 17)) {
          ok = false;
          break;
        }
        if constexpr (IN == tc::kInFp8)
          (void)tc::convert_fp8_tile<64, 128, Cfg::kConv>(&S.xf[s][0], &S.x[ps][0][0], nullptr, t, scales, ld,
                                                          (int64_t)ks * kKStage, tt * kNTile, I, M);
        else if constexpr (IN == tc::kInF32S)
          (void)tc::convert_tile_plain<64, Cfg::kConv, NP>(&S.xf[s][0], &S.x[ps][0][0], &S.x[ps][1][0], t,
                                                           NP == 3 ? &S.x[ps][NP - 1][0] : nullptr);
        else
          (void)tc::convert_tile<128, Cfg::kConv, NP>(&S.xf[s][0], &S.x[ps][0][0], &S.x[ps][1][0], t,
                                                      NP == 3 ? &S.x[ps][NP - 1][0] : nullptr);
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&S.f32empty[s]);
        tc::mbar_arrive(&S.full[ps]);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, tmem_cols);
}

// A = [bf16(Q)^T; bf16(Q - bf16(Q))^T] as a 128 x I row-major BF16 matrix with leading dimension
// ldA >= I (ldA % 8 == 0 for the tensor map); rows >= ell and columns >= I are zero.
template <typename TQ>
__global__ void q_pieces_kernel(const TQ* __restrict__ Q, int64_t I, int ell, int64_t ldA, uint16_t* __restrict__ A) {
  const int64_t total = 128 * ldA;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % ldA;
    const int r = (int)(e / ldA);
    const int c = r & 63;
    uint16_t out = 0;
    if (c < ell && i < I) {
      const float q = (float)Q[i + I * c];   // FP64 -> FP32 first (24 bits >= the 16 kept)
      const uint16_t h = tc::bf16_rne(q);
      out = (r < 64) ? h : tc::bf16_rne(q - tc::bf16_to_f(h));
    }
    A[e] = out;
  }
}

}  // namespace

bool ttm_tc_supported(const ModeView& v, int ell) {
  return v.L == 1 && v.I % 8 == 0 && ell >= 1 && ell <= 64 && v.M() < (int64_t(1) << 31);
}

int ttm_tc_ctas(const ModeView& v) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), ceil_div(v.M(), kNTile)));
}

// The launch of a form whose input the producer warp loads as it is (BF16 pieces) or converts
// in one piece (E4M3), with or without the Gram partials of B.
template <int IN>
static rh_status launch_ttm_plain(const CUtensorMap& mA, const CUtensorMap& m0, const CUtensorMap& m1, int np,
                                  const ModeView& v, int ell, float* B, int32_t* err, const float* scales, int64_t ld,
                                  cudaStream_t st, double* gram_part) {
  if (gram_part != nullptr && !ttm_tc_gram_supported(ell)) {
    set_error("internal: Gram partials with the mode product need ell <= 60");
    return RH_EUNSUPPORTED;
  }
  const size_t smem = sizeof(TtmSmem<IN>) + 1024;
  if (gram_part != nullptr) {
    RH_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<IN, false, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    ttm_tc_kernel<IN, false, 2, true><<<ttm_tc_ctas(v), TtmCfg<IN>::kThreads, smem, st>>>(
        mA, m0, m1, np, v.I, v.M(), ell, B, err, scales, ld, CoreOut{}, tc_probe_next(), 1, gram_part);
  } else {
    RH_CUDA_TRY(cudaFuncSetAttribute(ttm_tc_kernel<IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ttm_tc_kernel<IN><<<ttm_tc_ctas(v), TtmCfg<IN>::kThreads, smem, st>>>(
        mA, m0, m1, np, v.I, v.M(), ell, B, err, scales, ld, CoreOut{}, tc_probe_next(), 1, nullptr);
  }
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_ttm_tc(const ModeView& v, int ell, const uint16_t* piece0, const uint16_t* piece1, const double* Q,
                        uint16_t* qa, float* B, int32_t* err, cudaStream_t st, double* gram_part) {
  if (!ttm_tc_supported(v, ell)) {
    set_error("tensor-core mode product: unsupported shape (needs the first mode, I % 8 == 0, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  {
    const int64_t total = 128 * v.I;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 2 * num_sms()));
    q_pieces_kernel<double><<<blocks, 256, 0, st>>>(Q, v.I, ell, v.I, qa);
    RH_LAUNCH_CHECK();
  }
  CUtensorMap mA, m0, m1;
  rh_status s = make_bf16_map_2d(&mA, qa, v.I, 128, 128);
  if (s != RH_OK) return s;
  if ((s = make_bf16_map_2d(&m0, piece0, v.I, v.M(), kNTile)) != RH_OK) return s;
  const int np = piece1 ? 2 : 1;
  if (piece1) {
    if ((s = make_bf16_map_2d(&m1, piece1, v.I, v.M(), kNTile)) != RH_OK) return s;
  } else {
    m1 = m0;
  }
  return launch_ttm_plain<tc::kInPieces>(mA, m0, m1, np, v, ell, B, err, nullptr, 0, st, gram_part);
}

// A converted-input launch (FP32 split on the fly into NP pieces); kG: with the Gram partials of B.
template <int IN, bool kT, int NP, bool kG = false>
static rh_status launch_ttm_conv(const CUtensorMap& mA, const CUtensorMap& m0, const ModeView& v, int64_t I, int64_t M,
                                 int ell, float* B, int32_t* err, CoreOut co, int64_t L, cudaStream_t st,
                                 double* gram_part = nullptr) {
  const size_t smem = sizeof(TtmSmem<IN, NP>) + 1024;
  RH_CUDA_TRY(
      cudaFuncSetAttribute(ttm_tc_kernel<IN, kT, NP, kG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ttm_tc_kernel<IN, kT, NP, kG><<<ttm_tc_ctas(v), TtmCfg<IN, NP>::kThreads, smem, st>>>(
      mA, m0, m0, NP, I, M, ell, B, err, nullptr, 0, co, tc_probe_next(), L, gram_part);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

// The Gram partials of B ride along with the mode product when its rows fit the epilogue's blocks.
bool ttm_tc_gram_supported(int ell) { return ell >= 1 && ell <= 60; }

rh_status launch_ttm_tc_f32(const ModeView& v, int ell, const float* X, const double* Q, uint16_t* qa, float* B,
                            int32_t* err, cudaStream_t st, int pieces, double* gram_part) {
  if (!ttm_tc_supported(v, ell)) {
    set_error("tensor-core mode product: unsupported shape (needs the first mode, I % 8 == 0, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  {
    const int64_t total = 128 * v.I;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 2 * num_sms()));
    q_pieces_kernel<double><<<blocks, 256, 0, st>>>(Q, v.I, ell, v.I, qa);
    RH_LAUNCH_CHECK();
  }
  CUtensorMap mA, m0;
  rh_status s = make_bf16_map_2d(&mA, qa, v.I, 128, 128);
  if (s != RH_OK) return s;
  if ((s = make_map_2d(&m0, X, 4, v.I, v.M(), kNTile)) != RH_OK) return s;
  if (gram_part != nullptr && !ttm_tc_gram_supported(ell)) {
    set_error("internal: Gram partials with the mode product need ell <= 60");
    return RH_EUNSUPPORTED;
  }
  if (gram_part != nullptr)
    return pieces == 3
               ? launch_ttm_conv<tc::kInF32, false, 3, true>(mA, m0, v, v.I, v.M(), ell, B, err, CoreOut{}, 1, st,
                                                             gram_part)
               : launch_ttm_conv<tc::kInF32, false, 2, true>(mA, m0, v, v.I, v.M(), ell, B, err, CoreOut{}, 1, st,
                                                             gram_part);
  return pieces == 3 ? launch_ttm_conv<tc::kInF32, false, 3>(mA, m0, v, v.I, v.M(), ell, B, err, CoreOut{}, 1, st)
                     : launch_ttm_conv<tc::kInF32, false, 2>(mA, m0, v, v.I, v.M(), ell, B, err, CoreOut{}, 1, st);
}

rh_status make_map_3d_f32(CUtensorMap* map, const void* base, int64_t L, int64_t I, int64_t R, int box0, int box1);

// A mode with L > 1 on the tensor cores: L a multiple of 128 (every 128-column tile inside one r
// block), ell <= 64, B in the (L, ell, R) layout of the mode product.
bool ttm_tc_strided_supported(const ModeView& v, int ell) {
  return v.L > 1 && v.L % 128 == 0 && v.I >= 1 && ell >= 1 && ell <= 64 && v.M() < (int64_t(1) << 31) &&
         v.R < (int64_t(1) << 31);
}

rh_status launch_ttm_tc_f32s(const ModeView& v, int ell, const float* X, const double* Q, uint16_t* qa, float* B,
                             int32_t* err, cudaStream_t st, int pieces, double* gram_part) {
  if (!ttm_tc_strided_supported(v, ell)) {
    set_error("tensor-core mode product: unsupported strided shape (needs L % 128 == 0, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  const int64_t ldA = (v.I + 7) / 8 * 8;
  {
    const int64_t total = 128 * ldA;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 2 * num_sms()));
    q_pieces_kernel<double><<<blocks, 256, 0, st>>>(Q, v.I, ell, ldA, qa);
    RH_LAUNCH_CHECK();
  }
  CUtensorMap mA, m0;
  rh_status s = make_bf16_map_2d(&mA, qa, ldA, 128, 128);
  if (s != RH_OK) return s;
  if ((s = make_map_3d_f32(&m0, X, v.L, v.I, v.R, kNTile, kKStage)) != RH_OK) return s;
  const CoreOut co = CoreOut::make(1, v.L, 1, v.M());
  if (gram_part != nullptr && !ttm_tc_gram_supported(ell)) {
    set_error("internal: Gram partials with the mode product need ell <= 60");
    return RH_EUNSUPPORTED;
  }
  if (gram_part != nullptr)
    return pieces == 3
               ? launch_ttm_conv<tc::kInF32S, false, 3, true>(mA, m0, v, v.I, v.M(), ell, B, err, co, v.L, st, gram_part)
               : launch_ttm_conv<tc::kInF32S, false, 2, true>(mA, m0, v, v.I, v.M(), ell, B, err, co, v.L, st, gram_part);
  return pieces == 3 ? launch_ttm_conv<tc::kInF32S, false, 3>(mA, m0, v, v.I, v.M(), ell, B, err, co, v.L, st)
                     : launch_ttm_conv<tc::kInF32S, false, 2>(mA, m0, v, v.I, v.M(), ell, B, err, co, v.L, st);
}

bool core_product_tc_supported(int ell, int ko, int64_t M) {
  return ell >= 1 && ell <= 64 && ell % 4 == 0 && ko >= 1 && ko <= 64 && M >= 1 && M < (int64_t(1) << 31);
}

rh_status launch_core_product_tc(const float* B, int ell, int ko, int64_t M, CoreOut co, const float* U, uint16_t* qa,
                                 float* out, int32_t* err, cudaStream_t st, int pieces) {
  if (!core_product_tc_supported(ell, ko, M) || co.S < 1 || co.I < 1 || co.Ln < 1 || M % (co.S * co.I) != 0) {
    set_error("tensor-core core product: unsupported shape (needs ell % 4 == 0, ell, r <= 64)");
    return RH_EUNSUPPORTED;
  }
  const int64_t ldA = (ell + 7) / 8 * 8;
  {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(128 * ldA, 256), 2 * num_sms()));
    q_pieces_kernel<float><<<blocks, 256, 0, st>>>(U, ell, ko, ldA, qa);
    RH_LAUNCH_CHECK();
  }
  CUtensorMap mA, m0;
  rh_status s = make_bf16_map_2d(&mA, qa, ldA, 128, 128);
  if (s != RH_OK) return s;
  if ((s = make_map_2d(&m0, B, 4, ell, M, kNTile)) != RH_OK) return s;
  const ModeView v{1, (int64_t)ell, M};
  return pieces == 3 ? launch_ttm_conv<tc::kInF32, true, 3>(mA, m0, v, ell, M, ko, out, err, co, 1, st)
                     : launch_ttm_conv<tc::kInF32, true, 2>(mA, m0, v, ell, M, ko, out, err, co, 1, st);
}

rh_status launch_ttm_tc_fp8(const ModeView& v, int ell, const uint8_t* X, const float* scales, int64_t ld,
                            const double* Q, uint16_t* qa, float* B, int32_t* err, cudaStream_t st, double* gram_part) {
  if (!ttm_tc_supported(v, ell) || ld < v.I || ld % 16 != 0) {
    set_error("tensor-core mode product: unsupported E4M3 shape (needs the first mode, I % 8 == 0, ell <= 64, "
              "a leading dimension that is a multiple of 16)");
    return RH_EUNSUPPORTED;
  }
  {
    const int64_t total = 128 * v.I;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 2 * num_sms()));
    q_pieces_kernel<double><<<blocks, 256, 0, st>>>(Q, v.I, ell, v.I, qa);
    RH_LAUNCH_CHECK();
  }
  CUtensorMap mA, m0;
  rh_status s = make_bf16_map_2d(&mA, qa, v.I, 128, 128);
  if (s != RH_OK) return s;
  if ((s = make_u8_map_2d(&m0, X, v.I, ld, v.M(), 64, kNTile)) != RH_OK) return s;
  return launch_ttm_plain<tc::kInFp8>(mA, m0, m0, 1, v, ell, B, err, scales, ld, st, gram_part);
}

}  // namespace rh
