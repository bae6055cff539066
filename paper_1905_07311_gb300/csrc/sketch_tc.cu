// Tensor-core (tcgen05) sketch Y = X_(1) Omega for the first mode of a tensor held as BF16
// pieces (Alg. 1 step 1 on the unfolding whose rows are contiguous, i.e. the mode with L = 1).
//
// Input representation ("BF16 pieces"): X = X_1 + ... + X_np with each X_k a BF16 array of the
// tensor's shape (np = 1: a BF16 tensor; np = 2: an FP32 tensor split exactly into a BF16 head
// and a BF16 tail, 16 significant bits).  Omega is the library's Gaussian stream rounded to
// BF16 (ties to even), so every product is exact and sums run in FP32 inside TMEM.
//
// Grid: persistent CTAs, each taking every gridDim.x-th 64-column chunk of X_(1) (split-K).
// A CTA keeps the accumulators of all row tiles (I <= 128 * kMaxTiles rows x 64 columns, FP32)
// in TMEM, so each Omega tile is generated once and used by every row tile.
// Warp roles (192 threads): warp 0 issues TMA loads of the X pieces (128 x 64 tiles, MN-major
// operand A, 128-byte swizzle); warp 1 owns TMEM and issues the MMAs (M = 128, N = 64, K = 16);
// warps 2-5 generate the 64 x 64 Omega tile (K-major operand B, 128-byte swizzle) and, at the
// end, read the accumulators back and write this CTA's partial sketch [I x ell] (FP32).
//
// FP32 input (448 threads): TMA brings FP32 tiles (one unswizzled 128 x 64 box: 512-byte column
// segments) and warps 6-13 split them in shared memory into the same head / tail pieces that the
// separate split produces, so the products, and the sketch, are bit-identical to the two-piece
// form; they also accumulate ||head + tail||^2 for the norm of the input.
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"
#include "tc.cuh"

namespace rh {
namespace {

constexpr int kRowsTile = 128;
constexpr int kPChunk = 64;
constexpr int kMaxTiles = 8;     // 8 x 64 FP32 columns = all 512 TMEM columns
constexpr uint32_t kHalfBox = 64 * 64 * 2;          // one TMA box: 64 rows x 64 columns, BF16
constexpr uint32_t kPieceTile = 2 * kHalfBox;       // 128 x 64 BF16
constexpr uint32_t kOmegaTile = 64 * 64 * 2;        // 64 x 64 BF16
constexpr uint32_t kF32Box = 32 * 64 * 4;           // FP32 TMA box: 32 rows x 64 columns
constexpr uint32_t kF32Tile = 4 * kF32Box;          // 128 x 64 FP32

constexpr uint32_t kFp8Tile = 128 * 64;           // E4M3 TMA box: 128 rows (bytes) x 64 columns
constexpr int kOmBufs = 2;                        // Omega tiles in flight (generated ahead of the MMAs)

// BF16 pieces in: 4 stages filled by TMA.  FP32 in: 3 stages of FP32 tiles filled by TMA, split by
// eight converter warps into 2 stages of BF16 pieces (a fourth stage measured no faster).  E4M3
// in: 12 stages of byte tiles (96 KB in flight), dequantized and split the same way.
template <int IN>
struct SketchCfg {
  static constexpr bool kConvIn = IN != tc::kInPieces;
  static constexpr int kPStages = kConvIn ? 2 : 4;
  static constexpr bool kF32Like = IN == tc::kInF32 || IN == tc::kInF32S;
  static constexpr int kF32Stages = kF32Like ? 3 : (IN == tc::kInFp8 ? 12 : 1);
  static constexpr uint32_t kStageBytes = kF32Like ? kF32Tile : (IN == tc::kInFp8 ? kFp8Tile : 1024);
  static constexpr int kConv = 256;   // converter threads (warps 6..13)
  static constexpr int kThreads = kConvIn ? 192 + kConv : 192;
};

template <int IN, int NP = 2>
struct alignas(1024) SketchSmem {
  uint8_t xf[SketchCfg<IN>::kF32Stages][SketchCfg<IN>::kStageBytes];
  uint8_t x[SketchCfg<IN>::kPStages][NP][kPieceTile];   // [stage][piece][128 x 64]
  uint8_t om[kOmBufs][kOmegaTile];
  uint64_t f32full[SketchCfg<IN>::kF32Stages], f32empty[SketchCfg<IN>::kF32Stages];
  uint64_t full[SketchCfg<IN>::kPStages], empty[SketchCfg<IN>::kPStages], om_full[kOmBufs], om_empty[kOmBufs], done;
  uint32_t tmem_slot;
  double nrm[16];
};

// byte offset of element (row, col) of a K-major 128B-swizzled tile whose rows hold 64 BF16
__device__ __forceinline__ uint32_t sw128_off(int row, int col) {
  const int chunk = (col >> 3) ^ (row & 7);
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + chunk * 16 + (col & 7) * 2);
}

// IN = kInPieces: map0 / map1 are the BF16 pieces (box 64 x 64).  IN = kInF32: map0 is the FP32
// tensor (one unswizzled 128 x 64 box), split on the fly.  IN = kInF32S: a mode with L > 1 (L a
// multiple of 64): map0 is the 3-D view (l, i, r) of the FP32 tensor, each chunk one box of 64 l x
// 128 i at one r (chunk c covers Kolda columns 64 c .. 64 c + 63, all inside one r block), split on
// the fly into K-major pieces (rows i, K = l).  IN = kInFp8: map0 is the E4M3 tensor
// (box 128 x 64 bytes, leading dimension ld), dequantized with ``scales`` and rounded to one BF16
// piece on the fly (npieces = 1).  With converted
// input, norm_part[blockIdx.x] receives this CTA's sum of squares of the split values (head + tail).
// NP = 3 (FP32 input): the values are split exactly into three BF16 pieces (npieces = 3), three
// MMAs per K step, and the norm is that of the FP32 values themselves.
template <int IN, int NP = 2>
__global__ void __launch_bounds__(SketchCfg<IN>::kThreads, 1)
    sketch_tc_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1, int npieces,
                     int64_t I, int64_t M, int ell, int mtiles, int64_t chunks_per_cta, uint32_t k0, uint32_t k1,
                     uint32_t sid, float* __restrict__ part, double* __restrict__ norm_part,
                     int32_t* __restrict__ err, const float* __restrict__ scales, int64_t ld, int probe,
                     int64_t row0, int64_t L) {
  using Cfg = SketchCfg<IN>;
  constexpr bool F32IN = Cfg::kConvIn;   // any converted input (FP32 or E4M3)
  constexpr int NS = Cfg::kPStages;
  constexpr int NF = Cfg::kF32Stages;
  extern __shared__ uint8_t smem_raw[];
  SketchSmem<IN, NP>& S =
      *reinterpret_cast<SketchSmem<IN, NP>*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nchunks = (M + kPChunk - 1) / kPChunk;
  // chunks are dealt round-robin (c = blockIdx.x, blockIdx.x + gridDim.x, ...)
  (void)chunks_per_cta;
  const int64_t c_begin = blockIdx.x, c_step = gridDim.x, c_end = nchunks;
  const uint32_t tmem_cols = (uint32_t)(mtiles <= 1 ? 64 : (mtiles <= 2 ? 128 : (mtiles <= 4 ? 256 : 512)));

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&S.full[s], F32IN ? Cfg::kConv : 1);
      tc::mbar_init(&S.empty[s], 1);
    }
    if (F32IN) {
      for (int s = 0; s < NF; ++s) {
        tc::mbar_init(&S.f32full[s], 1);
        tc::mbar_init(&S.f32empty[s], Cfg::kConv);
      }
    }
    for (int b = 0; b < kOmBufs; ++b) {
      tc::mbar_init(&S.om_full[b], 128);
      tc::mbar_init(&S.om_empty[b], 1);
    }
    tc::mbar_init(&S.done, 1);
    tc::fence_mbar_init();
  }
  if (probe) {   // wait-timeout probe: nothing allocated or issued yet
    if (threadIdx.x == 0) tc::mbar_wait(&S.done, 0, err, tc::kProbeCode, tc::kProbeSpin);
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
    // ---------------- TMA producer ----------------
    if (lane == 0 && c_begin < c_end) {
      tc::prefetch_tmap(&map0);
      if (!F32IN && npieces > 1) tc::prefetch_tmap(&map1);
      uint32_t it = 0;
      for (int64_t c = c_begin; c < c_end; c += c_step) {
        const int32_t p0 = (int32_t)(c * kPChunk);
        for (int m = 0; m < mtiles; ++m, ++it) {
          if constexpr (F32IN) {
            const uint32_t s = it % NF;
            if (it >= NF && !tc::mbar_wait(&S.f32empty[s], ((it / NF) - 1) & 1, err, 1)) break;
            if constexpr (IN == tc::kInFp8) {
              tc::mbar_arrive_expect_tx(&S.f32full[s], kFp8Tile);
              tc::tma_load_2d(&S.xf[s][0], &map0, m * kRowsTile, p0, &S.f32full[s]);
            } else if constexpr (IN == tc::kInF32S) {
              tc::mbar_arrive_expect_tx(&S.f32full[s], kF32Tile);
              tc::tma_load_3d(&S.xf[s][0], &map0, (int32_t)(((int64_t)p0) % L), m * kRowsTile,
                              (int32_t)(((int64_t)p0) / L), &S.f32full[s]);   // 64 l x 128 i at one r
            } else {
              tc::mbar_arrive_expect_tx(&S.f32full[s], kF32Tile);
              tc::tma_load_2d(&S.xf[s][0], &map0, m * kRowsTile, p0, &S.f32full[s]);   // 128 x 64, unswizzled
            }
          } else {
            const uint32_t s = it % NS;
            if (it >= NS && !tc::mbar_wait(&S.empty[s], ((it / NS) - 1) & 1, err, 1)) break;
            tc::mbar_arrive_expect_tx(&S.full[s], kPieceTile * (uint32_t)npieces);
            for (int pc = 0; pc < npieces; ++pc) {
              const CUtensorMap* mp = pc == 0 ? &map0 : &map1;
              tc::tma_load_2d(&S.x[s][pc][0], mp, m * kRowsTile, p0, &S.full[s]);
              tc::tma_load_2d(&S.x[s][pc][kHalfBox], mp, m * kRowsTile + 64, p0, &S.full[s]);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0 && c_begin < c_end) {
      // A (the X pieces) MN-major, or K-major for a strided mode; B (Omega) K-major
      constexpr uint32_t idesc = tc::idesc_bf16(128, 64, IN == tc::kInF32S ? 0 : 1, 0);
      uint32_t it = 0, oc = 0;
      bool first = true;
      for (int64_t c = c_begin; c < c_end; c += c_step, ++oc) {
        const uint32_t b = oc % kOmBufs;
        if (!tc::mbar_wait(&S.om_full[b], (oc / kOmBufs) & 1, err, 2)) break;
        tc::tc_fence_after();
        const uint32_t om_addr = tc::smem_u32(&S.om[b][0]);
        for (int m = 0; m < mtiles; ++m, ++it) {
          const uint32_t s = it % NS;
          if (!tc::mbar_wait(&S.full[s], (it / NS) & 1, err, 3)) break;
          tc::tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(m * 64);
          for (int kk = 0; kk < kPChunk / 16; ++kk) {
            const uint64_t bdesc = tc::sdesc_sw128(om_addr + kk * 32, 16, 1024);
            for (int pc = 0; pc < npieces; ++pc) {
              const uint64_t adesc = IN == tc::kInF32S
                                         ? tc::sdesc_sw128(tc::smem_u32(&S.x[s][pc][0]) + kk * 32, 16, 1024)
                                         : tc::sdesc_sw128(tc::smem_u32(&S.x[s][pc][0]) + kk * 2048, 8192, 1024);
              tc::mma_bf16(d, adesc, bdesc, idesc, (first && kk == 0 && pc == 0) ? 0u : 1u);
            }
          }
          tc::mma_commit(&S.empty[s]);
        }
        tc::mma_commit(&S.om_empty[b]);
        first = false;
      }
      tc::mma_commit(&S.done);
    }
  } else if (warp < 6) {
    // ---------------- Omega generators (warps 2..5) ----------------
    const int t = threadIdx.x - 64;   // 0..127
    const int p = t & 63;             // column of X_(1) within the chunk (K index)
    // only the ceil(ell / 4) quads of Omega that reach the output are generated; the N columns
    // past them are zeroed once in both buffers (their accumulator columns are never read)
    const int nq = (ell + 3) / 4;
    for (int b = 0; b < kOmBufs; ++b)
      for (int n = 4 * nq + (t >> 6); n < 64; n += 2) *reinterpret_cast<uint16_t*>(&S.om[b][0] + sw128_off(n, p)) = 0;
    uint32_t oc = 0;
    for (int64_t c = c_begin; c < c_end; c += c_step, ++oc) {
      const uint32_t b = oc % kOmBufs;
      if (oc >= kOmBufs && !tc::mbar_wait(&S.om_empty[b], ((oc / kOmBufs) - 1) & 1, err, 4)) break;
      uint8_t* om = &S.om[b][0];
      const int64_t row = row0 + c * kPChunk + p;
      for (int q = t >> 6; q < nq; q += 2) {
        float4 v = rng::omega4(k0, k1, sid, row, (uint32_t)q);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = 4 * q + j;    // column of Omega (N index); columns ell .. 4 nq - 1 are unused
          *reinterpret_cast<uint16_t*>(om + sw128_off(n, p)) = tc::bf16_rne(vv[j]);
        }
      }
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&S.om_full[b]);
    }
    // ---------------- epilogue ----------------
    if (c_begin < c_end && tc::mbar_wait(&S.done, 0, err, 5)) {
      tc::tc_fence_after();
      const int quad = warp & 3;      // TMEM lanes 32 quad .. 32 quad + 31
      for (int m = 0; m < mtiles; ++m) {
        const int64_t i = (int64_t)m * kRowsTile + quad * 32 + lane;
        for (int cc = 0; cc < 4; ++cc) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(m * 64 + cc * 16), v);
          if (i < I) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int col = cc * 16 + j;
              if (col < ell) part[((int64_t)blockIdx.x * ell + col) * I + i] = v[j];
            }
          }
        }
      }
    } else if (c_begin >= c_end) {
      // no work: this CTA's partial is zero
      for (int64_t e = t; e < (int64_t)ell * I; e += 128) part[(int64_t)blockIdx.x * ell * I + e] = 0.0f;
    }
  } else if constexpr (F32IN) {
    // ---------------- converters (warps 6..13): FP32 / E4M3 tile -> BF16 head + tail -----------
    const int t = threadIdx.x - 192;   // 0..kConv-1
    double acc = 0.0;
    uint32_t it = 0;
    bool ok = true;
    for (int64_t c = c_begin; c < c_end && ok; c += c_step) {
      for (int m = 0; m < mtiles; ++m, ++it) {
        const uint32_t s = it % NF, ps = it % NS;
        if (!tc::mbar_wait(&S.f32full[s], (it / NF) & 1, err, 6) ||
            (it >= NS && !tc::mbar_wait(&S.empty[ps], ((it / NS) - 1) & 1, err, 7))) {
          ok = false;
          break;
        }
        if constexpr (IN == tc::kInFp8)
          acc += (double)tc::convert_fp8_tile<128, 64, Cfg::kConv>(&S.xf[s][0], &S.x[ps][0][0], nullptr, t, scales,
                                                                   ld, (int64_t)m * kRowsTile, c * kPChunk, I, M);
        else if constexpr (IN == tc::kInF32S)
          acc += (double)tc::convert_tile_kmajor<Cfg::kConv, NP>(&S.xf[s][0], &S.x[ps][0][0], &S.x[ps][1][0], t,
                                                                 NP == 3 ? &S.x[ps][NP - 1][0] : nullptr);
        else
          acc += (double)tc::convert_tile_plain<64, Cfg::kConv, NP>(&S.xf[s][0], &S.x[ps][0][0], &S.x[ps][1][0], t,
                                                                    NP == 3 ? &S.x[ps][NP - 1][0] : nullptr);
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&S.f32empty[s]);
        tc::mbar_arrive(&S.full[ps]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) S.nrm[warp - 6] = acc;
    asm volatile("bar.sync 2, %0;" ::"n"(Cfg::kConv) : "memory");
    if (t == 0 && norm_part != nullptr) {
      double sum = 0.0;
      for (int w = 0; w < Cfg::kConv / 32; ++w) sum += S.nrm[w];
      norm_part[blockIdx.x] = sum;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, tmem_cols);
}

// X_1 = bf16(x), X_2 = bf16(x - X_1): an exact-to-16-bits split of an FP32 tensor.
__global__ void split_bf16x2_kernel(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ h,
                                    uint16_t* __restrict__ l) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[e];
    const uint16_t a = tc::bf16_rne(v);
    h[e] = a;
    l[e] = tc::bf16_rne(v - tc::bf16_to_f(a));
  }
}

// ||a + b||^2 of BF16 pieces: head + tail is exact in FP32 (16 significant bits), each square is
// formed exactly as p + e (p = v v, e = fma(v, v, -p)) and summed in double-float (TwoSum on the
// high part, the rounding errors and e collected in the low part: ~2^-44 relative), converted to
// FP64 once per thread -- FP64 itself runs at a small fraction of the FP32 rate on this part.
// 16-byte loads when both pieces are 16-byte aligned.
__global__ void pieces_sumsq_kernel(const uint16_t* __restrict__ a, const uint16_t* __restrict__ b, int64_t n,
                                    double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const bool vec = (reinterpret_cast<uintptr_t>(a) % 16 == 0) && (b == nullptr || reinterpret_cast<uintptr_t>(b) % 16 == 0);
  int64_t done = 0;
  if (vec) {
    float sh = 0.0f, sl = 0.0f;
    const int64_t n8 = n / 8;
    for (int64_t q = tid; q < n8; q += nth) {
      const uint4 ha = __ldg(reinterpret_cast<const uint4*>(a) + q);
      uint4 hb = make_uint4(0u, 0u, 0u, 0u);
      if (b) hb = __ldg(reinterpret_cast<const uint4*>(b) + q);
      const uint32_t wa[4] = {ha.x, ha.y, ha.z, ha.w}, wb[4] = {hb.x, hb.y, hb.z, hb.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t ua = (k & 1) ? (wa[k >> 1] & 0xFFFF0000u) : (wa[k >> 1] << 16);
        const uint32_t ub = (k & 1) ? (wb[k >> 1] & 0xFFFF0000u) : (wb[k >> 1] << 16);
        const float v = __fadd_rn(__uint_as_float(ua), __uint_as_float(ub));
        const float pr = __fmul_rn(v, v);
        const float pe = fmaf(v, v, -pr);
        const float t = __fadd_rn(sh, pr);
        const float bb = __fsub_rn(t, sh);
        const float se = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(pr, bb));
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(se, pe));
      }
    }
    s = (double)sh + (double)sl;
    done = n8 * 8;
  }
  for (int64_t e = done + tid; e < n; e += nth) {
    double v = (double)tc::bf16_to_f(a[e]);
    if (b) v += (double)tc::bf16_to_f(b[e]);
    s = fma(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    part[blockIdx.x] = t;
  }
}

// *out (+)= sum of part[0 .. n): one warp, lane l sums part[l], part[l + 32], ..., then a fixed
// butterfly over the lanes (deterministic)
__global__ void sum_n_kernel(const double* __restrict__ part, int n, double* __restrict__ out, int accumulate) {
  if (blockIdx.x != 0) return;
  const int l = threadIdx.x;
  double t = 0.0;
  for (int k = l; k < n; k += 32) t += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (l == 0) *out = accumulate ? *out + t : t;
}

// ---- tensor maps (driver entry point, no link-time dependency on libcuda) ----------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_enc_mu;
EncodeTiledFn g_enc = nullptr;

rh_status get_encoder(EncodeTiledFn* fn) {
  std::lock_guard<std::mutex> lk(g_enc_mu);
  if (!g_enc) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    // the cuTensorMapEncodeTiled ABI as introduced in CUDA 12.0
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return RH_ECUDA;
    }
    g_enc = reinterpret_cast<EncodeTiledFn>(p);
  }
  *fn = g_enc;
  return RH_OK;
}

}  // namespace

// 2-D tensor map over a rows x cols column-major matrix (rows contiguous) of BF16 (esize 2) or
// FP32 (esize 4) values; box (128 bytes of rows) x box_cols, 128-byte swizzle, zero fill outside.
rh_status make_map_2d(CUtensorMap* map, const void* base, int esize, int64_t rows, int64_t cols, int box_cols) {
  EncodeTiledFn enc;
  rh_status s = get_encoder(&enc);
  if (s != RH_OK) return s;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)rows * (cuuint64_t)esize};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return RH_ECUDA;
  }
  return RH_OK;
}

rh_status make_bf16_map_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_cols) {
  return make_map_2d(map, base, 2, rows, cols, box_cols);
}

// 2-D tensor map over a rows x cols column-major FP32 / BF16 matrix, box box_rows x box_cols, no
// swizzle (rows of box_rows * esize bytes, at most 256 elements), zero fill outside.
rh_status make_map_2d_plain(CUtensorMap* map, const void* base, int esize, int64_t rows, int64_t cols, int box_rows,
                            int box_cols) {
  EncodeTiledFn enc;
  rh_status s = get_encoder(&enc);
  if (s != RH_OK) return s;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)rows * (cuuint64_t)esize};
  const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, esize == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (plain) failed with code " + std::to_string((int)r));
    return RH_ECUDA;
  }
  return RH_OK;
}

// 2-D tensor map over bytes: rows x cols, column-major with leading dimension ld (a multiple of
// 16), box box_rows x box_cols, no swizzle, zero fill outside rows x cols.
rh_status make_u8_map_2d(CUtensorMap* map, const void* base, int64_t rows, int64_t ld, int64_t cols, int box_rows,
                         int box_cols) {
  EncodeTiledFn enc;
  rh_status s = get_encoder(&enc);
  if (s != RH_OK) return s;
  const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (bytes) failed with code " + std::to_string((int)r));
    return RH_ECUDA;
  }
  return RH_OK;
}

// 3-D tensor map over an FP32 tensor viewed as (L, I, R) (l fastest), box 64 l x 128 i x 1 r, no
// swizzle, zero fill outside; needs L % 4 == 0 (16-byte strides).
rh_status make_map_3d_f32(CUtensorMap* map, const void* base, int64_t L, int64_t I, int64_t R, int box0, int box1) {
  EncodeTiledFn enc;
  rh_status s = get_encoder(&enc);
  if (s != RH_OK) return s;
  const cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)I, (cuuint64_t)R};
  const cuuint64_t strides[2] = {(cuuint64_t)L * 4, (cuuint64_t)L * (cuuint64_t)I * 4};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (3-D) failed with code " + std::to_string((int)r));
    return RH_ECUDA;
  }
  return RH_OK;
}

// A mode with L > 1 on the tensor cores: L a multiple of 64 (every 64-column chunk inside one r
// block; 16-byte strides), at most 1024 rows, ell <= 64.
bool sketch_tc_strided_supported(const ModeView& v, int ell) {
  return v.L > 1 && v.L % 64 == 0 && v.I >= 1 && v.I <= (int64_t)kRowsTile * kMaxTiles && ell >= 1 && ell <= 64 &&
         v.M() < (int64_t(1) << 31) && v.R < (int64_t(1) << 31);
}

template <int IN, int NP>
static rh_status launch_sketch_tc_conv(const CUtensorMap& m0, const ModeView& v, int ell, uint64_t seed, uint32_t sid,
                                       float* part, double* norm_part, int32_t* err, cudaStream_t st, int64_t row0,
                                       int64_t L) {
  const int ctas = sketch_tc_ctas(v);
  const int64_t nchunks = ceil_div(v.M(), kPChunk);
  const int64_t cpc = ceil_div(nchunks, ctas);
  const int mtiles = (int)ceil_div(v.I, kRowsTile);
  const size_t smem = sizeof(SketchSmem<IN, NP>) + 1024;
  RH_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<IN, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sketch_tc_kernel<IN, NP><<<ctas, SketchCfg<IN>::kThreads, smem, st>>>(
      m0, m0, NP, v.I, v.M(), ell, mtiles, cpc, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), sid, part,
      norm_part, err, nullptr, 0, tc_probe_next(), row0, L);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_sketch_tc_f32s(const ModeView& v, int ell, const float* X, uint64_t seed, uint32_t sid, float* part,
                                double* norm_part, int32_t* err, cudaStream_t st, int64_t row0, int pieces) {
  if (!sketch_tc_strided_supported(v, ell)) {
    set_error("tensor-core sketch: unsupported strided shape (needs L % 64 == 0, I <= 1024, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  CUtensorMap m0;
  rh_status s = make_map_3d_f32(&m0, X, v.L, v.I, v.R, 64, kRowsTile);
  if (s != RH_OK) return s;
  return pieces == 3 ? launch_sketch_tc_conv<tc::kInF32S, 3>(m0, v, ell, seed, sid, part, norm_part, err, st, row0, v.L)
                     : launch_sketch_tc_conv<tc::kInF32S, 2>(m0, v, ell, seed, sid, part, norm_part, err, st, row0, v.L);
}

bool sketch_tc_supported(const ModeView& v, int ell) {
  return v.L == 1 && v.I % 8 == 0 && v.I <= (int64_t)kRowsTile * kMaxTiles && ell >= 1 && ell <= 64 &&
         v.M() < (int64_t(1) << 31);
}

int sketch_tc_ctas(const ModeView& v) {
  const int64_t nchunks = ceil_div(v.M(), kPChunk);
  return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), nchunks));
}

rh_status launch_sketch_tc(const ModeView& v, int ell, const uint16_t* piece0, const uint16_t* piece1, uint64_t seed,
                           uint32_t sid, float* part, int32_t* err, cudaStream_t st, int64_t row0) {
  if (!sketch_tc_supported(v, ell)) {
    set_error("tensor-core sketch: unsupported shape (needs the first mode, I % 8 == 0, I <= 1024, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  CUtensorMap m0, m1;
  rh_status s = make_bf16_map_2d(&m0, piece0, v.I, v.M(), 64);
  if (s != RH_OK) return s;
  const int np = piece1 ? 2 : 1;
  if (piece1) {
    if ((s = make_bf16_map_2d(&m1, piece1, v.I, v.M(), 64)) != RH_OK) return s;
  } else {
    m1 = m0;
  }
  const int ctas = sketch_tc_ctas(v);
  const int64_t nchunks = ceil_div(v.M(), kPChunk);
  const int64_t cpc = ceil_div(nchunks, ctas);
  const int mtiles = (int)ceil_div(v.I, kRowsTile);
  constexpr int IN = tc::kInPieces;
  const size_t smem = sizeof(SketchSmem<IN>) + 1024;
  RH_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sketch_tc_kernel<IN><<<ctas, SketchCfg<IN>::kThreads, smem, st>>>(
      m0, m1, np, v.I, v.M(), ell, mtiles, cpc, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), sid, part,
      nullptr, err, nullptr, 0, tc_probe_next(), row0, 1);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_sketch_tc_f32(const ModeView& v, int ell, const float* X, uint64_t seed, uint32_t sid, float* part,
                               double* norm_part, int32_t* err, cudaStream_t st, int64_t row0, int pieces) {
  if (!sketch_tc_supported(v, ell)) {
    set_error("tensor-core sketch: unsupported shape (needs the first mode, I % 8 == 0, I <= 1024, ell <= 64)");
    return RH_EUNSUPPORTED;
  }
  CUtensorMap m0;
  rh_status s = make_map_2d_plain(&m0, X, 4, v.I, v.M(), kRowsTile, 64);
  if (s != RH_OK) return s;
  return pieces == 3 ? launch_sketch_tc_conv<tc::kInF32, 3>(m0, v, ell, seed, sid, part, norm_part, err, st, row0, 1)
                     : launch_sketch_tc_conv<tc::kInF32, 2>(m0, v, ell, seed, sid, part, norm_part, err, st, row0, 1);
}

rh_status launch_sketch_tc_fp8(const ModeView& v, int ell, const uint8_t* X, const float* scales, int64_t ld,
                               uint64_t seed, uint32_t sid, float* part, double* norm_part, int32_t* err,
                               cudaStream_t st, int64_t row0) {
  if (!sketch_tc_supported(v, ell) || ld < v.I || ld % 16 != 0) {
    set_error("tensor-core sketch: unsupported E4M3 shape (needs the first mode, I % 8 == 0, I <= 1024, "
              "ell <= 64, a leading dimension that is a multiple of 16)");
    return RH_EUNSUPPORTED;
  }
  CUtensorMap m0;
  rh_status s = make_u8_map_2d(&m0, X, v.I, ld, v.M(), 128, 64);
  if (s != RH_OK) return s;
  const int ctas = sketch_tc_ctas(v);
  const int64_t nchunks = ceil_div(v.M(), kPChunk);
  const int64_t cpc = ceil_div(nchunks, ctas);
  const int mtiles = (int)ceil_div(v.I, kRowsTile);
  constexpr int IN = tc::kInFp8;
  const size_t smem = sizeof(SketchSmem<IN>) + 1024;
  RH_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sketch_tc_kernel<IN><<<ctas, SketchCfg<IN>::kThreads, smem, st>>>(
      m0, m0, 1, v.I, v.M(), ell, mtiles, cpc, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), sid, part,
      norm_part, err, scales, ld, tc_probe_next(), row0, 1);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_pieces_sumsq(const uint16_t* piece0, const uint16_t* piece1, int64_t n, double* part, double* out,
                              cudaStream_t st) {
  pieces_sumsq_kernel<<<1024, 256, 0, st>>>(piece0, piece1, n, part);
  RH_LAUNCH_CHECK();
  sum_n_kernel<<<1, 32, 0, st>>>(part, 1024, out, 0);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_sum_n(const double* part, int n, double* out, cudaStream_t st, int accumulate) {
  sum_n_kernel<<<1, 32, 0, st>>>(part, n, out, accumulate);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

rh_status launch_split_bf16x2(const float* x, int64_t n, uint16_t* hi, uint16_t* lo, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * num_sms()));
  split_bf16x2_kernel<<<blocks, 256, 0, st>>>(x, n, hi, lo);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

}  // namespace rh
