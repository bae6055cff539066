// Tensor-core (tcgen05) sketch and mode product of a first mode with few rows: Alg. 1 steps 1 and 3
// on X_(1) for I <= 128 and ell <= 32 with the unfolding's columns contiguous (L = 1), for a tensor
// held as BF16 values, as the two BF16 pieces of the two-piece form, as FP32 values split on the fly
// into the same exact BF16 head and tail, or as E4M3 bytes with block scales (dequantized and
// rounded to one BF16 piece).
//
// Both are grouped operations (a body over block coordinates), so a batch of small tensors runs
// each stage as one launch.  A TMA tile of X_(1) would need its rows (I values) to be a multiple of
// 16 bytes; here every thread reads consecutive elements of the contiguous column run of its tile
// with plain loads instead (any I), eight consecutive rows of one column at a time, converts them
// into the BF16 operand layout in shared memory (one 16-byte unit per piece), and one thread issues
// the MMAs.  The next tile's loads are in registers while the current
// tile is multiplied.
//
//   sketch   part[by](i, c) = sum over the CTA's columns p of X(i, p) Omega(p, c):
//            D (128 rows i x N = 16 or 32 columns c, FP32 in TMEM) += A (X pieces, rows i, K = 64
//            columns p, MN-major) B (Omega rounded to BF16, ties to even; K-major), so every product
//            is exact and the sums are FP32 in TMEM over the CTA's columns, FP64 across CTAs
//            (launch_sketch_reduce).  Also the partial sum of the squares of the values read.
//   product  B(c, p) = sum_i Q(i, c) X(i, p):  D (128 rows p x 2 ellp columns) = A (X pieces,
//            rows p, K = i, K-major) B ([Q_h | Q_t], rows c, K-major) with Q_h = bf16(fl32(Q)),
//            Q_t = bf16(fl32(Q) - Q_h), and B(c, p) = D(p, c) + D(p, ellp + c).
//
// Every wait on the MMA completion barrier is bounded (tc::mbar_wait); a wait that gives up sets
// *err, the CTA skips its remaining tiles and its outputs, and frees its tensor memory.
#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"
#include "tc.cuh"

namespace rh {
namespace {

// Input kinds: FP32 values split into head + tail, BF16 values (one piece), the two BF16 pieces of
// the two-piece form (head array followed by the tail array, n values each), or E4M3 bytes with
// block scales (mode-1 fibres at stride ld, one FP32 scale per 128 bytes), dequantized in FP32 and
// rounded to one BF16 piece.
constexpr int kSmF32 = 0, kSmBf16 = 1, kSmPieces = 2, kSmFp8 = 3;

struct SmallSrc {
  const void* X;
  int64_t n;              // I M: the offset of the tail piece
  int64_t ld;             // E4M3: stride of the columns in bytes
  const float* scales;    // E4M3: the block scales
};

// Eight consecutive rows i0 .. i0 + 7 of column p of X_(1) as raw 32-bit registers: the FP32 bits,
// the BF16 bits, head | tail << 16 (two pieces), or the FP32 bits of the dequantized E4M3 value;
// rows >= I and a column outside the tensor (valid = false) read as zero.
template <int IN>
__device__ __forceinline__ void chunk_load(uint32_t (&r)[8], const SmallSrc& src, int64_t I, int64_t p, int i0,
                                           bool valid) {
  const int lim = valid ? (int)min((int64_t)8, I - i0) : 0;
  if constexpr (IN == kSmFp8) {
    const uint8_t* x8 = static_cast<const uint8_t*>(src.X);
    const int64_t b0 = src.ld * p + i0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      r[j] = j < lim ? __float_as_uint(__fmul_rn(tc::e4m3_to_f32(__ldg(x8 + b0 + j)), __ldg(src.scales + ((b0 + j) >> 7))))
                     : 0u;
  } else {
    const int64_t e0 = I * p + i0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t v = 0u;
      if (j < lim) {
        if constexpr (IN == kSmF32) {
          v = __float_as_uint(__ldg(static_cast<const float*>(src.X) + e0 + j));
        } else if constexpr (IN == kSmBf16) {
          v = (uint32_t)__ldg(static_cast<const unsigned short*>(src.X) + e0 + j);
        } else {
          const unsigned short* q = static_cast<const unsigned short*>(src.X);
          v = (uint32_t)__ldg(q + e0 + j) | ((uint32_t)__ldg(q + src.n + e0 + j) << 16);
        }
      }
      r[j] = v;
    }
  }
}

// A chunk's eight values written as one 16-byte unit per piece at byte offset off: FP32 split into
// head bf16(x) and tail bf16(x - head) (ties to even, packed conversions; head + tail holds the 16
// leading significant bits of x), E4M3 values rounded to one piece, BF16 values and given pieces as
// they are.  Returns the sum of the squares of the values represented.
template <int IN>
__device__ __forceinline__ float chunk_put(uint8_t* p0, uint8_t* p1, uint32_t off, const uint32_t (&r)[8]) {
  uint32_t h[4], t[4];
  float ss = 0.0f;
  if constexpr (IN == kSmF32 || IN == kSmFp8) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x0 = __uint_as_float(r[2 * q]), x1 = __uint_as_float(r[2 * q + 1]);
      h[q] = tc::pack_bf16x2(x0, x1);
      const float h0 = __uint_as_float(h[q] << 16), h1 = __uint_as_float(h[q] & 0xFFFF0000u);
      if constexpr (IN == kSmF32) {
        t[q] = tc::pack_bf16x2(x0 - h0, x1 - h1);
        const float g0 = h0 + __uint_as_float(t[q] << 16), g1 = h1 + __uint_as_float(t[q] & 0xFFFF0000u);
        ss = fmaf(g0, g0, ss);
        ss = fmaf(g1, g1, ss);
      } else {
        ss = fmaf(h0, h0, ss);
        ss = fmaf(h1, h1, ss);
      }
    }
  } else if constexpr (IN == kSmBf16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = r[2 * q] | (r[2 * q + 1] << 16);
      const float h0 = __uint_as_float(h[q] << 16), h1 = __uint_as_float(h[q] & 0xFFFF0000u);
      ss = fmaf(h0, h0, ss);
      ss = fmaf(h1, h1, ss);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h[q] = (r[2 * q] & 0xFFFFu) | (r[2 * q + 1] << 16);
      t[q] = (r[2 * q] >> 16) | (r[2 * q + 1] & 0xFFFF0000u);
      const float g0 = __uint_as_float(h[q] << 16) + __uint_as_float(t[q] << 16);
      const float g1 = __uint_as_float(h[q] & 0xFFFF0000u) + __uint_as_float(t[q] & 0xFFFF0000u);
      ss = fmaf(g0, g0, ss);
      ss = fmaf(g1, g1, ss);
    }
  }
  *reinterpret_cast<uint4*>(p0 + off) = make_uint4(h[0], h[1], h[2], h[3]);
  if constexpr (IN == kSmF32 || IN == kSmPieces) *reinterpret_cast<uint4*>(p1 + off) = make_uint4(t[0], t[1], t[2], t[3]);
  else (void)p1;
  return ss;
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return p + ((1024u - (tc::smem_u32(p) & 1023u)) & 1023u);
}

// ------------------------------------------------------------------------------------------------
struct SmallTcSketchArgs {
  SmallSrc src;
  int64_t I, M;
  int ell, ellp;          // ellp = N of the MMA: 16 or 32
  int64_t chunk;          // columns per CTA (a multiple of 64)
  uint32_t k0, k1, sid;
  int64_t row0;           // Omega row of column 0
  float* part;            // [S][ell][I]
  double* part_norm;      // [S] (NULL: no norm)
  int32_t* err;
  int32_t nch, dnc, rnc;  // chunks of eight rows per column; 256 = dnc nch + rnc
  FastDiv fN;
  int32_t probe;          // wait-timeout probe (test support): wait on a barrier nothing arrives at
};

template <int IN, int TI>
struct SmallTcSketchOp {
  using Args = SmallTcSketchArgs;
  static constexpr int kThreads = 256, kMinBlocks = TI == 128 ? 2 : 3;
  static constexpr int NP = (IN == kSmBf16 || IN == kSmFp8) ? 1 : 2;
  static constexpr int KT = 64;                         // columns per tile
  static constexpr int ITEMS = KT * (TI / 8) / 256;     // eight-row chunks per thread per tile (bound)
  static constexpr uint32_t kPiece = 128 * KT * 2;      // 128 rows x 64 columns BF16
  static constexpr uint32_t kOm = 32 * KT * 2;          // up to 32 Omega columns x 64 rows BF16
  static constexpr size_t kDynSmem = 1024 + NP * kPiece + 2 * kOm + 64;
  __device__ static void body(const Grid g, const Args& a);
};

template <int IN, int TI>
__device__ __forceinline__ void SmallTcSketchOp<IN, TI>::body(const Grid g, const Args& a) {
  using Op = SmallTcSketchOp<IN, TI>;
  constexpr int KT = Op::KT, ITEMS = Op::ITEMS, NP = Op::NP;
  constexpr uint32_t kPiece = Op::kPiece, kOm = Op::kOm;
  extern __shared__ uint8_t dsm_raw[];
  uint8_t* base = align1024(dsm_raw);
  uint8_t* xs0 = base;
  uint8_t* xs1 = base + (NP - 1) * kPiece;
  uint8_t* oms = base + NP * kPiece;                    // two Omega buffers
  uint64_t* bar = reinterpret_cast<uint64_t*>(oms + 2 * kOm);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ int s_abort;
  __shared__ double s_nrm[8];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t I = a.I, M = a.M;
  const int Ii = (int)I;
  const int ell = a.ell, ellp = a.ellp;
  const int nq = (ell + 3) / 4;
  const int64_t pb = (int64_t)g.by * a.chunk;
  const int64_t pe = min(M, pb + a.chunk);

  // rows i >= I of the X pieces and Omega columns >= 4 nq stay zero for the whole launch
  for (int e = tid; e < (int)((NP * kPiece + 2 * kOm) / 16); e += 256)
    reinterpret_cast<uint4*>(base)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (a.probe) {   // wait-timeout probe: nothing allocated or issued yet
    if (tid == 0) tc::mbar_wait(bar, 0, a.err, tc::kProbeCode, tc::kProbeSpin);
    return;
  }
  if (warp == 0) {
    tc::tmem_alloc(slot, 32);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *slot;

  // items of a tile: chunks of eight rows (ch) of one column (k); item u = tid + 256 j is
  // (k, ch) = (u / nch, u % nch), later ones step by 256 = dnc nch + rnc
  const int nch = a.nch;
  const int k_first = (int)a.fN.div((uint32_t)tid);
  const int c_first = tid - k_first * nch;
  uint32_t xr[ITEMS][8];
  auto load = [&](int64_t p0) {
    const int64_t nv = min(pe, p0 + KT) - p0;
    int k = k_first, ch = c_first;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (k < KT) chunk_load<IN>(xr[j], a.src, I, p0 + k, 8 * ch, k < nv);
      ch += a.rnc;
      k += a.dnc;
      if (ch >= nch) {
        ch -= nch;
        ++k;
      }
    }
  };
  // chunk (ch, k) of the MN-major 128-byte-swizzled pieces (two 64-row halves of 64 x 128 B) is the
  // 16-byte unit at (ch / 8) 8192 + 128 k + ((ch % 8) ^ (k % 8)) 16
  auto store = [&]() {
    float ss = 0.f;
    int k = k_first, ch = c_first;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (k < KT) {
        const uint32_t off = (uint32_t)((ch >> 3) * 8192 + k * 128 + (((ch & 7) ^ (k & 7)) << 4));
        ss += chunk_put<IN>(xs0, xs1, off, xr[j]);
      }
      ch += a.rnc;
      k += a.dnc;
      if (ch >= nch) {
        ch -= nch;
        ++k;
      }
    }
    return ss;
  };
  // Omega rows p0 .. p0 + 63 (quads q < nq of columns) into K-major buffer b: (c, k) at
  // (c / 8) 1024 + (c % 8) 128 + ((k / 8) ^ (c % 8)) 16 + 2 (k % 8)
  auto omega = [&](int64_t p0, int b) {
    uint8_t* om = oms + b * kOm;
    for (int t = tid; t < KT * nq; t += 256) {
      const int k = t & (KT - 1), q = t / KT;
      const float4 v = rng::omega4(a.k0, a.k1, a.sid, p0 + k + a.row0, (uint32_t)q);
      const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * q + u;
        const uint32_t off = (uint32_t)((c >> 3) * 1024 + (c & 7) * 128 + ((((k >> 3) ^ (c & 7))) << 4) + ((k & 7) << 1));
        *reinterpret_cast<uint16_t*>(om + off) = tc::bf16_rne(vv[u]);
      }
    }
  };

  const uint32_t idesc = tc::idesc_bf16(128, ellp, 1, 0);
  double nrm = 0.0;   // FP32 sums of a thread's at most PER squares of a tile, FP64 across tiles
  int tl = 0;
  bool ok = true;
  if (pb < pe) {
    load(pb);
    omega(pb, 0);
  }
  for (int64_t p0 = pb; p0 < pe; p0 += KT, ++tl) {
    nrm += (double)store();
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t xa0 = tc::smem_u32(xs0), xa1 = tc::smem_u32(xs1);
      const uint32_t oa = tc::smem_u32(oms + (tl & 1) * kOm);
#pragma unroll
      for (int kk = 0; kk < KT / 16; ++kk) {
        const uint64_t bdesc = tc::sdesc_sw128(oa + kk * 32, 16, 1024);
        tc::mma_bf16(tmem, tc::sdesc_sw128(xa0 + kk * 2048, 8192, 1024), bdesc, idesc, (tl > 0 || kk > 0) ? 1u : 0u);
        if (NP == 2) tc::mma_bf16(tmem, tc::sdesc_sw128(xa1 + kk * 2048, 8192, 1024), bdesc, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    if (p0 + KT < pe) {
      load(p0 + KT);               // in flight during the MMAs
      omega(p0 + KT, (tl + 1) & 1);
    }
    if (tid == 0 && !tc::mbar_wait(bar, (uint32_t)(tl & 1), a.err, 21)) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      ok = false;
      break;
    }
  }
  tc::tc_fence_after();
  if (ok) {
    // rows i = 32 warp + lane of D (warps 0..3), columns c < ell
    if (warp < 4) {
      const int i = 32 * warp + lane;
      for (int cc = 0; cc < ellp / 16; ++cc) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cc * 16), v);
        if (i < Ii) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = cc * 16 + j;
            if (c < ell) a.part[((int64_t)g.by * ell + c) * I + i] = tl > 0 ? v[j] : 0.f;
          }
        }
      }
    }
    if (a.part_norm != nullptr) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
      if (lane == 0) s_nrm[warp] = nrm;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (ok && a.part_norm != nullptr && tid == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += s_nrm[k];
    a.part_norm[g.by] = t;
  }
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// ------------------------------------------------------------------------------------------------
struct SmallTcTtmArgs {
  SmallSrc src;
  int64_t I, M;
  const double* Q;        // I x ell, column-major
  int ell, ellp;          // ellp: 8, 16 or 32 (the MMA's N is 2 ellp)
  float* B;               // B[c + ell p]
  int64_t tiles_per_cta;  // 128-column tiles
  int32_t* err;
  int32_t nch, dnc, rnc;  // chunks of eight rows per column; the block size = dnc nch + rnc
  FastDiv fN;
  int32_t probe;
};

template <int IN, int TI>
struct SmallTcTtmOp {
  using Args = SmallTcTtmArgs;
  // 128-row tiles hold 16384 values: 512 threads (32 registers of loads each), one CTA per SM
  static constexpr int kThreads = TI == 128 ? 512 : 256, kMinBlocks = TI == 128 ? 1 : 2;
  static constexpr int NP = (IN == kSmBf16 || IN == kSmFp8) ? 1 : 2;
  static constexpr int KB = TI > 64 ? 2 : 1;            // 64-wide blocks of K = i
  static constexpr int PT = 128;                        // columns p per tile (the MMA's M)
  static constexpr int ITEMS = PT * (TI / 8) / kThreads;   // eight-row chunks per thread per tile (bound)
  static constexpr uint32_t kPiece = KB * 128 * 128;    // KB blocks of 128 rows x 128 B
  static constexpr uint32_t kQ = KB * 64 * 128;         // [Q_h | Q_t]: up to 64 rows x KB blocks
  static constexpr uint32_t kStage = PT * 32 * 4;       // the tile's output, FP32
  static constexpr size_t kDynSmem = 1024 + NP * kPiece + kQ + kStage + 64;
  __device__ static void body(const Grid g, const Args& a);
};

template <int IN, int TI>
__device__ __forceinline__ void SmallTcTtmOp<IN, TI>::body(const Grid g, const Args& a) {
  using Op = SmallTcTtmOp<IN, TI>;
  constexpr int PT = Op::PT, ITEMS = Op::ITEMS, NP = Op::NP, KB = Op::KB, NT = Op::kThreads;
  constexpr uint32_t kPiece = Op::kPiece, kQ = Op::kQ;
  extern __shared__ uint8_t dsm_raw[];
  uint8_t* base = align1024(dsm_raw);
  uint8_t* xs0 = base;
  uint8_t* xs1 = base + (NP - 1) * kPiece;
  uint8_t* qs = base + NP * kPiece;
  float* stage = reinterpret_cast<float*>(qs + kQ);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + PT * 32);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t I = a.I, M = a.M;
  const int Ii = (int)I;
  const int ell = a.ell, ellp = a.ellp, n2 = 2 * ellp;
  const int64_t ntiles = (M + PT - 1) / PT;
  const int64_t t0 = (int64_t)g.bx * a.tiles_per_cta;
  const int64_t t1 = min(ntiles, t0 + a.tiles_per_cta);
  if (t0 >= t1) return;

  for (int e = tid; e < (int)((NP * kPiece + kQ) / 16); e += NT)
    reinterpret_cast<uint4*>(base)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // [Q_h | Q_t] as rows c (head) and ellp + c (tail), K = i: (row, i) at
  // (i / 64) n2 128 + (row / 8) 1024 + (row % 8) 128 + ((i % 64 / 8) ^ (row % 8)) 16 + 2 (i % 8)
  for (int e = tid; e < Ii * ell; e += NT) {
    const int c = e / Ii, i = e - c * Ii;
    const float q = (float)__ldg(a.Q + (int64_t)c * I + i);
    const uint16_t h = tc::bf16_rne(q);
    const uint16_t t = tc::bf16_rne(q - tc::bf16_to_f(h));
    const int il = i & 63;
    const int rh = c, rt = ellp + c;
    const uint32_t kb = (uint32_t)((i >> 6) * n2 * 128);
    *reinterpret_cast<uint16_t*>(qs + kb + (rh >> 3) * 1024 + (rh & 7) * 128 + ((((il >> 3) ^ (rh & 7))) << 4) +
                                 ((il & 7) << 1)) = h;
    *reinterpret_cast<uint16_t*>(qs + kb + (rt >> 3) * 1024 + (rt & 7) * 128 + ((((il >> 3) ^ (rt & 7))) << 4) +
                                 ((il & 7) << 1)) = t;
  }
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  if (a.probe) {
    if (tid == 0) tc::mbar_wait(bar, 0, a.err, tc::kProbeCode, tc::kProbeSpin);
    return;
  }
  if (warp == 0) {
    tc::tmem_alloc(slot, 128);   // two accumulators of up to 64 columns
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *slot;

  // items of a tile: chunks of eight rows (ch) of one column (p); item u = tid + NT j is
  // (p, ch) = (u / nch, u % nch), later ones step by NT = dnc nch + rnc
  const int nch = a.nch;
  const int k_first = (int)a.fN.div((uint32_t)tid);
  const int c_first = tid - k_first * nch;
  uint32_t xr[ITEMS][8];
  auto load = [&](int64_t tile) {
    const int64_t p0 = tile * PT;
    const int64_t nv = min(M, p0 + PT) - p0;
    int p = k_first, ch = c_first;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (p < PT) chunk_load<IN>(xr[j], a.src, I, p0 + p, 8 * ch, p < nv);
      ch += a.rnc;
      p += a.dnc;
      if (ch >= nch) {
        ch -= nch;
        ++p;
      }
    }
  };
  // chunk (p, ch) of the K-major pieces is the 16-byte unit at (ch / 8) 16384 + (p / 8) 1024 +
  // (p % 8) 128 + ((ch % 8) ^ (p % 8)) 16
  auto store = [&]() {
    int p = k_first, ch = c_first;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (p < PT) {
        const uint32_t off =
            (uint32_t)((ch >> 3) * 16384 + (p >> 3) * 1024 + (p & 7) * 128 + (((ch & 7) ^ (p & 7)) << 4));
        (void)chunk_put<IN>(xs0, xs1, off, xr[j]);
      }
      ch += a.rnc;
      p += a.dnc;
      if (ch >= nch) {
        ch -= nch;
        ++p;
      }
    }
  };
  // D(p, c) + D(p, ellp + c) of accumulator b -> stage[p ell + c] -> B[ell p0 + e] (coalesced)
  auto epilogue = [&](int64_t tile, int b) {
    if (warp < 4) {
      const int p = 32 * warp + lane;
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * 64);
      if (ellp == 8) {
        float v[16];
        tc::tmem_ld16(ta, v);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < ell) stage[p * ell + c] = v[c] + v[8 + c];
      } else {
        for (int cc = 0; cc < ellp / 16; ++cc) {
          float h[16], t[16];
          tc::tmem_ld16(ta + (uint32_t)(cc * 16), h);
          tc::tmem_ld16(ta + (uint32_t)(ellp + cc * 16), t);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = cc * 16 + j;
            if (c < ell) stage[p * ell + c] = h[j] + t[j];
          }
        }
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    const int64_t p0 = tile * PT;
    const int n = (int)(min(M, p0 + PT) - p0) * ell;
    float* dst = a.B + (int64_t)ell * p0;
    for (int e = tid; e < n; e += NT) dst[e] = stage[e];
    __syncthreads();   // stage is free again
  };

  const uint32_t idesc = tc::idesc_bf16(128, n2, 0, 0);
  const int nks = (Ii + 15) / 16;   // 16-wide K steps that hold rows i < I
  load(t0);
  int tl = 0;
  bool ok = true;
  for (int64_t tile = t0; tile < t1; ++tile, ++tl) {
    store();
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const uint32_t d = tmem + (uint32_t)((tl & 1) * 64);
      const uint32_t xa0 = tc::smem_u32(xs0), xa1 = tc::smem_u32(xs1), qa = tc::smem_u32(qs);
      for (int ks = 0; ks < nks; ++ks) {
        const int kb = ks >> 2, kk = ks & 3;
        const uint64_t bdesc = tc::sdesc_sw128(qa + kb * n2 * 128 + kk * 32, 16, 1024);
        tc::mma_bf16(d, tc::sdesc_sw128(xa0 + kb * 16384 + kk * 32, 16, 1024), bdesc, idesc, ks > 0 ? 1u : 0u);
        if (NP == 2) tc::mma_bf16(d, tc::sdesc_sw128(xa1 + kb * 16384 + kk * 32, 16, 1024), bdesc, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    if (tile + 1 < t1) load(tile + 1);   // in flight during the MMAs and the previous epilogue
    if (tl > 0) epilogue(tile - 1, (tl - 1) & 1);
    if (tid == 0 && !tc::mbar_wait(bar, (uint32_t)(tl & 1), a.err, 22)) s_abort = 1;
    __syncthreads();
    tc::tc_fence_after();
    if (s_abort) {
      ok = false;
      break;
    }
  }
  if (ok) epilogue(t1 - 1, (tl - 1) & 1);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
  (void)KB;
}

template <int IN, int TI>
rh_status emit_small_tc_sketch(const SketchPlan& pl, const SmallTcSketchArgs& a, cudaStream_t st, int site) {
  using Op = SmallTcSketchOp<IN, TI>;
  return emit<Op>(site, 0, dim3(1, pl.S), Op::kDynSmem, st, a);
}

template <int IN, int TI>
rh_status emit_small_tc_ttm(int64_t ctas, const SmallTcTtmArgs& a, cudaStream_t st, int site) {
  using Op = SmallTcTtmOp<IN, TI>;
  return emit<Op>(site, 0, dim3((unsigned)ctas), Op::kDynSmem, st, a);
}

}  // namespace

bool small_tc_supported(const ModeView& v, int ell) {
  return v.L == 1 && v.I >= 1 && v.I <= 128 && ell >= 1 && ell <= 32 && v.M() >= 1 &&
         v.M() < (int64_t(1) << 31) && v.I * v.M() < (int64_t(1) << 40);
}

SketchPlan plan_sketch_small_tc(const ModeView& v, int ell) {
  SketchPlan pl;
  pl.v = v;
  pl.ell = ell;
  pl.ellp = ell <= 16 ? 16 : 32;
  pl.gx = 1;
  pl.ti = v.I <= 32 ? 32 : (v.I <= 64 ? 64 : 128);
  const int64_t tiles = ceil_div(v.M(), 64);
  // at least tune(min_tiles) tiles per CTA, tune(ctas_per_sm) CTAs per SM at most (tuning_table.inc)
  const int64_t S = std::max<int64_t>(1, std::min<int64_t>((int64_t)tune(TUNE_SMALL_TC_SKETCH_CTAS_PER_SM) * num_sms(),
                                                           ceil_div(tiles, tune(TUNE_SMALL_TC_SKETCH_MIN_TILES))));
  pl.chunk = ceil_div(tiles, S) * 64;
  pl.S = (int)ceil_div(v.M(), pl.chunk);
  return pl;
}

rh_status launch_sketch_small_tc(const SketchPlan& pl, const SmallInput& in, uint64_t seed, uint32_t sid, float* part,
                                 double* part_norm, int32_t* err, cudaStream_t st, int site) {
  if (!small_tc_supported(pl.v, pl.ell) || pl.chunk % 64 != 0 || pl.ti < pl.v.I) {
    set_error("internal: small-row tensor-core sketch outside its shapes");
    return RH_EUNSUPPORTED;
  }
  const int nch = (int)((pl.v.I + 7) / 8);
  const int32_t form = in.form;
  SmallTcSketchArgs a{SmallSrc{in.X, pl.v.I * pl.v.M(), in.ld, in.scales}, pl.v.I, pl.v.M(), pl.ell, pl.ellp, pl.chunk, (uint32_t)(seed & 0xFFFFFFFFu),
                      (uint32_t)(seed >> 32), sid, pl.row0, part, part_norm, err, nch, 256 / nch, 256 % nch,
                      FastDiv((uint32_t)nch), tc_probe_next()};
  if (form == RH_BF16) {
    if (pl.ti == 32) return emit_small_tc_sketch<kSmBf16, 32>(pl, a, st, site);
    if (pl.ti == 64) return emit_small_tc_sketch<kSmBf16, 64>(pl, a, st, site);
    return emit_small_tc_sketch<kSmBf16, 128>(pl, a, st, site);
  }
  if (form == RH_FP8_E4M3) {
    if (pl.ti == 32) return emit_small_tc_sketch<kSmFp8, 32>(pl, a, st, site);
    if (pl.ti == 64) return emit_small_tc_sketch<kSmFp8, 64>(pl, a, st, site);
    return emit_small_tc_sketch<kSmFp8, 128>(pl, a, st, site);
  }
  if (form == RH_BF16X2) {
    if (pl.ti == 32) return emit_small_tc_sketch<kSmPieces, 32>(pl, a, st, site);
    if (pl.ti == 64) return emit_small_tc_sketch<kSmPieces, 64>(pl, a, st, site);
    return emit_small_tc_sketch<kSmPieces, 128>(pl, a, st, site);
  }
  if (pl.ti == 32) return emit_small_tc_sketch<kSmF32, 32>(pl, a, st, site);
  if (pl.ti == 64) return emit_small_tc_sketch<kSmF32, 64>(pl, a, st, site);
  return emit_small_tc_sketch<kSmF32, 128>(pl, a, st, site);
}

rh_status launch_ttm_small_tc(const ModeView& v, const SmallInput& in, const double* Q, int ell, float* B, int32_t* err,
                              cudaStream_t st, int site) {
  if (!small_tc_supported(v, ell)) {
    set_error("internal: small-row tensor-core mode product outside its shapes");
    return RH_EUNSUPPORTED;
  }
  const int nch = (int)((v.I + 7) / 8);
  const int ti = v.I <= 32 ? 32 : (v.I <= 64 ? 64 : 128);
  const int64_t ntiles = ceil_div(v.M(), 128);
  // at least tune(min_tiles) tiles per CTA (two keep the pipeline busy), at most the resident CTAs
  const int64_t ctas = std::max<int64_t>(
      1, std::min<int64_t>((ti == 128 ? 1LL : 2LL) * num_sms(), ceil_div(ntiles, tune(TUNE_SMALL_TC_TTM_MIN_TILES))));
  const int64_t tpc = ceil_div(ntiles, ctas);
  const int nt = ti == 128 ? 512 : 256;
  const int32_t form = in.form;
  const SmallTcTtmArgs a{SmallSrc{in.X, v.I * v.M(), in.ld, in.scales}, v.I, v.M(), Q, ell, ell <= 8 ? 8 : (ell <= 16 ? 16 : 32), B, tpc, err, nch, nt / nch, nt % nch,
                         FastDiv((uint32_t)nch), tc_probe_next()};
  const int64_t g = ceil_div(ntiles, tpc);
  if (form == RH_BF16) {
    if (ti == 32) return emit_small_tc_ttm<kSmBf16, 32>(g, a, st, site);
    if (ti == 64) return emit_small_tc_ttm<kSmBf16, 64>(g, a, st, site);
    return emit_small_tc_ttm<kSmBf16, 128>(g, a, st, site);
  }
  if (form == RH_FP8_E4M3) {
    if (ti == 32) return emit_small_tc_ttm<kSmFp8, 32>(g, a, st, site);
    if (ti == 64) return emit_small_tc_ttm<kSmFp8, 64>(g, a, st, site);
    return emit_small_tc_ttm<kSmFp8, 128>(g, a, st, site);
  }
  if (form == RH_BF16X2) {
    if (ti == 32) return emit_small_tc_ttm<kSmPieces, 32>(g, a, st, site);
    if (ti == 64) return emit_small_tc_ttm<kSmPieces, 64>(g, a, st, site);
    return emit_small_tc_ttm<kSmPieces, 128>(g, a, st, site);
  }
  if (ti == 32) return emit_small_tc_ttm<kSmF32, 32>(g, a, st, site);
  if (ti == 64) return emit_small_tc_ttm<kSmF32, 64>(g, a, st, site);
  return emit_small_tc_ttm<kSmF32, 128>(g, a, st, site);
}

}  // namespace rh
