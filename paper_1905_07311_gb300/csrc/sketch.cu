// Range-finder sketch Y_n = G_(n) Omega_n with Omega generated on the fly
// (Alg. 1 step 1; Sec. 3.1: Omega need not be stored).
//
// G is read through its 3-D mode view (L, I, R): element (i, p) of the unfolding,
// p = l + L r its Kolda column index, sits at (p % L) + L I (p / L) + L i.  Nothing is
// materialised: the unfolding is an index map.
//
// Parallelisation: CTA (bx, s) owns rows i in [128 bx, 128 bx + 128) and the column
// range p in [s chunk, (s+1) chunk) of X_(n) (split-K over the long dimension).  Per
// k-step of 32 columns it generates the 32 x ellp Omega tile into shared memory,
// stages the 32 x 128 tile of G, and accumulates a 128 x ellp register tile.  Each
// element of G is read exactly once over the whole grid, so the same pass also
// accumulates ||G||_F^2.  Partial sketches land in a workspace and are summed in FP64
// in a fixed order (deterministic).
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"
#include "tc.cuh"

namespace rh {

namespace {

constexpr int kTI = 128;   // rows of Y per CTA
constexpr int kKP = 32;    // columns of X_(n) per k-step
constexpr int kNT = 256;   // threads per CTA
constexpr int kFlush = 16; // FP32: k-steps per inner accumulator before folding into the outer one

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
};

// Swizzled column of the (k, col) element of a [32][128] staging tile: groups of one
// 16-byte vector are XOR-permuted by the row so that both the column-wise stores and
// the row-wise vector loads are free of bank conflicts.
template <typename T>
__device__ __forceinline__ int swz(int k, int col) {
  return col ^ ((k & 7) * Vec<T>::n);
}

// head + tail of the exact two-piece BF16 split of an FP32 value (ties to even), as the tensor-core
// kernels form it: h = bf16(x), t = bf16(x - h), value h + t (exact in FP32)
__device__ __forceinline__ float split_value(float x) {
  const float h = tc::bf16_to_f(tc::bf16_rne(x));
  return h + tc::bf16_to_f(tc::bf16_rne(x - h));
}
__device__ __forceinline__ double split_value(double x) { return x; }

template <typename T>
struct SketchArgs {
  const T* G;
  int64_t L, I, R;
  int ell;
  int64_t chunk;
  uint32_t k0, k1, sid;
  T* part;
  double* part_norm;   // may be NULL
  const T* W;          // dense operand (OPD != 0), laid out like the mode product's output (L, ell, R)
  int64_t row0;        // Omega row of Kolda column 0 (a slab of a larger tensor: its global offset)
};

// Operand of the sketch: kOpOmega, the Gaussian stream generated on the fly (Alg. 1 step 1);
// kOpDense, a dense M x ell matrix W read from memory (the G_(n) W product of a subspace-iteration
// step), element (p, c) at (p % L) + L (c + ell (p / L)); kOpDenseSplit, the same with every
// element x of G replaced by the sum of its BF16 head and tail (the value the tensor-core kernels
// read for an FP32 input), FP32 only.
enum { kOpOmega = 0, kOpDense = 1, kOpDenseSplit = 2 };

template <typename T, int ELLP, bool KCONTIG, int OPD = kOpOmega>
struct SketchOp {
  using Args = SketchArgs<T>;
  static constexpr int kThreads = kNT, kMinBlocks = 2;
  // the dense operand tile lives in dynamic shared memory (kKP x ELLP elements of T)
  static constexpr size_t kDynSmem = OPD == kOpOmega ? 0 : sizeof(T) * kKP * ELLP;
  __device__ static void body(const Grid g, const Args& args);
};

template <typename T, int ELLP, bool KCONTIG, int OPD>
__device__ __forceinline__ void SketchOp<T, ELLP, KCONTIG, OPD>::body(const Grid g, const Args& args) {
  const T* __restrict__ G = args.G;
  const int64_t L = args.L, I = args.I, R = args.R;
  const int ell = args.ell;
  const int64_t chunk = args.chunk;
  const uint32_t k0 = args.k0, k1 = args.k1, sid = args.sid;
  T* __restrict__ part = args.part;
  double* __restrict__ part_norm = args.part_norm;
  constexpr int CG = ELLP / 4;      // groups of 4 Omega columns
  constexpr int IG = kNT / CG;      // groups of rows
  constexpr int TM = kTI / IG;      // rows per thread
  constexpr int VN = Vec<T>::n;
  using V = typename Vec<T>::type;
  using OT = std::conditional_t<OPD == kOpOmega, float, T>;   // element type of the operand tile
  static_assert(TM % VN == 0, "row group must be a whole number of vectors");
  static_assert(OPD != kOpDenseSplit || sizeof(T) == 4, "the split form reads FP32 data");

  __shared__ __align__(16) T Xs[kKP][kTI];
  __shared__ __align__(16) float Os_gen[OPD == kOpOmega ? kKP : 1][OPD == kOpOmega ? ELLP : 4];
  extern __shared__ __align__(16) unsigned char sketch_dense_raw[];
  OT(*Os)[ELLP] = OPD == kOpOmega ? reinterpret_cast<OT(*)[ELLP]>(&Os_gen[0][0])
                                  : reinterpret_cast<OT(*)[ELLP]>(sketch_dense_raw);
  __shared__ int64_t base_s[kKP];
  __shared__ double red[kNT / 32];
  const T* __restrict__ W = args.W;

  const int tid = threadIdx.x;
  const int tc = tid % CG;
  const int ti = tid / CG;
  const int64_t i0 = (int64_t)g.bx * kTI;
  const int64_t M = L * R;
  const int64_t pb = (int64_t)g.by * chunk;
  const int64_t pe = min(M, pb + chunk);

  T acc[TM][4];
  T acc2[TM][4];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = acc2[a][b] = T(0);
  double nrm = 0.0;

  int step = 0;
  for (int64_t p0 = pb; p0 < pe; p0 += kKP, ++step) {
    // -- column offsets of this k-step (non-contiguous view only)
    if (!KCONTIG) {
      if (tid < kKP) {
        const int64_t p = p0 + tid;
        base_s[tid] = (p < pe) ? (p % L) + L * I * (p / L) : int64_t(-1);
      }
      __syncthreads();
    }
    // -- operand tile: Omega generated, or rows p0 .. p0 + 31 of the dense W
    if constexpr (OPD == kOpOmega) {
      for (int t = tid; t < kKP * CG; t += kNT) {
        const int kp = t / CG, q = t % CG;
        const int64_t p = p0 + kp;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < pe) v = rng::omega4(k0, k1, sid, p + args.row0, (uint32_t)q);
        *reinterpret_cast<float4*>(&Os[kp][4 * q]) = v;
      }
    } else {
      for (int t = tid; t < kKP * ELLP; t += kNT) {
        const int kp = t / ELLP, c = t % ELLP;
        const int64_t p = p0 + kp;
        T v = T(0);
        if (p < pe && c < ell) v = __ldg(W + (KCONTIG ? (int64_t)ell * p : (p % L) + L * (int64_t)ell * (p / L)) + L * c);
        Os[kp][c] = v;
      }
    }
    // -- G tile, Xs[kp][ii] = G(i0 + ii, p0 + kp)
    T ss = T(0);
    if (KCONTIG) {
      // L == 1: element at I p + i, rows contiguous.
#pragma unroll 4
      for (int j = 0; j < (kKP * kTI) / kNT; ++j) {
        const int t = tid + j * kNT;
        const int ii = t % kTI, kp = t / kTI;
        const int64_t p = p0 + kp, i = i0 + ii;
        T x = T(0);
        if (p < pe && i < I) x = __ldg(G + I * p + i);
        if constexpr (OPD == kOpDenseSplit) x = split_value(x);
        ss += x * x;
        Xs[kp][swz<T>(kp, ii)] = x;
      }
    } else {
      const int lane = tid & 31, w = tid >> 5;
#pragma unroll 4
      for (int j = 0; j < (kKP * kTI) / kNT; ++j) {
        const int kp = (lane & 7) + 8 * (j & 3);
        const int ii = (lane >> 3) + 4 * w + 32 * (j >> 2);
        const int64_t b = base_s[kp];
        const int64_t i = i0 + ii;
        T x = T(0);
        if (b >= 0 && i < I) x = __ldg(G + b + L * i);
        if constexpr (OPD == kOpDenseSplit) x = split_value(x);
        ss += x * x;
        Xs[kp][swz<T>(kp, ii)] = x;
      }
    }
    nrm += (double)ss;
    __syncthreads();
    // -- accumulate the 128 x ELLP register tile
#pragma unroll 8
    for (int kp = 0; kp < kKP; ++kp) {
      T xv[TM];
#pragma unroll
      for (int a = 0; a < TM; a += VN) {
        const V v = *reinterpret_cast<const V*>(&Xs[kp][swz<T>(kp, ti * TM + a)]);
        if constexpr (VN == 4) {
          xv[a] = v.x; xv[a + 1] = v.y; xv[a + 2] = v.z; xv[a + 3] = v.w;
        } else {
          xv[a] = v.x; xv[a + 1] = v.y;
        }
      }
      T ov[4];
      if constexpr (OPD == kOpOmega) {
        const float4 o = *reinterpret_cast<const float4*>(&Os[kp][4 * tc]);
        ov[0] = T(o.x); ov[1] = T(o.y); ov[2] = T(o.z); ov[3] = T(o.w);
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) ov[b] = Os[kp][4 * tc + b];
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv[a], ov[b], acc[a][b]);
    }
    if (sizeof(T) == 4 && (step % kFlush) == kFlush - 1) {
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc2[a][b] += acc[a][b];
          acc[a][b] = T(0);
        }
    }
    __syncthreads();
  }
  // -- write the partial sketch part[s][c][i]
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int64_t i = i0 + ti * TM + a;
    if (i >= I) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = 4 * tc + b;
      if (c < ell) part[((int64_t)g.by * ell + c) * I + i] = acc2[a][b] + acc[a][b];
    }
  }
  // -- partial ||G||^2 of the elements this CTA loaded
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((tid & 31) == 0) red[tid >> 5] = nrm;
  __syncthreads();
  if (tid == 0 && part_norm != nullptr) {
    double s = 0.0;
    for (int k = 0; k < kNT / 32; ++k) s += red[k];
    part_norm[(int64_t)g.by * g.gx + g.bx] = s;
  }
}

// Small-row sketch (I <= 128, ell <= 32): the CTA keeps every row of its columns (TI >= I rows,
// TI in {32, 64, 128}), so each Omega row is generated once, and only the ceil(ell / 4) quads of
// it that are used.  A k-step covers KP = NTE / TI columns -- a tile of NTE elements (4096 FP32,
// 2048 FP64: 16 KB) whatever I is -- and the next tile is loaded into registers while the current
// one is multiplied.  The 256 threads are KS slices x TI/4 row groups x E/4 column groups; slice
// ks sums the columns kk = ks, ks + KS, ... of each tile and the slices are added at the end in a
// fixed order, so the result is deterministic.
template <typename T>
struct SketchSmallArgs {
  const T* G;
  int64_t L, I, R;
  int ell;
  int64_t chunk;
  uint32_t k0, k1, sid;
  T* part;
  double* part_norm;
  FastDiv fI, fL;   // division by I (unit-stride view) and by L (strided view)
  int64_t row0;     // Omega row of Kolda column 0
};

template <typename T>
struct SmallTile {
  static constexpr int NTE = sizeof(T) == 4 ? 4096 : 2048;   // tile elements (16 KB)
};

template <typename T, int TI, int E, bool KC>
struct SketchSmallOp {
  using Args = SketchSmallArgs<T>;
  static constexpr int kThreads = 256, kMinBlocks = 2;
  static constexpr int NTE = SmallTile<T>::NTE;
  static constexpr int KP = NTE / TI;              // columns per k-step
  static constexpr int IG = TI / 4, CG = E / 4;    // groups of 4 rows, of 4 columns
  static constexpr int KS = 256 / (IG * CG);       // column slices
  static constexpr int PER = NTE / 256;            // tile elements each thread loads
  static_assert(KS >= 1 && IG * CG * KS == 256, "thread split");
  static_assert(KP % 8 == 0 && KP % KS == 0, "tile shape");
  __device__ static void body(const Grid g, const Args& args);
};

template <typename T, int TI, int E, bool KC>
__device__ __forceinline__ void SketchSmallOp<T, TI, E, KC>::body(const Grid g, const Args& args) {
  using Op = SketchSmallOp<T, TI, E, KC>;
  constexpr int KP = Op::KP, CG = Op::CG, IG = Op::IG, KS = Op::KS, PER = Op::PER;
  constexpr int VN = Vec<T>::n;
  using V = typename Vec<T>::type;
  constexpr int TERMS = KP / KS;                   // products per accumulator per k-step
  constexpr int FLUSH = TERMS >= 512 ? 1 : 512 / TERMS;
  union Smem {
    struct {
      T Xs[KP][TI];
      float Os[KP][E];
    } t;
    T red[4096];
  };
  __shared__ __align__(16) Smem sm;
  __shared__ double nred[8];

  const T* __restrict__ G = args.G;
  const int64_t L = args.L, I = args.I, R = args.R;
  const int ell = args.ell;
  const int64_t M = L * R;
  const int64_t pb = (int64_t)g.by * args.chunk;
  const int64_t pe = min(M, pb + args.chunk);
  const int tid = threadIdx.x;
  const int cg = tid % CG, ig = (tid / CG) % IG, ks = tid / (CG * IG);
  const int nq = (ell + 3) / 4;
  const int Ii = (int)I;

  // -- loads of one tile into registers.  Unit-stride view: the tile is the contiguous run
  // G[I p0, I (p0 + KP)), element e at (kp, ii) = (e / I, e % I).  Strided view: each warp covers
  // 8 consecutive columns x 4 rows (32-byte runs), so a thread keeps one or two columns.
  T xr[PER];
  auto load_tile = [&](int64_t p0) {
    if (KC) {
      const int64_t lim = (min(pe, p0 + KP) - p0) * I;
      const T* src = G + I * p0;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = tid + 256 * j;
        xr[j] = (e < lim) ? __ldg(src + e) : T(0);
      }
    } else {
      const int lane = tid & 31;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int w = (tid >> 5) + 8 * j;
        const int kp = (lane & 7) + 8 * (w % (KP / 8));
        const int ii = (lane >> 3) + 4 * (w / (KP / 8));
        const int64_t p = p0 + kp;
        T x = T(0);
        if (p < pe && ii < Ii) {
          const uint32_t q = args.fL.div((uint32_t)p);
          x = __ldg(G + ((int64_t)((uint32_t)p - q * (uint32_t)L) + L * I * (int64_t)q + L * (int64_t)ii));
        }
        xr[j] = x;
      }
    }
  };
  auto store_tile = [&]() {
    T ss = T(0);
    if (KC) {
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = tid + 256 * j;
        if (e < KP * Ii) {
          const int kp = (int)args.fI.div((uint32_t)e), ii = e - kp * Ii;
          sm.t.Xs[kp][swz<T>(kp, ii)] = xr[j];
        }
        ss += xr[j] * xr[j];
      }
      // rows ii in [I, TI) of the tile stay zero (written once before the loop)
    } else {
      const int lane = tid & 31;
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int w = (tid >> 5) + 8 * j;
        const int kp = (lane & 7) + 8 * (w % (KP / 8));
        const int ii = (lane >> 3) + 4 * (w / (KP / 8));
        sm.t.Xs[kp][swz<T>(kp, ii)] = xr[j];
        ss += xr[j] * xr[j];
      }
    }
    return ss;
  };

  if (KC) {
    for (int e = tid; e < KP * TI; e += 256) (&sm.t.Xs[0][0])[e] = T(0);
    __syncthreads();
  }
  T acc[4][4], acc2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = acc2[a][b] = T(0);
  double nrm = 0.0;
  if (pb < pe) load_tile(pb);
  int step = 0;
  for (int64_t p0 = pb; p0 < pe; p0 += KP, ++step) {
    nrm += (double)store_tile();
    // Omega tile: quads q < nq of columns p0 .. p0 + KP - 1; the padded quads are zero
    for (int t = tid; t < KP * CG; t += 256) {
      const int kp = t / CG, q = t % CG;
      const int64_t p = p0 + kp;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (p < pe && q < nq) v = rng::omega4(args.k0, args.k1, args.sid, p + args.row0, (uint32_t)q);
      *reinterpret_cast<float4*>(&sm.t.Os[kp][4 * q]) = v;
    }
    __syncthreads();
    if (p0 + KP < pe) load_tile(p0 + KP);   // in flight during the products below
#pragma unroll 4
    for (int kk = ks; kk < KP; kk += KS) {
      T xv[4];
#pragma unroll
      for (int a = 0; a < 4; a += VN) {
        const V v = *reinterpret_cast<const V*>(&sm.t.Xs[kk][swz<T>(kk, 4 * ig + a)]);
        if constexpr (VN == 4) {
          xv[0] = v.x; xv[1] = v.y; xv[2] = v.z; xv[3] = v.w;
        } else {
          xv[a] = v.x; xv[a + 1] = v.y;
        }
      }
      const float4 o = *reinterpret_cast<const float4*>(&sm.t.Os[kk][4 * cg]);
      const T ov[4] = {T(o.x), T(o.y), T(o.z), T(o.w)};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xv[a], ov[b], acc[a][b]);
    }
    if (sizeof(T) == 4 && (step % FLUSH) == FLUSH - 1) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc2[a][b] += acc[a][b];
          acc[a][b] = T(0);
        }
    }
    __syncthreads();
  }
  // -- slices: red[ks][c][i], summed over ks in order; then part[by][c][i]
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sm.red[(ks * E + 4 * cg + b) * TI + 4 * ig + a] = acc2[a][b] + acc[a][b];
  __syncthreads();
  for (int t = tid; t < TI * E; t += 256) {
    const int i = t % TI, c = t / TI;
    T v = sm.red[c * TI + i];
#pragma unroll
    for (int k = 1; k < KS; ++k) v += sm.red[(k * E + c) * TI + i];
    if (i < Ii && c < ell) args.part[((int64_t)g.by * ell + c) * I + i] = v;
  }
  // -- partial ||G||^2 of the elements this CTA loaded
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if ((tid & 31) == 0) nred[tid >> 5] = nrm;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += nred[k];
    args.part_norm[(int64_t)g.by * g.gx + g.bx] = t;
  }
}

// Y(i, c) = sum over the S splits of part[k][c][i], in FP64.  CTA (bx, c) owns rows
// i in [32 bx, 32 bx + 32) of column c; warp w sums the splits k = w, w + 8, ... (each warp
// load is 32 consecutive rows, one 128-byte line for FP32), and warp 0 adds the 8 warp sums in
// a fixed order, so the result does not depend on timing.  CTA (0, 0) also sums the per-CTA
// squared norms with a fixed-shape tree.
constexpr int kRedWarps = 8;

template <typename T>
struct SketchReduceArgs {
  const T* part;
  int S;
  int64_t I;
  int ell;
  double* Y;
  const double* part_norm;
  int nnorm;
  double* norm2;
  int accumulate;   // 1: add to Y (and *norm2) instead of overwriting them
};

template <typename T>
struct SketchReduceOp {
  using Args = SketchReduceArgs<T>;
  static constexpr int kThreads = 32 * kRedWarps, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};

template <typename T>
__device__ __forceinline__ void SketchReduceOp<T>::body(const Grid g, const Args& args) {
  const T* __restrict__ part = args.part;
  const int S = args.S;
  const int64_t I = args.I;
  const int ell = args.ell;
  double* __restrict__ Y = args.Y;
  const double* __restrict__ part_norm = args.part_norm;
  const int nnorm = args.nnorm;
  double* __restrict__ norm2 = args.norm2;
  __shared__ double red[kRedWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t c = g.by;
  const int64_t i = (int64_t)g.bx * 32 + lane;
  if constexpr (sizeof(T) == 4) {
    // FP32 partials, summed in FP32 pairs (hi, lo) that keep every rounding error (Knuth's TwoSum):
    // ~2^-44 relative error at FP32 arithmetic rate, converted to FP64 once per output (FP64 runs
    // at a small fraction of the FP32 rate on this part).  Eight chains per lane (loads in flight
    // together) and the eight warps are combined in a fixed order, so the result is deterministic.
    __shared__ float redh[kRedWarps][33], redl[kRedWarps][33];
    auto acc = [](float& h, float& l, float v) {
      const float t = __fadd_rn(h, v);
      const float bp = __fsub_rn(t, h);
      l = __fadd_rn(l, __fadd_rn(__fsub_rn(h, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
      h = t;
    };
    float H = 0.0f, L = 0.0f;
    if (i < I) {
      const T* src = part + c * I + i;
      const int64_t step = (int64_t)ell * I;
      int k = w;
      float hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) hi[j] = lo[j] = 0.0f;
      for (; k + 7 * kRedWarps < S; k += 8 * kRedWarps) {
#pragma unroll
        for (int j = 0; j < 8; ++j) acc(hi[j], lo[j], (float)src[(int64_t)(k + j * kRedWarps) * step]);
      }
      for (; k < S; k += kRedWarps) acc(hi[0], lo[0], (float)src[(int64_t)k * step]);
      H = hi[0];
      L = lo[0];
#pragma unroll
      for (int j = 1; j < 8; ++j) {
        acc(H, L, hi[j]);
        L = __fadd_rn(L, lo[j]);
      }
    }
    redh[w][lane] = H;
    redl[w][lane] = L;
    __syncthreads();
    if (w == 0 && i < I) {
      float h = redh[0][lane], l = redl[0][lane];
#pragma unroll
      for (int j = 1; j < kRedWarps; ++j) {
        acc(h, l, redh[j][lane]);
        l = __fadd_rn(l, redl[j][lane]);
      }
      const double t = (double)h + (double)l;
      Y[i + I * c] = args.accumulate ? Y[i + I * c] + t : t;
    }
  } else {
    double s = 0.0;
    if (i < I) {
      const T* src = part + c * I + i;
      const int64_t step = (int64_t)ell * I;
      int k = w;
      // eight independent chains per lane (loads in flight together), combined in a fixed order
      double cc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (; k + 7 * kRedWarps < S; k += 8 * kRedWarps) {
#pragma unroll
        for (int j = 0; j < 8; ++j) cc[j] += (double)src[(int64_t)(k + j * kRedWarps) * step];
      }
      for (; k < S; k += kRedWarps) cc[0] += (double)src[(int64_t)k * step];
      s = ((cc[0] + cc[1]) + (cc[2] + cc[3])) + ((cc[4] + cc[5]) + (cc[6] + cc[7]));
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < I) {
      double t = red[0][lane];
#pragma unroll
      for (int j = 1; j < kRedWarps; ++j) t += red[j][lane];
      Y[i + I * c] = args.accumulate ? Y[i + I * c] + t : t;
    }
  }
  if (norm2 != nullptr && g.bx == 0 && g.by == 0) {
    __syncthreads();
    double t = 0.0;
    for (int k = threadIdx.x; k < nnorm; k += blockDim.x) t += part_norm[k];
    double* flat = &red[0][0];
    flat[threadIdx.x] = t;   // 256 <= 8 * 33
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) flat[threadIdx.x] += flat[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) *norm2 = args.accumulate ? *norm2 + flat[0] : flat[0];
  }
}

}  // namespace

SketchPlan plan_sketch(const ModeView& v, int ell) {
  SketchPlan pl;
  pl.v = v;
  pl.ell = ell;
  const int64_t M = v.M();
  if (v.I <= 128 && ell <= 32 && M < (int64_t(1) << 31)) {
    // small-row kernel: one row tile; at least tune(min_steps) k-steps per CTA, tune(ctas_per_sm)
    // CTAs per SM at most (tuning_table.inc)
    pl.ti = v.I <= 32 ? 32 : (v.I <= 64 ? 64 : 128);
    pl.ellp = ell <= 8 ? 8 : (ell <= 16 ? 16 : 32);
    pl.gx = 1;
    const int64_t kp = 4096 / pl.ti;   // FP32 tile columns (a multiple of the FP64 ones)
    const int64_t ksteps = ceil_div(M, kp);
    const int64_t S = std::max<int64_t>(1, std::min<int64_t>((int64_t)tune(TUNE_SKETCH_SMALL_CTAS_PER_SM) * num_sms(),
                                                             ceil_div(ksteps, tune(TUNE_SKETCH_SMALL_MIN_STEPS))));
    pl.chunk = ceil_div(ksteps, S) * kp;
    pl.S = (int)ceil_div(M, pl.chunk);
    return pl;
  }
  pl.ellp = ell_pad_of(ell);
  pl.gx = (int)ceil_div(v.I, kTI);
  const int64_t ksteps = ceil_div(M, kKP);
  // about 4 CTAs per SM (the partial sums are reduced by warps over the splits, so many splits
  // stay cheap even for small I)
  const int64_t target = 4LL * num_sms();
  const int64_t S = std::max<int64_t>(1, std::min<int64_t>(ceil_div(target, pl.gx), ksteps));
  pl.chunk = ceil_div(ceil_div(M, S), kKP) * kKP;
  pl.S = (int)ceil_div(M, pl.chunk);
  return pl;
}

template <typename T, int TI, int E>
static rh_status emit_sketch_small(const SketchPlan& pl, const SketchSmallArgs<T>& a, cudaStream_t st) {
  const dim3 grid(1, pl.S);
  return pl.v.L == 1 ? emit<SketchSmallOp<T, TI, E, true>>(SITE_SKETCH, 0, grid, 0, st, a)
                     : emit<SketchSmallOp<T, TI, E, false>>(SITE_SKETCH, 0, grid, 0, st, a);
}

template <typename T, int TI>
static rh_status emit_sketch_small_e(const SketchPlan& pl, const SketchSmallArgs<T>& a, cudaStream_t st) {
  if (pl.ellp == 8) return emit_sketch_small<T, TI, 8>(pl, a, st);
  if (pl.ellp == 16) return emit_sketch_small<T, TI, 16>(pl, a, st);
  return emit_sketch_small<T, TI, 32>(pl, a, st);
}

template <typename T>
rh_status launch_sketch(const SketchPlan& pl, const T* G, uint64_t seed, uint32_t sid, T* part, double* part_norm,
                        cudaStream_t st) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  if (pl.ti > 0) {
    const SketchSmallArgs<T> a{G, pl.v.L, pl.v.I, pl.v.R, pl.ell, pl.chunk, k0, k1, sid, part, part_norm,
                               FastDiv((uint32_t)pl.v.I), FastDiv((uint32_t)pl.v.L), pl.row0};
    if (pl.ti == 32) return emit_sketch_small_e<T, 32>(pl, a, st);
    if (pl.ti == 64) return emit_sketch_small_e<T, 64>(pl, a, st);
    return emit_sketch_small_e<T, 128>(pl, a, st);
  }
  const dim3 grid(pl.gx, pl.S);
  const bool kc = (pl.v.L == 1);
  const SketchArgs<T> a{G, pl.v.L, pl.v.I, pl.v.R, pl.ell, pl.chunk, k0, k1, sid, part, part_norm, nullptr, pl.row0};
  if (pl.ellp == 32)
    return kc ? emit<SketchOp<T, 32, true>>(SITE_SKETCH, 0, grid, 0, st, a)
              : emit<SketchOp<T, 32, false>>(SITE_SKETCH, 0, grid, 0, st, a);
  return kc ? emit<SketchOp<T, 64, true>>(SITE_SKETCH, 0, grid, 0, st, a)
            : emit<SketchOp<T, 64, false>>(SITE_SKETCH, 0, grid, 0, st, a);
}

SketchPlan plan_sketch_dense(const ModeView& v, int ell) {
  SketchPlan pl;
  pl.v = v;
  pl.ell = ell;
  pl.ellp = ell_pad_of(ell);
  pl.gx = (int)ceil_div(v.I, kTI);
  const int64_t ksteps = ceil_div(v.M(), kKP);
  const int64_t target = 4LL * num_sms();
  const int64_t S = std::max<int64_t>(1, std::min<int64_t>(ceil_div(target, pl.gx), ksteps));
  pl.chunk = ceil_div(ceil_div(v.M(), S), kKP) * kKP;
  pl.S = (int)ceil_div(v.M(), pl.chunk);
  return pl;
}

template <typename T, int ELLP, int OPD>
static rh_status emit_sketch_dense(const SketchPlan& pl, const SketchArgs<T>& a, cudaStream_t st, int site) {
  const dim3 grid(pl.gx, pl.S);
  using OpC = SketchOp<T, ELLP, true, OPD>;
  using OpS = SketchOp<T, ELLP, false, OPD>;
  return pl.v.L == 1 ? emit<OpC>(site, 0, grid, OpC::kDynSmem, st, a) : emit<OpS>(site, 0, grid, OpS::kDynSmem, st, a);
}

template <typename T>
rh_status launch_sketch_dense(const SketchPlan& pl, const T* G, const T* W, bool split, T* part, cudaStream_t st,
                              int site) {
  if (pl.ti != 0) {
    set_error("dense sketch: needs the plan of plan_sketch_dense");
    return RH_EUNSUPPORTED;
  }
  const SketchArgs<T> a{G, pl.v.L, pl.v.I, pl.v.R, pl.ell, pl.chunk, 0u, 0u, 0u, part, nullptr, W, 0};
  if constexpr (sizeof(T) == 4) {
    if (split)
      return pl.ellp == 32 ? emit_sketch_dense<T, 32, kOpDenseSplit>(pl, a, st, site)
                           : emit_sketch_dense<T, 64, kOpDenseSplit>(pl, a, st, site);
  }
  return pl.ellp == 32 ? emit_sketch_dense<T, 32, kOpDense>(pl, a, st, site)
                       : emit_sketch_dense<T, 64, kOpDense>(pl, a, st, site);
}

template <typename T>
rh_status launch_sketch_reduce(const SketchPlan& pl, const T* part, const double* part_norm, double* Y, double* norm2,
                               cudaStream_t st, int site, int accumulate) {
  if (pl.ell > 65535) {
    set_error("sketch reduce: too many columns");
    return RH_EUNSUPPORTED;
  }
  const dim3 grid((unsigned)ceil_div(pl.v.I, 32), (unsigned)pl.ell);
  return emit<SketchReduceOp<T>>(site, 0, grid, 0, st,
                                 SketchReduceArgs<T>{part, pl.S, pl.v.I, pl.ell, Y, part_norm, (int)pl.norm_elems(), norm2,
                                                     accumulate});
}

template rh_status launch_sketch<float>(const SketchPlan&, const float*, uint64_t, uint32_t, float*, double*,
                                        cudaStream_t);
template rh_status launch_sketch<double>(const SketchPlan&, const double*, uint64_t, uint32_t, double*, double*,
                                         cudaStream_t);
template rh_status launch_sketch_reduce<float>(const SketchPlan&, const float*, const double*, double*, double*,
                                               cudaStream_t, int, int);
template rh_status launch_sketch_reduce<double>(const SketchPlan&, const double*, const double*, double*, double*,
                                                cudaStream_t, int, int);
template rh_status launch_sketch_dense<float>(const SketchPlan&, const float*, const float*, bool, float*, cudaStream_t,
                                              int);
template rh_status launch_sketch_dense<double>(const SketchPlan&, const double*, const double*, bool, double*,
                                               cudaStream_t, int);

}  // namespace rh
