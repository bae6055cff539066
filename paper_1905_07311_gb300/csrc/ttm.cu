// Mode-n product B = G x_n Q^T (Sec. 2.1: Y_(n) = A X_(n) with A = Q^T), the step that
// forms B = Q^T X in Alg. 1 step 3, the truncated core G <- U_r^T B of Alg. 3 step 6, the core
// of Alg. 2 step 6 and, with Q^T replaced by a factor A, the Tucker reconstruction.
//
// With G viewed as (L, I, R) and p = l + L r:
//   B[(p % L) + L ko (p / L) + L c] = sum_i Q(i, c) G[(p % L) + L I (p / L) + L i],  c < ko,
// where Q(i, c) = Q[i qsi + c qsc] (qsi = 1, qsc = I for an I x ko column-major Q; qsi = ko,
// qsc = 1 for a ko x I column-major A used untransposed).  The output keeps the layout of G
// with mode n resized to ko, i.e. it is directly the column-major tensor G x_n Q^T.  No
// unfolding is materialised.
//
// CTA tile: 128 columns p of the unfolding x 64 output rows (blockIdx.y selects the group of
// 64); the reduction over i runs in steps of 32 through shared memory.  The residual variant
// does not store the tile: it adds sum (X - B)^2 over the tile to a per-CTA FP64 partial.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace rh {

namespace {

constexpr int kTP = 128;
constexpr int kKI = 32;
constexpr int kNT = 256;

template <typename T>
struct V2;
template <>
struct V2<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct V2<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ int swz(int k, int col) {
  return col ^ ((k & 7) * V2<T>::n);
}

template <typename T, typename TO>
struct TtmArgs {
  const T* G;
  int64_t L, I, R;
  const T* Q;
  int64_t qsi, qsc;
  int ko;
  TO* B;
  const T* Xref;
  double* part;
};

template <typename T, typename TO, int ELLP, bool KCONTIG, bool RESID>
struct TtmOp {
  using Args = TtmArgs<T, TO>;
  static constexpr int kThreads = kNT, kMinBlocks = 2;
  __device__ static void body(const Grid g, const Args& args);
};

template <typename T, typename TO, int ELLP, bool KCONTIG, bool RESID>
__device__ __forceinline__ void TtmOp<T, TO, ELLP, KCONTIG, RESID>::body(const Grid g, const Args& args) {
  const T* __restrict__ G = args.G;
  const int64_t L = args.L, I = args.I, R = args.R;
  const T* __restrict__ Q = args.Q;
  const int64_t qsi = args.qsi, qsc = args.qsc;
  const int ko = args.ko;
  TO* __restrict__ B = args.B;
  const T* __restrict__ Xref = args.Xref;
  double* __restrict__ part = args.part;
  constexpr int CG = ELLP / 4;
  constexpr int PG = kNT / CG;
  constexpr int TM = kTP / PG;
  constexpr int VN = V2<T>::n;
  using V = typename V2<T>::type;
  static_assert(TM % VN == 0, "column group must be a whole number of vectors");

  __shared__ __align__(16) T Gs[kKI][kTP];
  __shared__ __align__(16) T Qs[kKI][ELLP];

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  const int tc = tid % CG;
  const int tp = tid / CG;
  const int64_t M = L * R;
  const int64_t p0 = (int64_t)g.bx * kTP;
  const int cb = (int)g.by * ELLP;  // first output row of this CTA

  // Per-thread column offset for the non-contiguous view: thread owns column pp = tid % 128.
  int64_t mybase = -1;
  if (!KCONTIG) {
    const int64_t p = p0 + (tid % kTP);
    if (p < M) mybase = (p % L) + L * I * (p / L);
  }

  T acc[TM][4];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

  for (int64_t i0 = 0; i0 < I; i0 += kKI) {
    // Q tile: Qs[ki][c] = Q[(i0 + ki) + I c]
#pragma unroll
    for (int j = 0; j < (kKI * ELLP) / kNT; ++j) {
      const int ki = (lane & 7) + 8 * (j & 3);
      const int c = (lane >> 3) + 4 * w + 32 * (j >> 2);
      const int64_t i = i0 + ki;
      T q = T(0);
      if (cb + c < ko && i < I) q = __ldg(Q + i * qsi + (int64_t)(cb + c) * qsc);
      Qs[ki][swz<T>(ki, c)] = q;
    }
    // G tile: Gs[ki][pp] = G(i0 + ki, p0 + pp)
    if (KCONTIG) {
#pragma unroll 4
      for (int j = 0; j < (kKI * kTP) / kNT; ++j) {
        const int ki = (lane & 7) + 8 * (j & 3);
        const int pp = (lane >> 3) + 4 * w + 32 * (j >> 2);
        const int64_t p = p0 + pp, i = i0 + ki;
        T x = T(0);
        if (p < M && i < I) x = __ldg(G + I * p + i);
        Gs[ki][swz<T>(ki, pp)] = x;
      }
    } else {
      const int pp = tid % kTP;
#pragma unroll 4
      for (int j = 0; j < (kKI * kTP) / kNT; ++j) {
        const int ki = tid / kTP + 2 * j;
        const int64_t i = i0 + ki;
        T x = T(0);
        if (mybase >= 0 && i < I) x = __ldg(G + mybase + L * i);
        Gs[ki][swz<T>(ki, pp)] = x;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int ki = 0; ki < kKI; ++ki) {
      T gv[TM];
#pragma unroll
      for (int a = 0; a < TM; a += VN) {
        const V v = *reinterpret_cast<const V*>(&Gs[ki][swz<T>(ki, tp * TM + a)]);
        if constexpr (VN == 4) {
          gv[a] = v.x; gv[a + 1] = v.y; gv[a + 2] = v.z; gv[a + 3] = v.w;
        } else {
          gv[a] = v.x; gv[a + 1] = v.y;
        }
      }
      T qv[4];
#pragma unroll
      for (int b = 0; b < 4; b += VN) {
        const V v = *reinterpret_cast<const V*>(&Qs[ki][swz<T>(ki, 4 * tc + b)]);
        if constexpr (VN == 4) {
          qv[0] = v.x; qv[1] = v.y; qv[2] = v.z; qv[3] = v.w;
        } else {
          qv[b] = v.x; qv[b + 1] = v.y;
        }
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(gv[a], qv[b], acc[a][b]);
    }
    __syncthreads();
  }

  if (RESID) {
    // sum over the tile of (Xref - B)^2, Xref laid out like the output
    double acc2 = 0.0;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int64_t p = p0 + tp * TM + a;
      if (p >= M) continue;
      const int64_t ob = (p % L) + L * (int64_t)ko * (p / L);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = cb + 4 * tc + b;
        if (c < ko) {
          const double dlt = (double)Xref[ob + L * (int64_t)c] - (double)acc[a][b];
          acc2 += dlt * dlt;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
    __shared__ double red[kNT / 32];
    if (lane == 0) red[w] = acc2;
    __syncthreads();
    if (tid == 0) {
      double s2 = 0.0;
      for (int k = 0; k < kNT / 32; ++k) s2 += red[k];
      part[(int64_t)g.by * g.gx + g.bx] = s2;
    }
  } else if (KCONTIG) {
    // B[c + ko p]: a row p holds ko contiguous outputs.
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int64_t p = p0 + tp * TM + a;
      if (p >= M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = cb + 4 * tc + b;
        if (c < ko) B[(int64_t)ko * p + c] = (TO)acc[a][b];
      }
    }
  } else {
    // Stage 32 output rows at a time through Gs, then store along p (contiguous).
    int64_t obase = -1;
    {
      const int64_t p = p0 + (tid % kTP);
      if (p < M) obase = (p % L) + L * (int64_t)ko * (p / L);
    }
    for (int h = 0; h < ELLP / 32; ++h) {
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int c = 4 * tc + b - 32 * h;
          if (c >= 0 && c < 32) Gs[c][swz<T>(c, tp * TM + a)] = acc[a][b];
        }
      __syncthreads();
      const int pp = tid % kTP;
#pragma unroll 4
      for (int j = 0; j < (32 * kTP) / kNT; ++j) {
        const int cl = tid / kTP + 2 * j;
        const int c = cb + cl + 32 * h;
        if (obase >= 0 && c < ko) B[obase + L * (int64_t)c] = (TO)Gs[cl][swz<T>(cl, pp)];
      }
      __syncthreads();
    }
  }
}

// Small mode product (FP32, I <= 128, ko <= 32): E = 16 or 32 output rows (ko padded), tiles of
// PT = 4096 / E columns, the reduction over i in chunks of KI = E rows (a 16 KB tile of G per
// chunk).  Each CTA loads Q once into shared memory and walks a contiguous range of column tiles;
// the G block of the next (tile, chunk) is loaded into registers while the current one is
// multiplied.  Every output sums over i in increasing order in one FP32 accumulator, as the
// general kernel does.  A finished tile is staged through shared memory and stored along the
// contiguous direction of B.
template <typename TO>
struct TtmSmallArgs {
  const float* G;
  int64_t L, I, R;
  const float* Q;
  int64_t qsi, qsc;
  int ko;
  TO* B;
  int64_t tiles_per_cta;
  FastDiv fL, fko;
};

template <typename TO, int E, bool KC>
struct TtmSmallOp {
  using Args = TtmSmallArgs<TO>;
  static constexpr int kThreads = 256, kMinBlocks = 2;
  static constexpr int CG = E / 4;        // column groups of 4 outputs
  static constexpr int PT = 4096 / E;     // columns per tile (4 per thread)
  static constexpr int KI = E;            // rows per chunk
  __device__ static void body(const Grid g, const Args& args);
};

template <typename TO, int E, bool KC>
__device__ __forceinline__ void TtmSmallOp<TO, E, KC>::body(const Grid g, const Args& args) {
  using Op = TtmSmallOp<TO, E, KC>;
  constexpr int CG = Op::CG, PT = Op::PT, KI = Op::KI;
  __shared__ __align__(16) float Gs[KI][PT];
  __shared__ __align__(16) float Qs[128][E];
  const float* __restrict__ G = args.G;
  const int64_t L = args.L, I = args.I, R = args.R;
  const int64_t M = L * R;
  const int ko = args.ko;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int tc = tid % CG, tp = tid / CG;
  const int nch = (int)((I + KI - 1) / KI);
  const int64_t ntiles = (M + PT - 1) / PT;
  const int64_t t0 = (int64_t)g.bx * args.tiles_per_cta;
  const int64_t t1 = min(ntiles, t0 + args.tiles_per_cta);
  if (t0 >= t1) return;
  for (int e = tid; e < 128 * E; e += 256) {
    const int i = e / E, c = e % E;
    Qs[i][c] = (i < I && c < ko) ? __ldg(args.Q + i * args.qsi + (int64_t)c * args.qsc) : 0.f;
  }
  // register block of one (tile, chunk): 16 elements per thread.  Unit stride: warp task (kq, pq)
  // covers rows 8 kq .. 8 kq + 7 of columns 4 pq .. 4 pq + 3 (32-byte runs); strided view: a warp
  // covers 32 consecutive columns of one row, and each thread keeps one column.
  float xr[16];
  auto load = [&](int64_t tile, int ch) {
    const int64_t p0 = tile * PT;
    const int64_t i0 = (int64_t)ch * KI;
    if (KC) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int task = w + 8 * j;
        const int ki = (lane & 7) + 8 * (task % (KI / 8));
        const int pp = (lane >> 3) + 4 * (task / (KI / 8));
        const int64_t p = p0 + pp, i = i0 + ki;
        xr[j] = (p < M && i < I) ? __ldg(G + I * p + i) : 0.f;
      }
    } else {
      const int pp = lane + 32 * (w % (PT / 32));
      const int64_t p = p0 + pp;
      int64_t base = -1;
      if (p < M) {
        const uint32_t q = args.fL.div((uint32_t)p);
        base = (int64_t)((uint32_t)p - q * (uint32_t)L) + L * I * (int64_t)q;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int task = w + 8 * j;
        const int ki = task / (PT / 32);
        const int64_t i = i0 + ki;
        xr[j] = (base >= 0 && i < I) ? __ldg(G + base + L * i) : 0.f;
      }
    }
  };
  auto store = [&]() {
    if (KC) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int task = w + 8 * j;
        const int ki = (lane & 7) + 8 * (task % (KI / 8));
        const int pp = (lane >> 3) + 4 * (task / (KI / 8));
        Gs[ki][swz<float>(ki, pp)] = xr[j];
      }
    } else {
      const int pp = lane + 32 * (w % (PT / 32));
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int task = w + 8 * j;
        const int ki = task / (PT / 32);
        Gs[ki][swz<float>(ki, pp)] = xr[j];
      }
    }
  };
  float acc[4][4];
  load(t0, 0);
  __syncthreads();   // Qs
  for (int64_t tile = t0; tile < t1; ++tile) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int ch = 0; ch < nch; ++ch) {
      store();
      __syncthreads();
      if (ch + 1 < nch)
        load(tile, ch + 1);
      else if (tile + 1 < t1)
        load(tile + 1, 0);
      const int i0 = ch * KI;
#pragma unroll 8
      for (int ki = 0; ki < KI; ++ki) {
        const float4 gv = *reinterpret_cast<const float4*>(&Gs[ki][swz<float>(ki, 4 * tp)]);
        const float4 qv = *reinterpret_cast<const float4*>(&Qs[i0 + ki][4 * tc]);
        const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
        const float qq[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(gg[a], qq[b], acc[a][b]);
      }
      __syncthreads();
    }
    // stage the tile as Gs[c][pp] (E x PT = 4096 values) and store it
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = 4 * tc + b;
        Gs[c][swz<float>(c, 4 * tp + a)] = acc[a][b];
      }
    __syncthreads();
    const int64_t p0 = tile * PT;
    if (KC) {
      // B[ko p + c]: the tile is the contiguous run B[ko p0, ko (p0 + PT))
      const int64_t n = (min(M, p0 + PT) - p0) * ko;
      TO* dst = args.B + (int64_t)ko * p0;
      for (int e = tid; e < n; e += 256) {
        const int pp = (int)args.fko.div((uint32_t)e), c = e - pp * ko;
        dst[e] = (TO)Gs[c][swz<float>(c, pp)];
      }
    } else {
      for (int pp = tid; pp < PT; pp += 256) {
        const int64_t p = p0 + pp;
        if (p >= M) continue;
        const uint32_t q = args.fL.div((uint32_t)p);
        const int64_t ob = (int64_t)((uint32_t)p - q * (uint32_t)L) + L * (int64_t)ko * (int64_t)q;
        for (int c = 0; c < ko; ++c) args.B[ob + L * (int64_t)c] = (TO)Gs[c][swz<float>(c, pp)];
      }
    }
    __syncthreads();
  }
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double s2 = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s2 += part[e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    *out = t;
  }
}

}  // namespace

template <typename T, typename TO, bool RESID>
static rh_status launch_ttm_impl(const ModeView& v, const T* G, const T* Q, int64_t qsi, int64_t qsc, int ko, TO* B,
                                 const T* Xref, double* part, cudaStream_t st, int site = SITE_OTHER) {
  if (ko < 1) {
    set_error("internal: mode product output width < 1");
    return RH_EINVAL;
  }
  const int64_t M = v.M();
  const int64_t bx = ceil_div(M, kTP);
  const bool kc = (v.L == 1);
  const int ellp = ko <= 32 ? 32 : 64;
  const int64_t by = ceil_div(ko, ellp);
  if (bx > 0x7FFFFFFFLL || by > 65535) {
    set_error("internal: mode product grid too large");
    return RH_EUNSUPPORTED;
  }
  if constexpr (!RESID && sizeof(T) == 4) {
    if (v.I <= 128 && ko <= 32 && M < (int64_t(1) << 31) && (int64_t)ko * M < (int64_t(1) << 31)) {
      // small path: at least tune(min_tiles) tiles per CTA, tune(ctas_per_sm) CTAs per SM at most
      const int E = ko <= 16 ? 16 : 32;
      const int64_t ntiles = ceil_div(M, 4096 / E);
      const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>((int64_t)tune(TUNE_TTM_SMALL_CTAS_PER_SM) * num_sms(),
                                                                  ceil_div(ntiles, tune(TUNE_TTM_SMALL_MIN_TILES))));
      const int64_t tpc = ceil_div(ntiles, ctas);
      const dim3 g1((unsigned)ceil_div(ntiles, tpc));
      const TtmSmallArgs<TO> a{G, v.L, v.I, v.R, Q, qsi, qsc, ko, B, tpc, FastDiv((uint32_t)v.L),
                               FastDiv((uint32_t)ko)};
      if (E == 16)
        return kc ? emit<TtmSmallOp<TO, 16, true>>(site, 0, g1, 0, st, a)
                  : emit<TtmSmallOp<TO, 16, false>>(site, 0, g1, 0, st, a);
      return kc ? emit<TtmSmallOp<TO, 32, true>>(site, 0, g1, 0, st, a)
                : emit<TtmSmallOp<TO, 32, false>>(site, 0, g1, 0, st, a);
    }
  }
  const dim3 grid((unsigned)bx, (unsigned)by);
  const TtmArgs<T, TO> a{G, v.L, v.I, v.R, Q, qsi, qsc, ko, B, Xref, part};
  if (ellp == 32)
    return kc ? emit<TtmOp<T, TO, 32, true, RESID>>(site, 0, grid, 0, st, a)
              : emit<TtmOp<T, TO, 32, false, RESID>>(site, 0, grid, 0, st, a);
  return kc ? emit<TtmOp<T, TO, 64, true, RESID>>(site, 0, grid, 0, st, a)
            : emit<TtmOp<T, TO, 64, false, RESID>>(site, 0, grid, 0, st, a);
}

template <typename T, typename TO>
rh_status launch_ttm(const ModeView& v, const T* G, const T* Q, int ko, TO* B, cudaStream_t st, int site) {
  return launch_ttm_impl<T, TO, false>(v, G, Q, 1, v.I, ko, B, nullptr, nullptr, st, site);
}

template <typename T, typename TO>
rh_status launch_ttm_strided(const ModeView& v, const T* G, const T* Q, int64_t qsi, int64_t qsc, int ko, TO* B,
                             cudaStream_t st) {
  return launch_ttm_impl<T, TO, false>(v, G, Q, qsi, qsc, ko, B, nullptr, nullptr, st);
}

int64_t ttm_resid_parts(const ModeView& v, int ko) {
  const int ellp = ko <= 32 ? 32 : 64;
  return ceil_div(v.M(), kTP) * ceil_div(ko, ellp);
}

template <typename T>
rh_status launch_ttm_residual(const ModeView& v, const T* G, const T* Q, int64_t qsi, int64_t qsc, int ko,
                              const T* Xref, double* part, double* out, cudaStream_t st) {
  rh_status s = launch_ttm_impl<T, T, true>(v, G, Q, qsi, qsc, ko, nullptr, Xref, part, st);
  if (s != RH_OK) return s;
  sum_parts_kernel<<<1, 1024, 0, st>>>(part, ttm_resid_parts(v, ko), out);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template rh_status launch_ttm<float, float>(const ModeView&, const float*, const float*, int, float*, cudaStream_t, int);
template rh_status launch_ttm<float, double>(const ModeView&, const float*, const float*, int, double*, cudaStream_t,
                                             int);
template rh_status launch_ttm<double, double>(const ModeView&, const double*, const double*, int, double*,
                                              cudaStream_t, int);
template rh_status launch_ttm_strided<float, float>(const ModeView&, const float*, const float*, int64_t, int64_t, int,
                                                    float*, cudaStream_t);
template rh_status launch_ttm_strided<float, double>(const ModeView&, const float*, const float*, int64_t, int64_t,
                                                     int, double*, cudaStream_t);
template rh_status launch_ttm_strided<double, double>(const ModeView&, const double*, const double*, int64_t, int64_t,
                                                      int, double*, cudaStream_t);
template rh_status launch_ttm_residual<float>(const ModeView&, const float*, const float*, int64_t, int64_t, int,
                                              const float*, double*, double*, cudaStream_t);
template rh_status launch_ttm_residual<double>(const ModeView&, const double*, const double*, int64_t, int64_t, int,
                                               const double*, double*, double*, cudaStream_t);

}  // namespace rh
