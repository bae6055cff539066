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

template <typename T, typename TO, int ELLP, bool KCONTIG, bool RESID>
__global__ void __launch_bounds__(kNT, 2)
    ttm_kernel(const T* __restrict__ G, int64_t L, int64_t I, int64_t R, const T* __restrict__ Q, int64_t qsi,
               int64_t qsc, int ko, TO* __restrict__ B, const T* __restrict__ Xref, double* __restrict__ part) {
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
  const int64_t p0 = (int64_t)blockIdx.x * kTP;
  const int cb = blockIdx.y * ELLP;  // first output row of this CTA

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
      part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s2;
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
                                 const T* Xref, double* part, cudaStream_t st) {
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
  const dim3 grid((unsigned)bx, (unsigned)by);
#define RH_TTM(E, KC) \
  ttm_kernel<T, TO, E, KC, RESID><<<grid, kNT, 0, st>>>(G, v.L, v.I, v.R, Q, qsi, qsc, ko, B, Xref, part)
  if (ellp == 32) {
    if (kc) RH_TTM(32, true); else RH_TTM(32, false);
  } else {
    if (kc) RH_TTM(64, true); else RH_TTM(64, false);
  }
#undef RH_TTM
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template <typename T, typename TO>
rh_status launch_ttm(const ModeView& v, const T* G, const T* Q, int ko, TO* B, cudaStream_t st) {
  return launch_ttm_impl<T, TO, false>(v, G, Q, 1, v.I, ko, B, nullptr, nullptr, st);
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

template rh_status launch_ttm<float, float>(const ModeView&, const float*, const float*, int, float*, cudaStream_t);
template rh_status launch_ttm<float, double>(const ModeView&, const float*, const float*, int, double*, cudaStream_t);
template rh_status launch_ttm<double, double>(const ModeView&, const double*, const double*, int, double*,
                                              cudaStream_t);
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
