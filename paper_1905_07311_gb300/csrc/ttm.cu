// Mode-n product B = G x_n Q^T (Sec. 2.1: Y_(n) = A X_(n) with A = Q^T), the step that
// forms B = Q^T X in Alg. 1 step 3 and the truncated core G <- U_r^T B of Alg. 3 step 6.
//
// With G viewed as (L, I, R) and p = l + L r:
//   B[(p % L) + L ko (p / L) + L c] = sum_i Q[i + I c] G[(p % L) + L I (p / L) + L i],  c < ko.
// The output keeps the layout of G with mode n resized to ko, i.e. it is directly the
// column-major tensor G x_n Q^T.  No unfolding is materialised.
//
// CTA tile: 128 columns p of the unfolding x all ko (<= 64) output rows; the reduction
// over i runs in steps of 32 through shared memory.
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

template <typename T, typename TO, int ELLP, bool KCONTIG>
__global__ void __launch_bounds__(kNT, 2)
    ttm_kernel(const T* __restrict__ G, int64_t L, int64_t I, int64_t R, const T* __restrict__ Q, int ko,
               TO* __restrict__ B) {
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
      if (c < ko && i < I) q = __ldg(Q + i + I * (int64_t)c);
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

  if (KCONTIG) {
    // B[c + ko p]: a row p holds ko contiguous outputs.
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int64_t p = p0 + tp * TM + a;
      if (p >= M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = 4 * tc + b;
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
        const int c = cl + 32 * h;
        if (obase >= 0 && c < ko) B[obase + L * (int64_t)c] = (TO)Gs[cl][swz<T>(cl, pp)];
      }
      __syncthreads();
    }
  }
}

}  // namespace

template <typename T, typename TO>
rh_status launch_ttm(const ModeView& v, const T* G, const T* Q, int ko, TO* B, cudaStream_t st) {
  if (ko < 1 || ko > RH_MAX_ELL) {
    set_error("internal: ttm output width out of range");
    return RH_EINVAL;
  }
  const int64_t M = v.M();
  const int64_t blocks = ceil_div(M, kTP);
  const bool kc = (v.L == 1);
  const int ellp = ell_pad_of(ko);
#define RH_TTM(E, KC) ttm_kernel<T, TO, E, KC><<<(unsigned)blocks, kNT, 0, st>>>(G, v.L, v.I, v.R, Q, ko, B)
  if (ellp == 32) {
    if (kc) RH_TTM(32, true); else RH_TTM(32, false);
  } else {
    if (kc) RH_TTM(64, true); else RH_TTM(64, false);
  }
#undef RH_TTM
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template rh_status launch_ttm<float, float>(const ModeView&, const float*, const float*, int, float*, cudaStream_t);
template rh_status launch_ttm<float, double>(const ModeView&, const float*, const float*, int, double*, cudaStream_t);
template rh_status launch_ttm<double, double>(const ModeView&, const double*, const double*, int, double*,
                                              cudaStream_t);

}  // namespace rh
