// Small dense linear algebra of RandSVD (Alg. 1 steps 2 and 4-5), all on the device:
//
//   orthonormalize  thin QR of the sketch Y (I x ell): CholeskyQR2 in FP64; a Cholesky
//                   pivot below 1e-14 of its diagonal (kappa(Y) beyond ~1e7) raises a
//                   device flag and a single-CTA Householder QR then produces Q.  The
//                   branch is taken on the device, with no host synchronisation.
//   trunc_svd       SVD of B = Q^T G_(n) (ell x M): tall-skinny Householder QR of B^T
//                   (a tree of per-CTA QRs, never the Gram matrix B B^T, so the small
//                   singular values survive), then a one-sided Jacobi SVD of the final
//                   ell x ell triangle R.  B = R^T Q_B^T, so the left singular vectors of
//                   B are the right singular vectors of R, i.e. the accumulated rotations.
//   factor          A_n = Q U_B(:, 1:r) (Alg. 1 step 5).
#include <math.h>

#include <utility>

#include "common.cuh"
#include "dfloat.cuh"
#include "f32x2.cuh"
#include "kernels.cuh"

namespace rh {

// One launch of an Op through emit (direct, or recorded for a grouped launch); returns on failure.
#define RH_EMIT(OP, SITE, SUB, GRID, SMEM, ...)                                                 \
  do {                                                                                        \
    const rh_status rh_emit_s_ = emit<OP>(SITE, SUB, dim3(GRID), SMEM, st, typename OP::Args{__VA_ARGS__}); \
    if (rh_emit_s_ != RH_OK) return rh_emit_s_;                                               \
  } while (0)

namespace {

// Asynchronous global -> shared copies (cp.async): 4 or 16 bytes, zero-filled when !ok.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool ok) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x a multiple of 32 (<= 1024); every thread gets the result.
template <typename T>
__device__ T block_sum(T v, T* scratch /* >= 33 */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  if (w == 0) {
    T s = lane < nw ? scratch[lane] : T(0);
    s = warp_sum(s);
    if (lane == 0) scratch[32] = s;
  }
  __syncthreads();
  return scratch[32];
}

// ---------------------------------------------------------------------------------
// CholeskyQR2
// ---------------------------------------------------------------------------------
// Gpart[b] = A_b^T A_b over row block b (rows [b rb, b rb + rb)), upper triangle j <= k.
struct GramPartialOp {
  struct Args {
    const double* A;
    int64_t m;
    int n;
    int rb;
    double* Gpart;
    const int32_t* flag;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void GramPartialOp::body(const Grid g, const Args& args) {
  const double* __restrict__ A = args.A;
  int64_t m = args.m;
  int n = args.n;
  int rb = args.rb;
  double* __restrict__ Gpart = args.Gpart;
  const int32_t* __restrict__ flag = args.flag;

  if (flag != nullptr && *flag) return;
  extern __shared__ double As[];  // rb x n, row-major
  const int64_t r0 = (int64_t)g.bx * rb;
  const int rows = (int)(m - r0 < rb ? m - r0 : rb);
  for (int t = threadIdx.x; t < rb * n; t += blockDim.x) {
    const int r = t % rb, c = t / rb;
    As[r * n + c] = (r < rows) ? A[r0 + r + m * (int64_t)c] : 0.0;
  }
  __syncthreads();
  const int npair = n * (n + 1) / 2;
  for (int e = threadIdx.x; e < npair; e += blockDim.x) {
    // e -> (j, k), j <= k, column-major upper triangle (an FP32 estimate of k, corrected exactly;
    // an FP64 square root per entry would cost more than the entry's products on this part)
    int k = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while ((k + 1) * (k + 2) / 2 <= e) ++k;
    while (k * (k + 1) / 2 > e) --k;
    const int j = e - k * (k + 1) / 2;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s = fma(As[r * n + j], As[r * n + k], s);
    Gpart[(int64_t)g.bx * n * n + j + n * k] = s;
  }
}

// C = sum_b Gpart[b], upper triangle.  A block of 256 threads owns 32 consecutive entries: warp w
// sums the partials w, w + 8, ... (eight chains, loads in flight together) and warp 0 adds the eight
// warp sums in a fixed order, so the result does not depend on timing.
struct GramReduceOp {
  struct Args {
    const double* Gpart;
    int nb;
    int n;
    double* C;
    const int32_t* flag;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void GramReduceOp::body(const Grid g, const Args& args) {
  const double* __restrict__ Gpart = args.Gpart;
  int nb = args.nb;
  int n = args.n;
  double* __restrict__ C = args.C;
  const int32_t* __restrict__ flag = args.flag;

  if (flag != nullptr && *flag) return;
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nn = n * n;
  const int e = g.bx * 32 + lane;
  const bool upper = e < nn && (e % n) <= (e / n);
  double s = 0.0;
  if (upper) {
    double ch[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int b = w;
    for (; b + 56 < nb; b += 64) {
#pragma unroll
      for (int q = 0; q < 8; ++q) ch[q] += Gpart[(int64_t)(b + 8 * q) * nn + e];
    }
    for (; b < nb; b += 8) ch[0] += Gpart[(int64_t)b * nn + e];
    s = ((ch[0] + ch[1]) + (ch[2] + ch[3])) + ((ch[4] + ch[5]) + (ch[6] + ch[7]));
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && upper) {
    double t = red[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][lane];
    C[e] = t;
  }
}

// Arithmetic of the small Cholesky factorizations: FP64, or double-float (about 48 bits on the FP32
// pipes) for the FP32 paths.  Both scale the matrix by a power of two first (exact), so that the
// pivot test, done on the leading FP32 part, stays in range.
struct ArithF64 {
  using V = double;
  static constexpr bool kScale = true;   // exact in FP64; keeps the FP32 pivot test in range
  static constexpr float kPivot = 1e-14f;
  __device__ static V from(double d) { return d; }
  __device__ static double to(V v) { return v; }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V fms(V x, V a, V b) { return fma(-a, b, x); }   // x - a b
  __device__ static V rsq(V x) { return rsqrt(x); }
  __device__ static float lead(V x) { return (float)x; }
  __device__ static bool finite(V x) { return isfinite(x); }
};
struct ArithF32 {
  using V = float;
  static constexpr bool kScale = true;
  // used on the Gram matrix of a nearly orthonormal Q_1 (pivots ~1): a small pivot means trouble
  static constexpr float kPivot = 1e-5f;
  __device__ static V from(double d) { return (float)d; }
  __device__ static double to(V v) { return (double)v; }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V fms(V x, V a, V b) { return fmaf(-a, b, x); }
  __device__ static V rsq(V x) { return rsqrtf(x); }
  __device__ static float lead(V x) { return x; }
  __device__ static bool finite(V x) { return isfinite(x); }
};
struct ArithDF {
  using V = dfl::F2;
  static constexpr bool kScale = true;
  static constexpr float kPivot = 1e-14f;
  __device__ static V from(double d) { return dfl::from_double(d); }
  __device__ static double to(V v) { return dfl::to_double(v); }
  __device__ static V mul(V a, V b) { return dfl::mul(a, b); }
  __device__ static V fms(V x, V a, V b) { return dfl::fms(x, a, b); }
  __device__ static V rsq(V x) { return dfl::rsqrt(x); }
  __device__ static float lead(V x) { return x.hi; }
  __device__ static bool finite(V x) { return isfinite(x.hi); }
};

// Trailing-triangle table: entry (i, j), 1 <= i <= j < n, sits at (n-i-1)(n-i)/2 + (j - i), so the
// entries with i > k -- the ones updated at step k -- are the first (n-k-1)(n-k)/2.  Packed i << 8 | j.
__device__ __forceinline__ void build_tri_table(uint16_t* tab, int n) {
  for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
    const int base = (n - i - 1) * (n - i) / 2;
    for (int j = i; j < n; ++j) tab[base + j - i] = (uint16_t)((i << 8) | j);
  }
}

// Largest diagonal entry of C and the power-of-two scale that brings it into [1, 4).  Warp 0;
// result in *scale / *dmax.
template <class Ar>
__device__ __forceinline__ void diag_scale(const double* C, int n, double* scale, int* half_exp, float* dmax,
                                           int* ok) {
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += 32) m = fmax(m, C[k + n * k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      const bool good = m > 0.0 && isfinite(m);
      int e = good ? ilogb(m) : 0;
      e &= ~1;   // even, so that the square root of the scale is a power of two too
      if (!Ar::kScale) e = 0;
      *scale = ldexp(1.0, -e);
      *half_exp = e / 2;
      *dmax = (float)(m * *scale);
      *ok = good ? 1 : 0;
    }
  }
}

constexpr int kCholThreads = 512;
constexpr int kCholPer = 4096 / kCholThreads;   // matrix elements per thread in the load / store passes

size_t chol_smem(int n, size_t velem) {
  const size_t a = velem * (size_t)(n | 1) * n;
  return ((a + 15) & ~size_t(15)) + sizeof(uint16_t) * (size_t)n * n / 2 + 16;
}

// Cholesky C = R^T R (R upper) in one CTA; also writes rdiag = 1 / diag(R).  flag <- 1 on a
// pivot <= kPivot C_kk (1e-14 in FP64 / double-float, 1e-5 in FP32) or not finite: CholeskyQR2 is then not accurate enough and the Householder
// branch takes over.  Right-looking on the unscaled Schur complement S (S_kj = R_kk R_kj after step
// k - 1): S_ij -= S_ki S_kj / S_kk for k < i <= j, one barrier per step.  Thread 0 updates the next
// pivot S_{k+1,k+1} first and prepares its 1 / sqrt; warps 1.. share the remaining
// entries of the trailing triangle through the table (no idle predicated work).
template <class Ar>
struct CholOp {
  struct Args {
    const double* C;
    int n;
    double* R;
    double* rdiag;
    int32_t* flag;
    double skip_tol;   // > 0: *flag <- 2 and no factorization when max |C - I| <= skip_tol
  };
  static constexpr int kThreads = kCholThreads, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <class Ar>
__device__ __forceinline__ void CholOp<Ar>::body(const Grid g, const Args& args) {
  const double* __restrict__ C = args.C;
  int n = args.n;
  double* __restrict__ R = args.R;
  double* __restrict__ rdiag = args.rdiag;
  int32_t* __restrict__ flag = args.flag;

  if (*flag) return;
  if (args.skip_tol > 0.0) {
    // the Gram matrix of an already orthonormal basis: the second CholeskyQR pass is not needed
    __shared__ int far_s;
    if (threadIdx.x == 0) far_s = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      if (i <= j && fabs(C[e] - (i == j ? 1.0 : 0.0)) > args.skip_tol) far_s = 1;
    }
    __syncthreads();
    if (!far_s) {
      if (threadIdx.x == 0) *flag = 2;
      return;
    }
  }
  using V = typename Ar::V;
  extern __shared__ __align__(16) unsigned char chol_raw[];
  const int ld = n | 1;   // odd leading dimension: 8-byte accesses along a row hit distinct banks
  V* S = reinterpret_cast<V*>(chol_raw);
  uint16_t* tab = reinterpret_cast<uint16_t*>(chol_raw + ((sizeof(V) * ld * n + 15) & ~size_t(15)));
  __shared__ V rinv[RH_MAX_ELL];
  __shared__ float cdiag[RH_MAX_ELL];
  __shared__ double scale_s;
  __shared__ float dmax_s;
  __shared__ int hexp_s, ok_s, bad;
  const int t = threadIdx.x;
  diag_scale<Ar>(C, n, &scale_s, &hexp_s, &dmax_s, &ok_s);
  build_tri_table(tab, n);
  __syncthreads();
  const double sc = scale_s;
  {
    double c[kCholPer];
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {   // all loads first
      const int e = t + kCholThreads * q;
      c[q] = (e < n * n && (e % n) <= (e / n)) ? C[e] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {
      const int e = t + kCholThreads * q;
      if (e < n * n) S[(e % n) + ld * (e / n)] = Ar::from(c[q] * sc);
    }
  }
  for (int k = t; k < n; k += blockDim.x) cdiag[k] = (float)(C[k + n * k] * sc);
  __syncthreads();
  if (t == 0) {
    bad = 0;
    const V d = S[0];
    if (!(Ar::lead(d) > 0.0f) || !Ar::finite(d))
      bad = 1;
    else
      rinv[0] = Ar::rsq(d);
  }
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    if (bad) break;  // uniform: read after the barrier
    const V ri = rinv[k];
    const V ri2 = Ar::mul(ri, ri);
    if (t == 0) {
      const V a = S[k + ld * (k + 1)];
      const V v = Ar::fms(S[(k + 1) + ld * (k + 1)], Ar::mul(a, ri2), a);
      S[(k + 1) + ld * (k + 1)] = v;
      if (!(Ar::lead(v) > Ar::kPivot * cdiag[k + 1]) || !Ar::finite(v))
        bad = 1;
      else
        rinv[k + 1] = Ar::rsq(v);
    } else if (t >= 32) {
      // warps 1.. share the trailing triangle, two table entries per pass, operands read before
      // either result is written; warp 0 is left to thread 0's pivot chain (lanes of one warp that
      // took both paths would run them one after the other)
      const int T = (n - k - 1) * (n - k) / 2;
      const int stride = blockDim.x - 32;
      for (int e = t - 32; e < T; e += 2 * stride) {
        const int e2 = e + stride;
        const int ij = tab[e];
        const int ij2 = e2 < T ? tab[e2] : ij;
        const int i = ij >> 8, j = ij & 255, i2 = ij2 >> 8, j2 = ij2 & 255;
        const V x1 = S[i + ld * j], a1 = S[k + ld * i], b1 = S[k + ld * j];
        const V x2 = S[i2 + ld * j2], a2 = S[k + ld * i2], b2 = S[k + ld * j2];
        const V v1 = Ar::fms(x1, Ar::mul(a1, ri2), b1);
        const V v2 = Ar::fms(x2, Ar::mul(a2, ri2), b2);
        if (!(i == k + 1 && j == k + 1)) S[i + ld * j] = v1;
        if (e2 < T && !(i2 == k + 1 && j2 == k + 1)) S[i2 + ld * j2] = v2;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (t == 0) *flag = 1;
    return;
  }
  // R = S diag(rinv) / sqrt(scale), rdiag = rinv sqrt(scale): exact powers of two
  const double up = ldexp(1.0, hexp_s), down = ldexp(1.0, -hexp_s);
  {
    double r[kCholPer];
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {
      const int e = t + kCholThreads * q;
      const int j = e % n, k = e / n;
      r[q] = (e < n * n && j <= k) ? Ar::to(Ar::mul(S[j + ld * k], rinv[j])) * up : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {
      const int e = t + kCholThreads * q;
      if (e < n * n) R[e] = r[q];
    }
  }
  for (int k = t; k < n; k += blockDim.x) rdiag[k] = Ar::to(rinv[k]) * down;
}

// Out = A R^{-1} row by row (forward substitution on x^T R = a^T); one warp per row, the
// diagonal applied through its precomputed reciprocals.
template <typename T>
struct TrsmRowsOp {
  struct Args {
    const T* A;
    int64_t m;
    int n;
    const double* R;
    const double* rdiag;
    T* Out;
    const int32_t* flag;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void TrsmRowsOp<T>::body(const Grid g, const Args& args) {
  const T* __restrict__ A = args.A;
  int64_t m = args.m;
  int n = args.n;
  const double* __restrict__ R = args.R;
  const double* __restrict__ rdiag = args.rdiag;
  T* __restrict__ Out = args.Out;
  const int32_t* __restrict__ flag = args.flag;

  if (*flag) return;
  extern __shared__ __align__(16) unsigned char trsm_raw[];
  T* Rs = reinterpret_cast<T*>(trsm_raw);   // n x n column-major (odd leading dimension ld), then n reciprocals
  const int ld = n | 1;           // lanes read a row of R: an odd stride keeps the banks distinct
  T* rd = Rs + ld * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Rs[(e % n) + ld * (e / n)] = (T)R[e];
  for (int e = threadIdx.x; e < n; e += blockDim.x) rd[e] = (T)rdiag[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)g.gx * (blockDim.x >> 5);
  for (int64_t row = (int64_t)g.bx * (blockDim.x >> 5) + (threadIdx.x >> 5); row < m; row += warps) {
    T y0 = lane < n ? A[row + m * lane] : T(0);
    T y1 = lane + 32 < n ? A[row + m * (lane + 32)] : T(0);
    for (int c = 0; c < n; ++c) {
      const T xc = __shfl_sync(0xffffffffu, c < 32 ? y0 : y1, c & 31) * rd[c];
      if (lane == (c & 31)) {
        if (c < 32) y0 = xc; else y1 = xc;
      }
      if (lane > c && lane < n) y0 -= xc * Rs[c + ld * lane];
      if (lane + 32 > c && lane + 32 < n) y1 -= xc * Rs[c + ld * (lane + 32)];
    }
    if (lane < n) Out[row + m * lane] = y0;
    if (lane + 32 < n) Out[row + m * (lane + 32)] = y1;
  }
}

// Householder QR of Y (m x n) with explicit thin Q, one CTA; runs only when *flag is set
// (or always when flag == nullptr).  W is an m x n FP64 scratch copy; beta has n slots.
struct HouseholderQOp {
  struct Args {
    const double* Y;
    int64_t m;
    int n;
    double* W;
    double* beta;
    double* Q;
    const int32_t* flag;
    int32_t* info;
  };
  static constexpr int kThreads = 1024, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void HouseholderQOp::body(const Grid g, const Args& args) {
  const double* __restrict__ Y = args.Y;
  int64_t m = args.m;
  int n = args.n;
  double* __restrict__ W = args.W;
  double* __restrict__ beta = args.beta;
  double* __restrict__ Q = args.Q;
  const int32_t* __restrict__ flag = args.flag;
  int32_t* __restrict__ info = args.info;

  const bool run = (flag == nullptr) || (*flag == 1);   // 2: the second pass was skipped
  if (info != nullptr && threadIdx.x == 0) *info = (*info & ~1) | (run ? 1 : 0);
  if (!run) return;
  __shared__ double scratch[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t e = threadIdx.x; e < m * n; e += blockDim.x) W[e] = Y[e];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double* x = W + m * (int64_t)k;
    double s = 0.0;
    for (int64_t i = k + threadIdx.x; i < m; i += blockDim.x) s += x[i] * x[i];
    s = block_sum(s, scratch);
    const double alpha = x[k];
    const double nrm = sqrt(s);
    double b = 0.0;
    if (nrm > 0.0) {
      const double sg = alpha >= 0.0 ? 1.0 : -1.0;
      b = 1.0 / (nrm * (nrm + fabs(alpha)));
      __syncthreads();
      if (threadIdx.x == 0) x[k] = alpha + sg * nrm;  // v = x + sign(alpha) ||x|| e_1
    }
    __syncthreads();
    if (threadIdx.x == 0) beta[k] = b;
    // apply H = I - b v v^T to columns j > k
    for (int j = k + 1 + w; j < n; j += nw) {
      double* y = W + m * (int64_t)j;
      double d = 0.0;
      for (int64_t i = k + lane; i < m; i += 32) d += x[i] * y[i];
      d = warp_sum(d) * b;
      for (int64_t i = k + lane; i < m; i += 32) y[i] -= d * x[i];
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{n-1} [I_n; 0], accumulated backwards
  for (int64_t e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int64_t i = e % m, j = e / m;
    Q[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    const double* v = W + m * (int64_t)k;
    const double b = beta[k];
    if (b != 0.0) {
      for (int j = k + w; j < n; j += nw) {
        double* q = Q + m * (int64_t)j;
        double d = 0.0;
        for (int64_t i = k + lane; i < m; i += 32) d += v[i] * q[i];
        d = warp_sum(d) * b;
        for (int64_t i = k + lane; i < m; i += 32) q[i] -= d * v[i];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Tall-skinny QR (R only) of B^T and the one-sided Jacobi SVD
// ---------------------------------------------------------------------------------
// In-shared-memory Householder triangularisation of a rows x n block (column-major,
// leading dimension ld, which the callers keep odd so that a warp reading one row of 32
// consecutive columns hits 32 different banks), leaving R in the upper triangle.
// Per column k: the norm of the trailing part of column k (block reduction); then
// w_j = v^T A(k:, j) for all j > k with the columns spread over the lanes and the rows
// over CW-wide thread groups (partials reduced through shared memory); then the rank-1
// update A(k:, j) -= beta w_j v with the same thread layout.  ``red`` holds >= nt + 64
// elements of T.
template <typename T>
__device__ void smem_householder_r(T* A, int rows, int n, int ld, T* scratch, T* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int CW = (n <= 32) ? 32 : 64;        // column slots
  const int NCH = nt / CW;                    // row groups
  const int jj = tid % CW, ch = tid / CW;
  const int kmax = min(rows, n);
  T* wv = red + nt;                            // CW scaled dot products
  for (int k = 0; k < kmax; ++k) {
    T* x = A + (int64_t)ld * k;
    T s = T(0);
    for (int i = k + tid; i < rows; i += nt) s += x[i] * x[i];
    s = block_sum(s, scratch);
    const T alpha = x[k];
    const T nrm = sqrt(s);
    if (nrm == T(0)) continue;  // uniform
    const T sg = alpha >= T(0) ? T(1) : T(-1);
    const T b = T(1) / (nrm * (nrm + fabs(alpha)));
    __syncthreads();
    if (tid == 0) x[k] = alpha + sg * nrm;     // v = x + sign(alpha) ||x|| e_1
    __syncthreads();
    const int j = k + 1 + jj;
    const bool active = j < n;
    const T* y = A + (int64_t)ld * (active ? j : k);
    T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
    int i = k + ch;
    if (active) {
      for (; i + 3 * NCH < rows; i += 4 * NCH) {
        d0 += x[i] * y[i];
        d1 += x[i + NCH] * y[i + NCH];
        d2 += x[i + 2 * NCH] * y[i + 2 * NCH];
        d3 += x[i + 3 * NCH] * y[i + 3 * NCH];
      }
      for (; i < rows; i += NCH) d0 += x[i] * y[i];
    }
    red[ch * CW + jj] = (d0 + d1) + (d2 + d3);
    __syncthreads();
    if (tid < CW) {
      T w = T(0);
      for (int c = 0; c < NCH; ++c) w += red[c * CW + tid];
      wv[tid] = w * b;
    }
    __syncthreads();
    if (active) {
      const T w = wv[jj];
      T* yy = A + (int64_t)ld * j;
      for (int r = k + ch; r < rows; r += NCH) yy[r] -= w * x[r];
    }
    __syncthreads();
    if (tid == 0) x[k] = -sg * nrm;            // R_kk
    __syncthreads();
  }
}

// Level 0: block b holds rows [b rows0, ...) of B^T, with B^T[p, c] = B[(p % L) + L n (p / L) + L c].
// CTAs loop over the blocks (the grid is capped), so a launch whose gate is off costs little.
template <typename T>
struct TsqrLeafOp {
  struct Args {
    const T* B;
    int64_t L;
    int64_t R;
    int n;
    int rows0;
    int ld;
    T* Rout;
    const int32_t* gate;
  };
  static constexpr int kThreads = 1024, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void TsqrLeafOp<T>::body(const Grid g, const Args& args) {
  const T* __restrict__ B = args.B;
  int64_t L = args.L;
  int64_t R = args.R;
  int n = args.n;
  int rows0 = args.rows0;
  int ld = args.ld;
  T* __restrict__ Rout = args.Rout;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* red = A + (int64_t)ld * n;
  __shared__ T scratch[33];
  const int64_t M = L * R;
  const int64_t nblk = (M + rows0 - 1) / rows0;
  for (int64_t blk = g.bx; blk < nblk; blk += g.gx) {
    const int64_t p0 = blk * rows0;
    const int rows = (int)(M - p0 < rows0 ? M - p0 : rows0);
    __syncthreads();
    if (L == 1) {
      // B^T rows are contiguous: element (r, c) at n (p0 + r) + c; read the block linearly
      const T* src = B + n * p0;
      for (int e = threadIdx.x; e < rows0 * n; e += blockDim.x) {
        const int r = e / n, c = e % n;
        A[r + (int64_t)ld * c] = (r < rows) ? src[e] : T(0);
      }
    } else {
      for (int r = threadIdx.x; r < rows0; r += blockDim.x) {
        const int64_t p = p0 + r;
        if (r < rows) {
          const int64_t base = (p % L) + L * (int64_t)n * (p / L);
          for (int c = 0; c < n; ++c) A[r + (int64_t)ld * c] = B[base + L * c];
        } else {
          for (int c = 0; c < n; ++c) A[r + (int64_t)ld * c] = T(0);
        }
      }
    }
    __syncthreads();
    smem_householder_r(A, max(rows, n), n, ld, scratch, red);
    T* o = Rout + blk * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int j = e % n, k = e / n;
      o[e] = (j <= k && j < rows) ? A[j + (int64_t)ld * k] : T(0);
    }
  }
}

// Higher level: block b stacks R's [b fan, b fan + fan) (each n x n) and re-triangularises.
template <typename T>
struct TsqrMergeOp {
  struct Args {
    const T* Rin;
    int64_t nin;
    int n;
    int fan;
    int ld;
    T* Rout;
    const int32_t* gate;
  };
  static constexpr int kThreads = 1024, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void TsqrMergeOp<T>::body(const Grid g, const Args& args) {
  const T* __restrict__ Rin = args.Rin;
  int64_t nin = args.nin;
  int n = args.n;
  int fan = args.fan;
  int ld = args.ld;
  T* __restrict__ Rout = args.Rout;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* red = A + (int64_t)ld * n;
  __shared__ T scratch[33];
  const int64_t nout = (nin + fan - 1) / fan;
  for (int64_t blk = g.bx; blk < nout; blk += g.gx) {
    const int64_t b0 = blk * fan;
    const int cnt = (int)(nin - b0 < fan ? nin - b0 : fan);
    const int rows = cnt * n;
    __syncthreads();
    for (int e = threadIdx.x; e < ld * n; e += blockDim.x) {
      const int r = e % ld, c = e / ld;
      const int q = r / n, j = r % n;
      A[r + (int64_t)ld * c] = (q < cnt && r < fan * n) ? Rin[(b0 + q) * n * n + j + n * c] : T(0);
    }
    __syncthreads();
    smem_householder_r(A, rows, n, ld, scratch, red);
    T* o = Rout + blk * n * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int j = e % n, k = e / n;
      o[e] = (j <= k) ? A[j + (int64_t)ld * k] : T(0);
    }
  }
}

// ---- FP32 tall-skinny QR with one row per thread ----------------------------------------------
// Householder QR of a block of up to 256 rows of B^T (n <= NC columns), every row held in the
// registers of one thread (the column loop is unrolled, so register indices are static).  Per
// column k: ||x||^2 of column k from the diagonal down (warp shuffles, 8 warp partials), the
// reflector v = x + sign(x_k) ||x|| e_k, the products v_r a_r[j] staged in shared memory and summed
// by columns (segments of NC rows, then the segment partials), and the update
// a_r[j] -= beta w_j v_r with beta = 1 / (||x|| (||x|| + |x_k|)).  Four barriers per column, all
// with 256 threads.  Leaf blocks read 256 rows of B^T from the (L, n, R) view of B; merge blocks
// stack ``fan`` upper triangles (n x n, column-major) of the previous level, fan n <= 256.
constexpr int kRowsQR = 256;

// ---- FP32 tall-skinny QR, 256-row blocks in shared memory -------------------------------------
// Householder QR of a block of up to 256 rows of B^T (n <= NC columns) held row-major in shared
// memory (odd leading dimension: conflict-free row and column access).  Per column k: ||x||^2 of
// column k from the diagonal down (warp shuffles, 8 warp partials), the reflector
// v = x + sign(x_k) ||x|| e_k, the products w_j = sum_r v_r A(r, j) summed by (segment, column)
// threads (256 / NC segments of NC rows) and then over segments, and the row update
// A(r, j) -= beta w_j v_r with beta = 1 / (||x|| (||x|| + |x_k|)).  Four barriers per column, all
// loops rolled (small code).  Leaf blocks read 256 rows of B^T from the (L, n, R) view of B; merge
// blocks stack ``fan`` upper triangles (n x n, column-major) of the previous level, fan n <= 256.
template <int NC>
struct TsqrRowsOp {
  struct Args {
    const float* B;
    int64_t L;
    int64_t R;
    int n;
    const float* Rin;
    int64_t nin;
    int fan;
    float* Rout;
    const int32_t* gate;
  };
  static constexpr int kThreads = kRowsQR, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <int NC>
__device__ __forceinline__ void TsqrRowsOp<NC>::body(const Grid g, const Args& args) {
  const float* __restrict__ B = args.B;
  int64_t L = args.L;
  int64_t R = args.R;
  int n = args.n;
  const float* __restrict__ Rin = args.Rin;
  int64_t nin = args.nin;
  int fan = args.fan;
  float* __restrict__ Rout = args.Rout;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate == 0) return;
  constexpr int LD = NC + 1;
  constexpr int SEG = kRowsQR / NC;   // row segments of the column sums, NC rows each
  extern __shared__ float qsm[];
  float* A = qsm;                      // [256][LD]
  float* Vs = A + kRowsQR * LD;        // [256]: v
  float* Sg = Vs + kRowsQR;            // [SEG][NC]
  float* Wv = Sg + SEG * NC;           // [NC]: beta w_j
  __shared__ float red[kRowsQR / 32];
  __shared__ float sh_alpha;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int cj = t % NC, cseg = t / NC;
  const bool leaf = (Rin == nullptr);
  const int64_t M = L * R;
  const int64_t nblk = leaf ? (M + kRowsQR - 1) / kRowsQR : (nin + fan - 1) / fan;
  float* Arow = A + t * LD;
  for (int64_t blk = g.bx; blk < nblk; blk += g.gx) {
    __syncthreads();   // shared buffers are free (previous block)
    if (leaf) {
      const int64_t p0 = blk * kRowsQR;
      const int rows = (int)(M - p0 < kRowsQR ? M - p0 : kRowsQR);
      if (L == 1) {
        // the block's rows of B^T are n consecutive floats each: a coalesced copy
        const float* src = B + (int64_t)n * p0;
        for (int e = t; e < kRowsQR * n; e += kRowsQR) {
          const int r = e / n, c = e - r * n;
          A[r * LD + c] = (r < rows) ? src[e] : 0.0f;
        }
      } else {
        const bool ok = t < rows;
        const int64_t p = p0 + t;
        const int64_t base = ok ? (p % L) + L * (int64_t)n * (p / L) : 0;
        for (int c = 0; c < n; ++c) Arow[c] = ok ? B[base + L * c] : 0.0f;
      }
    } else {
      const int64_t b0 = blk * fan;
      const int cnt = (int)(nin - b0 < fan ? nin - b0 : fan);
      const int q = t / n, j = t - q * n;
      const bool ok = q < cnt;
      const float* src = Rin + (b0 + (ok ? q : 0)) * (int64_t)n * n + j;
      for (int c = 0; c < n; ++c) Arow[c] = ok ? src[(int64_t)n * c] : 0.0f;
    }
    for (int k = 0; k < n; ++k) {
      __syncthreads();   // the previous column's updates are visible
      const float xk = (t >= k) ? Arow[k] : 0.0f;
      float sq = xk * xk;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) red[wid] = sq;
      if (t == k) sh_alpha = xk;
      __syncthreads();
      float ss = 0.0f;
#pragma unroll
      for (int w = 0; w < kRowsQR / 32; ++w) ss += red[w];
      const float alpha = sh_alpha;
      const float nrm = sqrtf(ss);
      if (!(nrm > 0.0f)) continue;   // uniform: every thread sums the same partials
      const float sg = alpha >= 0.0f ? 1.0f : -1.0f;
      const float beta = 1.0f / (nrm * (nrm + fabsf(alpha)));
      const float v = (t == k) ? alpha + sg * nrm : xk;
      Vs[t] = v;
      __syncthreads();
      if (cj > k && cj < n) {
        const int r0 = cseg * NC;
        // v vanishes above the diagonal; eight independent chains keep the loads in flight
        const int rb = r0 > k ? r0 : k;
        float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        int r = rb;
        for (; r + 7 < r0 + NC; r += 8) {
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[q] = fmaf(Vs[r + q], A[(r + q) * LD + cj], acc[q]);
        }
        for (; r < r0 + NC; ++r) acc[0] = fmaf(Vs[r], A[r * LD + cj], acc[0]);
        Sg[cseg * NC + cj] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
      }
      __syncthreads();
      if (t > k && t < n) {
        float w = 0.0f;
        for (int q = 0; q < SEG; ++q) w += Sg[q * NC + t];   // every segment wrote its partial
        Wv[t] = beta * w;
      }
      __syncthreads();
      if (t >= k) {
#pragma unroll 4
        for (int j = k + 1; j < n; ++j) Arow[j] = fmaf(-Wv[j], v, Arow[j]);
      }
      if (t == k)
        Arow[k] = -sg * nrm;
      else if (t > k)
        Arow[k] = 0.0f;
    }
    __syncthreads();
    if (t < n) {
      float* o = Rout + blk * (int64_t)n * n;
      for (int c = 0; c < n; ++c) o[t + (int64_t)n * c] = (c >= t) ? A[t * LD + c] : 0.0f;
    }
  }
}

size_t tsqr_rows_smem(int nc) {
  return sizeof(float) * ((size_t)kRowsQR * (nc + 1) + (size_t)kRowsQR + (size_t)kRowsQR + nc);
}

// R of B^T (M x n FP32) by levels of tsqr_rows_kernel; buf0 / buf1 hold ceil(M / 256) and
// ceil(M / 256 / fan) n x n triangles; returns the final triangle's buffer in *out.
rh_status launch_tsqr_rows(const float* B, int64_t L, int64_t R, int n, float* buf0, float* buf1,
                           const int32_t* gate, float** out, cudaStream_t st, int site = SITE_OTHER) {
  if (n < 1 || n > 64) {
    set_error("tall-skinny QR: n must be in [1, 64]");
    return RH_EUNSUPPORTED;
  }
  const int nc = n <= 32 ? 32 : 64;
  const size_t smem = tsqr_rows_smem(nc);
  const int64_t cap = 4 * (int64_t)num_sms();
  const int fan = kRowsQR / n;
  int64_t cnt = ceil_div(L * R, kRowsQR);
  auto level = [&](int sub, int64_t blocks, const float* Bs, int64_t Ls, int64_t Rs, const float* Rin, int64_t nin,
                   float* Rout) -> rh_status {
    const dim3 grid((unsigned)std::min<int64_t>(blocks, cap));
    if (nc == 32)
      return emit<TsqrRowsOp<32>>(site, sub, grid, smem, st,
                                  TsqrRowsOp<32>::Args{Bs, Ls, Rs, n, Rin, nin, fan, Rout, gate});
    return emit<TsqrRowsOp<64>>(site, sub, grid, smem, st, TsqrRowsOp<64>::Args{Bs, Ls, Rs, n, Rin, nin, fan, Rout, gate});
  };
  rh_status s = level(0, cnt, B, L, R, nullptr, 0, buf0);
  if (s != RH_OK) return s;
  float* cur = buf0;
  float* nxt = buf1;
  for (int lv = 1; cnt > 1; ++lv) {
    const int64_t nout = ceil_div(cnt, fan);
    if ((s = level(lv, nout, nullptr, 1, 1, cur, cnt, nxt)) != RH_OK) return s;
    cnt = nout;
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  *out = cur;
  return RH_OK;
}

// One-sided Jacobi on the columns of R (n x n, n <= 64): R V = U S.  Writes Ub = V with columns
// sorted by decreasing singular value and sv (both FP64).
// Schedule: np = n rounded up to even "players" (a zero dummy when n is odd, which never
// rotates); warp w owns the players at circle positions w and np-1-w.  In every round each warp
// rotates its pair, then the players at positions 1..np-1 move one place round the circle
// (position 0 stays), which pairs every two players once per sweep of np-1 rounds and brings
// every player back to its starting position at the end of the sweep.  Columns travel between
// warps through two alternating shared-memory buffers, so a round needs a single barrier; lane l
// keeps entries l and l + 32 of a column and of its V column as one 4-vector.
// Each player carries its squared norm: a round computes only the inner product g = a^T b and
// updates the norms of the rotated pair in closed form (a'^2 = a^2 - t g, b'^2 = b^2 + t g);
// the norms are re-measured at the start of every sweep.  A rotation is applied when
// |g| > tol |a| |b|, tol = 8 max(n, 8) eps: the computed inner product carries a rounding error
// up to n eps |a| |b|, so a threshold at that level is never met.  The rotation
// t = sign(z) / (|z| + sqrt(1 + z^2)), z = (b^2 - a^2) / (2 g), c = 1 / sqrt(1 + t^2), s = c t is
// formed in T.
template <typename T>
struct alignas(4 * sizeof(T)) JacobiQuad {
  T x0, x1, v0, v1;
};

__device__ __forceinline__ float jacobi_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jacobi_rsqrt(double x) { return 1.0 / sqrt(x); }

template <typename T>
struct JacobiSvdOp {
  struct Args {
    const T* Rin;
    int n;
    double* Ub;
    double* sv;
    const int32_t* gate;
    int32_t want;
    const int32_t* piv;   // non-NULL: preconditioned mode (see below)
  };
  static constexpr int kThreads = 1024, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void JacobiSvdOp<T>::body(const Grid g, const Args& args) {
  const T* __restrict__ Rin = args.Rin;
  int n = args.n;
  double* __restrict__ Ub = args.Ub;
  double* __restrict__ sv = args.sv;
  const int32_t* __restrict__ gate = args.gate;
  int32_t want = args.want;
  const int32_t* __restrict__ piv = args.piv;

  if (gate != nullptr && *gate != want) return;
  using Q4 = JacobiQuad<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int np = (n + 1) & ~1;
  const int half = np / 2;
  Q4* buf0 = reinterpret_cast<Q4*>(smem_raw);   // [position][lane]
  Q4* buf1 = buf0 + (size_t)np * 32;
  __shared__ T nrm2[2][RH_MAX_ELL];
  __shared__ T sig[RH_MAX_ELL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < np * 32; e += blockDim.x) {
    const int q = e >> 5, l = e & 31;
    Q4 z;
    const bool col = q < n;
    // preconditioned mode: the players are the rows of Rin (the columns of X = Rin^T)
    const int64_t s0 = piv ? q + (int64_t)n * l : l + (int64_t)n * q;
    const int64_t s1 = piv ? q + (int64_t)n * (l + 32) : l + 32 + (int64_t)n * q;
    z.x0 = (col && l < n) ? Rin[s0] : T(0);
    z.x1 = (col && l + 32 < n) ? Rin[s1] : T(0);
    z.v0 = (col && l == q) ? T(1) : T(0);
    z.v1 = (col && l + 32 == q) ? T(1) : T(0);
    buf0[e] = z;
  }
  __syncthreads();
  const T tol = T(8 * (n > 8 ? n : 8)) * ((sizeof(T) == 4) ? T(5.9604645e-8) : T(1.1102230246251565e-16));
  // fixed circle positions of this warp and where their players move after a round
  const int qa = w, qb = np - 1 - w;
  const int na = (qa == 0) ? 0 : (qa == np - 1 ? 1 : qa + 1);
  const int nb = (qb == 0) ? 0 : (qb == np - 1 ? 1 : qb + 1);
  int cur = 0;
  // columns whose norm is below n u ||R||_F are rounding noise: they cannot be made orthogonal to
  // the relative tolerance, so pairs involving one are not rotated (otherwise a spectrum that
  // reaches the rounding level, like the Hilbert tensor's, never meets the stopping test; a floor
  // as high as the tolerance itself was measured to move the leading subspace of the 200^3
  // Hilbert tensor by 1.6e-10)
  __shared__ T floor2_s, abs2_s;
  for (int sweep = 0; sweep < 40; ++sweep) {
    {
      const Q4* src = cur ? buf1 : buf0;
      for (int q = w; q < np; q += nw) {
        const Q4 z = src[q * 32 + lane];
        const T a = warp_sum(z.x0 * z.x0 + z.x1 * z.x1);
        if (lane == 0) nrm2[cur][q] = a;
      }
      __syncthreads();
      if (sweep == 0 && threadIdx.x == 0) {
        T fro2 = T(0);
        for (int q = 0; q < n; ++q) fro2 += nrm2[cur][q];
        const T u = (sizeof(T) == 4) ? T(5.9604645e-8) : T(1.1102230246251565e-16);
        const T nu = T(n) * u;
        floor2_s = nu * nu * fro2;
        abs2_s = T(16) * u * u * fro2;   // (4 u ||R||_F)^2
      }
      __syncthreads();
    }
    const T floor2 = floor2_s, abs2 = abs2_s;
    int rotated = 0;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      const Q4* src = cur ? buf1 : buf0;
      Q4* dst = cur ? buf0 : buf1;
      if (w < half) {
        Q4 A = src[qa * 32 + lane];
        Q4 Bq = src[qb * 32 + lane];
        T al = nrm2[cur][qa], be = nrm2[cur][qb];
        const T g = warp_sum(A.x0 * Bq.x0 + A.x1 * Bq.x1);
        // the decision and the rotation are the same for the whole warp: lane 0 evaluates them
        // (divisions and square roots are few and slow in FP64 on this part) and broadcasts.
        // Preconditioned mode: the test is on squares (no square roots), and a pair whose inner
        // product is within the absolute rounding noise 4 u ||R|| min(|a|, |b|) of the rotated
        // columns is left alone (such columns cannot be made orthogonal to the relative tolerance;
        // for a column with |a| >= 1e-5 ||R|| the coupling left is below 4.4e-11)
        T t = T(0), c = T(1), sn = T(0);
        int rot = 0;
        const T mn = al < be ? al : be;
        const bool go = piv ? (g * g > tol * tol * al * be && g * g > abs2 * mn)
                            : (g != T(0) && fabs(g) * jacobi_rsqrt(al) * jacobi_rsqrt(be) > tol);
        if (lane == 0 && mn > floor2 && go) {
          const T zeta = (be - al) / (T(2) * g);
          const T az = fabs(zeta);
          const T tm = az < T(1e18) ? T(1) / (az + sqrt(fma(az, az, T(1)))) : T(0.5) / az;
          t = zeta < T(0) ? -tm : tm;
          c = jacobi_rsqrt(fma(t, t, T(1)));
          sn = c * t;
          rot = 1;
        }
        rot = __shfl_sync(0xffffffffu, rot, 0);
        if (rot) {
          t = __shfl_sync(0xffffffffu, t, 0);
          c = __shfl_sync(0xffffffffu, c, 0);
          sn = __shfl_sync(0xffffffffu, sn, 0);
          T u;
          u = A.x0; A.x0 = c * u - sn * Bq.x0; Bq.x0 = sn * u + c * Bq.x0;
          u = A.x1; A.x1 = c * u - sn * Bq.x1; Bq.x1 = sn * u + c * Bq.x1;
          if (piv == nullptr) {   // the preconditioned mode outputs the columns, not V
            u = A.v0; A.v0 = c * u - sn * Bq.v0; Bq.v0 = sn * u + c * Bq.v0;
            u = A.v1; A.v1 = c * u - sn * Bq.v1; Bq.v1 = sn * u + c * Bq.v1;
          }
          al = al - t * g;
          be = be + t * g;
          rotated = 1;
        }
        dst[na * 32 + lane] = A;
        dst[nb * 32 + lane] = Bq;
        if (lane == 0) {
          nrm2[cur ^ 1][na] = al;
          nrm2[cur ^ 1][nb] = be;
        }
      }
      cur ^= 1;
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  // every sweep ends with player q at position q
  const Q4* fin = cur ? buf1 : buf0;
  for (int q = w; q < np; q += nw) {
    const Q4 z = fin[q * 32 + lane];
    const T s = warp_sum(z.x0 * z.x0 + z.x1 * z.x1);
    if (lane == 0) sig[q] = (q < n) ? sqrt(s) : T(-1);
  }
  __syncthreads();
  if (piv == nullptr) {
    for (int q = w; q < n; q += nw) {
      int rank = 0;
      for (int k = 0; k < n; ++k) rank += (sig[k] > sig[q]) || (sig[k] == sig[q] && k < q);
      const Q4 z = fin[q * 32 + lane];
      if (lane == 0) sv[rank] = (double)sig[q];
      if (lane < n) Ub[lane + n * rank] = (double)z.v0;
      if (lane + 32 < n) Ub[lane + 32 + n * rank] = (double)z.v1;
    }
    return;
  }
  // Preconditioned mode: X V = U' S with X = R2^T, so the left singular vectors are the rotated
  // columns divided by their norms.  They are staged in rank order in the free buffer, made
  // orthonormal by one modified Gram-Schmidt pass in that order (a no-op up to rounding for the
  // converged columns; columns at the rounding floor are completed with unit vectors), and row l
  // is written to row piv[l] (U_B = Pi U').
  T* Us = reinterpret_cast<T*>(cur ? buf0 : buf1);   // [rank][64]
  for (int q = w; q < n; q += nw) {
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += (sig[k] > sig[q]) || (sig[k] == sig[q] && k < q);
    const Q4 z = fin[q * 32 + lane];
    const T inv = sig[q] > T(0) ? T(1) / sig[q] : T(0);
    if (lane == 0) sv[rank] = (double)sig[q];
    Us[rank * 64 + lane] = z.x0 * inv;
    Us[rank * 64 + lane + 32] = z.x1 * inv;
  }
  __syncthreads();
  if (w == 0) {
    for (int k = 0; k < n; ++k) {
      T u0 = Us[k * 64 + lane], u1 = Us[k * 64 + lane + 32];
      for (int j = 0; j < k; ++j) {
        const T d = warp_sum(Us[j * 64 + lane] * u0 + Us[j * 64 + lane + 32] * u1);
        u0 -= d * Us[j * 64 + lane];
        u1 -= d * Us[j * 64 + lane + 32];
      }
      T nn2 = warp_sum(u0 * u0 + u1 * u1);
      for (int m = 0; m < n && nn2 < T(0.25); ++m) {
        // complete with e_m minus its projection on the columns before
        u0 = (lane == m) ? T(1) : T(0);
        u1 = (lane + 32 == m) ? T(1) : T(0);
        for (int j = 0; j < k; ++j) {
          const T d = warp_sum(Us[j * 64 + lane] * u0 + Us[j * 64 + lane + 32] * u1);
          u0 -= d * Us[j * 64 + lane];
          u1 -= d * Us[j * 64 + lane + 32];
        }
        nn2 = warp_sum(u0 * u0 + u1 * u1);
      }
      const T inv = T(1) / sqrt(nn2);
      Us[k * 64 + lane] = (lane < n) ? u0 * inv : T(0);
      Us[k * 64 + lane + 32] = (lane + 32 < n) ? u1 * inv : T(0);
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int l = e % n, k = e / n;
    Ub[piv[l] + n * k] = (double)Us[k * 64 + l];
  }
}

// Householder QR with column pivoting of an n x n matrix (n <= 64), one CTA: Rin P = Q R2, with
// R2 upper triangular (written n x n, zeros below the diagonal) and piv[j] the column of Rin in
// position j.  At step k the column of largest norm over rows k..n-1 moves to position k, and the
// reflector I - v v^T / (v^T v), v = x - alpha e_1, alpha = -sign(x_1) ||x||, zeroes it below row k.
template <typename T>
struct PivQrOp {
  struct Args {
    const T* Rin;
    int n;
    T* R2;
    int32_t* piv;
    const int32_t* gate;
    int32_t want;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void PivQrOp<T>::body(const Grid g, const Args& args) {
  if (args.gate != nullptr && *args.gate != args.want) return;
  constexpr int LD = 65;
  __shared__ T A[64 * LD];   // column-major, leading dimension 65
  __shared__ T cn[64];
  __shared__ int pv[64];
  __shared__ int jmax_s;
  const int n = args.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[(e % n) + LD * (e / n)] = args.Rin[e];
  for (int j = threadIdx.x; j < n; j += blockDim.x) pv[j] = j;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // norms of the trailing parts of the columns j >= k, one warp per column
    for (int j = k + w; j < n; j += nw) {
      T s = T(0);
      for (int i = k + lane; i < n; i += 32) s += A[i + LD * j] * A[i + LD * j];
      s = warp_sum(s);
      if (lane == 0) cn[j] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int jm = k;
      for (int j = k + 1; j < n; ++j)
        if (cn[j] > cn[jm]) jm = j;
      jmax_s = jm;
    }
    __syncthreads();
    const int jm = jmax_s;
    if (jm != k) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T t = A[i + LD * k];
        A[i + LD * k] = A[i + LD * jm];
        A[i + LD * jm] = t;
      }
      if (threadIdx.x == 0) {
        const int t = pv[k];
        pv[k] = pv[jm];
        pv[jm] = t;
        const T c = cn[k];
        cn[k] = cn[jm];
        cn[jm] = c;
      }
    }
    __syncthreads();
    const T nx2 = cn[k];
    if (nx2 > T(0) && k < n - 1) {
      const T x1 = A[k + LD * k];
      const T alpha = x1 >= T(0) ? -sqrt(nx2) : sqrt(nx2);
      const T v1 = x1 - alpha;                // v = (v1, A[k+1.., k])
      const T vtv = nx2 - x1 * x1 + v1 * v1;
      // apply to the columns j > k, one warp per column
      for (int j = k + 1 + w; j < n; j += nw) {
        T s = (lane == 0) ? v1 * A[k + LD * j] : T(0);
        for (int i = k + 1 + lane; i < n; i += 32) s += A[i + LD * k] * A[i + LD * j];
        s = warp_sum(s);
        const T f = T(2) * s / vtv;
        if (lane == 0) A[k + LD * j] -= f * v1;
        for (int i = k + 1 + lane; i < n; i += 32) A[i + LD * j] -= f * A[i + LD * k];
      }
      __syncthreads();
      for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + LD * k] = T(0);
      if (threadIdx.x == 0) A[k + LD * k] = alpha;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    args.R2[e] = (i <= j) ? A[i + LD * j] : T(0);
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) args.piv[j] = pv[j];
}

template <typename T>
struct FactorCastOp {
  struct Args {
    int64_t I;
    int ell;
    int r;
    const double* Q;
    const double* Ub;
    double* A;
    T* Uc;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void FactorCastOp<T>::body(const Grid g, const Args& args) {
  int64_t I = args.I;
  int ell = args.ell;
  int r = args.r;
  const double* __restrict__ Q = args.Q;
  const double* __restrict__ Ub = args.Ub;
  double* __restrict__ A = args.A;
  T* __restrict__ Uc = args.Uc;

  const int64_t total = I * r;
  for (int64_t e = g.bx * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)g.gx * blockDim.x) {
    const int64_t i = e % I;
    const int k = (int)(e / I);
    double s = 0.0;
    for (int c = 0; c < ell; ++c) s = fma(Q[i + I * c], Ub[c + (int64_t)ell * k], s);
    A[e] = s;
  }
  if (Uc != nullptr) {
    for (int64_t e = g.bx * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ell * r;
         e += (int64_t)g.gx * blockDim.x)
      Uc[e] = (T)Ub[e];
  }
}

// Column-sign convention shared with the oracle: flip column k of A (m x n) so that its
// largest-magnitude entry (first index on ties) is positive; apply the same flip to
// column k of ``other`` (rows_o x n, leading dimension rows_o) when given.  One CTA per column.
template <typename T>
struct ColsignOp {
  struct Args {
    double* A;
    int64_t m;
    int n;
    T* other;
    int rows_o;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void ColsignOp<T>::body(const Grid g, const Args& args) {
  double* __restrict__ A = args.A;
  int64_t m = args.m;
  int n = args.n;
  T* __restrict__ other = args.other;
  int rows_o = args.rows_o;

  __shared__ double sv[32];
  __shared__ int64_t si[32];
  __shared__ double sgn;
  const int k = g.bx;
  double* a = A + m * (int64_t)k;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double v = fabs(a[i]);
    if (v > best) {  // strictly greater keeps the first index within a thread
      best = v;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sv[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sv[0];
    int64_t ii = si[0];
    for (int q = 1; q < nw; ++q)
      if (sv[q] > b || (sv[q] == b && si[q] < ii)) {
        b = sv[q];
        ii = si[q];
      }
    sgn = (a[ii] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn < 0.0) {
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) a[i] = -a[i];
    if (other != nullptr)
      for (int i = threadIdx.x; i < rows_o; i += blockDim.x) other[i + (int64_t)rows_o * k] = -other[i + (int64_t)rows_o * k];
  }
}

template <typename T>
struct CastOp {
  struct Args {
    const double* src;
    T* dst;
    int64_t n;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void CastOp<T>::body(const Grid g, const Args& args) {
  const double* __restrict__ src = args.src;
  T* __restrict__ dst = args.dst;
  int64_t n = args.n;

  for (int64_t e = g.bx * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)g.gx * blockDim.x)
    dst[e] = (T)src[e];
}

struct SumsqOp {
  struct Args {
    const double* x;
    int64_t n;
    double* out;
  };
  static constexpr int kThreads = 1024, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void SumsqOp::body(const Grid g, const Args& args) {
  const double* __restrict__ x = args.x;
  int64_t n = args.n;
  double* __restrict__ out = args.out;

  __shared__ double scratch[33];
  // eight independent chains per thread (loads in flight together), combined in a fixed order
  double c[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t st = blockDim.x;
  int64_t e = threadIdx.x;
  for (; e + 7 * st < n; e += 8 * st) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const double v = x[e + j * st];
      c[j] = fma(v, v, c[j]);
    }
  }
  for (; e < n; e += st) c[0] = fma(x[e], x[e], c[0]);
  double s = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) *out = s;
}

// ||x||^2 over many CTAs (FP64 arithmetic runs at a small fraction of the FP32 rate on this part, so
// one CTA is bound by its SM's FP64 pipe): CTA b sums the contiguous range [b chunk, (b + 1) chunk)
// into part[b] (eight chains per thread, fixed-order combine), SumPartsOp adds the partials in a
// fixed order.
struct SumsqPartOp {
  struct Args {
    const double* x;
    int64_t n, chunk;
    double* part;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& a) {
    __shared__ double scratch[33];
    const int64_t b0 = (int64_t)g.bx * a.chunk, b1 = min(a.n, b0 + a.chunk);
    double c[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int64_t e = b0 + threadIdx.x;
    for (; e + 7 * 256 < b1; e += 8 * 256) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const double v = a.x[e + j * 256];
        c[j] = fma(v, v, c[j]);
      }
    }
    for (; e < b1; e += 256) c[0] = fma(a.x[e], a.x[e], c[0]);
    double s = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
    s = block_sum(s, scratch);
    if (threadIdx.x == 0) a.part[g.bx] = s;
  }
};
struct SumPartsOp {
  struct Args {
    const double* part;
    int n;
    double* out;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& a) {
    __shared__ double scratch[33];
    (void)g;
    double s = 0.0;
    for (int k = threadIdx.x; k < a.n; k += 256) s += a.part[k];
    s = block_sum(s, scratch);
    if (threadIdx.x == 0) *a.out = s;
  }
};

// Gram matrix W = B_(n) B_(n)^T (ell x ell) of a (L, ell, R) tensor, streamed once: CTAs walk
// tiles of 128 unfolding columns staged in shared memory (row pp = column p of B_(n), 16-byte
// aligned rows).  W is split into 4 x 4 blocks and thread t < NB (NB + 1) / 2 owns the t-th
// block of the upper triangle (NB = ELLP / 4); it sums a tile's 128 products in FP32 and adds
// the tile sum to FP64 accumulators.  Per-CTA FP64 partials (upper triangle) are reduced in a
// fixed order.
template <int ELLP>
struct GramCfg {
  static constexpr int NB = ELLP / 4;
  static constexpr int NBLK = NB * (NB + 1) / 2;
  static constexpr int THREADS = (NBLK + 31) / 32 * 32;
  static constexpr int LDS = ELLP + 4;
  static constexpr size_t SMEM = 2 * 128 * LDS * sizeof(float);   // two tiles (dynamic)
};

// DF = true: every product is formed exactly (p = x y, e = fma(x, y, -p)) and summed in double-float
// (TwoSum of the running sum and p, the rounding errors and e collected in a second FP32 term), so a
// tile's partial carries ~2^-44 relative error instead of the FP32 sum's ~128 u; the Gram matrix is
// then accurate enough for the Cholesky-Jacobi route at any condition number below ~1e6.
template <int ELLP, bool DF>
struct GramBOp {
  struct Args {
    const float* B;
    int64_t L;
    int64_t R;
    int ell;
    double* part;
    const int32_t* gate;
  };
  static constexpr int kThreads = GramCfg<ELLP>::THREADS, kMinBlocks = 3;
  __device__ static void body(const Grid g, const Args& args);
};
template <int ELLP, bool DF>
__device__ __forceinline__ void GramBOp<ELLP, DF>::body(const Grid g, const Args& args) {
  const float* __restrict__ B = args.B;
  int64_t L = args.L;
  int64_t R = args.R;
  int ell = args.ell;
  double* __restrict__ part = args.part;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate != 0) return;
  using C = GramCfg<ELLP>;
  extern __shared__ __align__(16) float gram_sm[];   // two tiles of 128 x LDS
  const int tid = threadIdx.x;
  int bi = 0, bj = tid;
  while (bi < C::NB && bj >= C::NB - bi) {
    bj -= C::NB - bi;
    ++bi;
  }
  bj += bi;
  const bool active = tid < C::NBLK;
  const int64_t M = L * R;
  const int64_t ntiles = (M + 127) / 128;
  for (int e = tid; e < 2 * 128 * (C::LDS - ell); e += blockDim.x) {
    const int w = C::LDS - ell;
    gram_sm[(e / w) * C::LDS + ell + e % w] = 0.0f;   // padding columns of both tiles
  }
  // asynchronous copy of tile t into Bs: rows pp = columns p0 + pp of B_(n), zero past M
  const int nthr = blockDim.x;
  auto issue = [&](int64_t t, float* Bs) {
    const int64_t p0 = t * 128;
    const int valid = (int)(M - p0 < 128 ? M - p0 : 128);
    if (L == 1) {
      // the tile is 128 x ell contiguous values starting 512 ell bytes into B: 16-byte aligned
      const float* src = B + (int64_t)ell * p0;
      const int nvalid = valid * ell;
      if ((ell & 3) == 0) {
        const int q4 = ell / 4, dq = nthr / q4, rq = nthr - dq * q4;
        int pp = tid / q4, cq = tid - pp * q4;
        for (int e4 = tid; e4 < 32 * ell; e4 += nthr) {
          const bool ok = 4 * e4 < nvalid;
          cp_async16(&Bs[pp * C::LDS + 4 * cq], ok ? src + 4 * e4 : B, ok);
          pp += dq;
          cq += rq;
          if (cq >= q4) {
            cq -= q4;
            ++pp;
          }
        }
      } else {
        const int de = nthr / ell, re = nthr - de * ell;
        int pp = tid / ell, c = tid - pp * ell;
        for (int e = tid; e < 128 * ell; e += nthr) {
          const bool ok = e < nvalid;
          cp_async4(&Bs[pp * C::LDS + c], ok ? src + e : B, ok);
          pp += de;
          c += re;
          if (c >= ell) {
            c -= ell;
            ++pp;
          }
        }
      }
    } else {
      for (int pp = tid; pp < 128; pp += nthr) {
        const bool ok = pp < valid;
        const int64_t p = p0 + pp;
        const float* src = ok ? B + (p % L) + L * (int64_t)ell * (p / L) : B;
        for (int c = 0; c < ell; ++c) cp_async4(&Bs[pp * C::LDS + c], ok ? src + L * c : B, ok);
      }
    }
    cp_async_commit();
  };
  // tile sums accumulate in FP32 pairs (hi, lo) that keep every rounding error (TwoSum): FP64
  // arithmetic runs at a small fraction of the FP32 rate on this part
  float acch[4][4], accl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acch[a][b] = accl[a][b] = 0.0f;
  float* bufs[2] = {gram_sm, gram_sm + 128 * C::LDS};
  int cur = 0;
  __syncthreads();   // padding written before any tile lands next to it
  if ((int64_t)g.bx < ntiles) issue(g.bx, bufs[0]);
  for (int64_t t = g.bx; t < ntiles; t += g.gx) {
    // the next tile streams in while this one is multiplied
    if (t + g.gx < ntiles) {
      issue(t + g.gx, bufs[cur ^ 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* Bs = bufs[cur];
    if (active) {
      float acc[4][4], err[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b] = 0.0f;
          err[a][b] = 0.0f;
        }
#pragma unroll 8
      for (int pp = 0; pp < 128; ++pp) {
        const float4 x = *reinterpret_cast<const float4*>(&Bs[pp * C::LDS + 4 * bi]);
        const float4 y = *reinterpret_cast<const float4*>(&Bs[pp * C::LDS + 4 * bj]);
        const float xa[4] = {x.x, x.y, x.z, x.w};
        const float yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if constexpr (DF) {
              const float pr = __fmul_rn(xa[a], yb[b]);
              const float pe = fmaf(xa[a], yb[b], -pr);           // x y = pr + pe exactly
              const float sm = __fadd_rn(acc[a][b], pr);
              const float bb = __fsub_rn(sm, acc[a][b]);
              const float se = __fadd_rn(__fsub_rn(acc[a][b], __fsub_rn(sm, bb)), __fsub_rn(pr, bb));
              acc[a][b] = sm;                                      // acc + pr = sm + se exactly
              err[a][b] = __fadd_rn(err[a][b], __fadd_rn(se, pe));
            } else {
              acc[a][b] = fmaf(xa[a], yb[b], acc[a][b]);
            }
          }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float v = acc[a][b];
          const float t = __fadd_rn(acch[a][b], v);
          const float bp = __fsub_rn(t, acch[a][b]);
          accl[a][b] = __fadd_rn(accl[a][b], __fadd_rn(__fsub_rn(acch[a][b], __fsub_rn(t, bp)), __fsub_rn(v, bp)));
          acch[a][b] = t;
          if constexpr (DF) accl[a][b] = __fadd_rn(accl[a][b], err[a][b]);
        }
    }
    __syncthreads();   // this tile's buffer is refilled two tiles later
    cur ^= 1;
  }
  if (!active) return;
  double* o = part + (int64_t)g.bx * ell * ell;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = 4 * bi + a, c = 4 * bj + b;
      if (r <= c && c < ell) o[r + ell * c] = (double)acch[a][b] + (double)accl[a][b];
    }
}

// W[r, c] = sum over CTAs of the upper-triangle partial at (min(r, c), max(r, c)).  A block of
// 256 threads owns 32 consecutive entries of W: warp k sums partials k, k + 8, ... and the eight
// warp sums are added in a fixed order.
struct GramBReduceOp {
  struct Args {
    const double* part;
    int nparts;
    int ell;
    double* W;
    const int32_t* gate;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void GramBReduceOp::body(const Grid g, const Args& args) {
  const double* __restrict__ part = args.part;
  int nparts = args.nparts;
  int ell = args.ell;
  double* __restrict__ W = args.W;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate != 0) return;
  __shared__ double red[8][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nn = ell * ell;
  const int e = g.bx * 32 + lane;
  double s = 0.0;
  if (e < nn) {
    const int r = e % ell, c = e / ell;
    const int u = r <= c ? e : c + ell * r;
    // eight independent chains (loads in flight together), combined in a fixed order
    double ch[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int k = wp;
    for (; k + 56 < nparts; k += 64) {
#pragma unroll
      for (int j = 0; j < 8; ++j) ch[j] += part[(int64_t)(k + 8 * j) * nn + u];
    }
    for (; k < nparts; k += 8) ch[0] += part[(int64_t)k * nn + u];
    s = ((ch[0] + ch[1]) + (ch[2] + ch[3])) + ((ch[4] + ch[5]) + (ch[6] + ch[7]));
  }
  red[wp][lane] = s;
  __syncthreads();
  if (wp == 0 && e < nn) {
    double t = red[0][lane];
    for (int k = 1; k < 8; ++k) t += red[k][lane];
    W[e] = t;
  }
}

// Diagonally pivoted Cholesky of the Gram matrix W (n x n, FP64 in, n <= 64) in one CTA, in
// double-float after scaling W by a power of two: W = sum_k r_k r_k^T with r_k the k-th pivot row
// of R in the original indexing.  Writes X(:, k) = r_k (FP32, n x n column-major), so X X^T = W and
// the left singular vectors of X are the eigenvectors of W; choosing the largest remaining diagonal
// at every step makes the columns of X graded and nearly orthogonal, which is what makes one-sided
// Jacobi on X converge in few sweeps.  flag[0] <- 1 when the largest remaining pivot is
// <= 1e-14 max diag(W) (numerically singular W) or not finite.
// S is kept in pivot positions (upper triangle, position -> original index in perm).  Step k: the
// next pivot (largest remaining diagonal, first index on ties) is known from a 64-bit atomicMax of
// (value, position) taken while the diagonal was updated; positions k and p are swapped
// symmetrically; then column k of X is written and the trailing triangle updated through the
// table of ArithDF / chol_kernel.  Two barriers per step.
struct PivotedCholeskyOp {
  struct Args {
    const double* W;
    int n;
    float* X;
    int32_t* flag;
    int32_t* clear_on_success;
  };
  static constexpr int kThreads = kCholThreads, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void PivotedCholeskyOp::body(const Grid g, const Args& args) {
  const double* __restrict__ W = args.W;
  int n = args.n;
  float* __restrict__ X = args.X;
  int32_t* __restrict__ flag = args.flag;
  int32_t* __restrict__ clear_on_success = args.clear_on_success;

  if (flag[0]) return;
  using Ar = ArithDF;
  using V = Ar::V;
  extern __shared__ __align__(16) unsigned char chol_raw[];
  const int ld = n | 1;
  V* S = reinterpret_cast<V*>(chol_raw);
  uint16_t* tab = reinterpret_cast<uint16_t*>(chol_raw + ((sizeof(V) * ld * n + 15) & ~size_t(15)));
  __shared__ int perm[RH_MAX_ELL];
  __shared__ unsigned long long key[2];
  __shared__ V rinv_s;
  __shared__ double scale_s;
  __shared__ float dmax_s;
  __shared__ int hexp_s, ok_s, bad;
  const int t = threadIdx.x;
  diag_scale<Ar>(W, n, &scale_s, &hexp_s, &dmax_s, &ok_s);
  build_tri_table(tab, n);
  if (t < RH_MAX_ELL) perm[t] = t;
  if (t == 0) {
    key[0] = 0ull;
    key[1] = 0ull;
  }
  __syncthreads();
  const double sc = scale_s;
  const float dmax = dmax_s;
  {
    double w[kCholPer];
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {   // all loads first
      const int e = t + kCholThreads * q;
      w[q] = (e < n * n && (e % n) <= (e / n)) ? W[e] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kCholPer; ++q) {
      const int e = t + kCholThreads * q;
      if (e < n * n) {
        S[(e % n) + ld * (e / n)] = Ar::from(w[q] * sc);
        X[e] = 0.0f;
      }
    }
  }
  __syncthreads();
  auto pack = [](float v, int pos) -> unsigned long long {
    const float c = (v > 0.0f && isfinite(v)) ? v : 0.0f;
    return ((unsigned long long)__float_as_uint(c) << 32) | (unsigned long long)(63 - pos);
  };
  for (int i = t; i < n; i += blockDim.x) atomicMax(&key[0], pack(S[i + ld * i].hi, i));
  if (t == 0) bad = ok_s ? 0 : 1;
  __syncthreads();
  const float unscale = ldexpf(1.0f, hexp_s);   // exact: 1 / sqrt(scale)
  for (int k = 0; k < n; ++k) {
    if (bad) break;  // uniform: read after the barrier
    const unsigned long long kk = key[k & 1];
    const int p = 63 - (int)(kk & 0xFFFFFFFFull);
    // swap positions k and p (p >= k): S(k, j) <-> S(j, p) for k < j < p, S(k, j) <-> S(p, j) for j > p
    if (t == 0) {
      key[(k + 1) & 1] = 0ull;
      const V dp = S[p + ld * p];
      if (!(dp.hi > 1e-14f * dmax) || !Ar::finite(dp)) {
        bad = 1;
      } else {
        S[p + ld * p] = S[k + ld * k];
        S[k + ld * k] = dp;
        const int q = perm[k];
        perm[k] = perm[p];
        perm[p] = q;
        rinv_s = Ar::rsq(dp);
      }
    } else if (p != k) {
      for (int j = k + t; j < n; j += blockDim.x - 1) {   // t >= 1: j > k
        if (j == p) continue;
        V* a = &S[k + ld * j];
        V* b = (j < p) ? &S[j + ld * p] : &S[p + ld * j];
        const V tmp = *a;
        *a = *b;
        *b = tmp;
      }
    }
    __syncthreads();
    if (bad) break;
    const V ri = rinv_s;
    // column k of X: r_k(j) = S(k, j) / sqrt(S(k, k)) at position j >= k, original index perm[j]
    for (int j = k + t; j < n; j += blockDim.x)
      X[perm[j] + n * k] = Ar::mul(S[k + ld * j], ri).hi * unscale;
    // trailing update; the updated diagonal proposes the next pivot
    const V ri2 = Ar::mul(ri, ri);
    const int T = (n - k - 1) * (n - k) / 2;
    const int stride = blockDim.x;
    for (int e = t; e < T; e += 2 * stride) {   // two entries per pass, operands read first
      const int e2 = e + stride;
      const int ij = tab[e];
      const int ij2 = e2 < T ? tab[e2] : ij;
      const int i = ij >> 8, j = ij & 255, i2 = ij2 >> 8, j2 = ij2 & 255;
      const V x1 = S[i + ld * j], a1 = S[k + ld * i], b1 = S[k + ld * j];
      const V x2 = S[i2 + ld * j2], a2 = S[k + ld * i2], b2 = S[k + ld * j2];
      const V v1 = Ar::fms(x1, Ar::mul(a1, ri2), b1);
      const V v2 = Ar::fms(x2, Ar::mul(a2, ri2), b2);
      S[i + ld * j] = v1;
      if (i == j) atomicMax(&key[(k + 1) & 1], pack(v1.hi, i));
      if (e2 < T) {
        S[i2 + ld * j2] = v2;
        if (i2 == j2) atomicMax(&key[(k + 1) & 1], pack(v2.hi, i2));
      }
    }
    __syncthreads();
  }
  if (bad && t == 0) flag[0] = 1;
  if (!bad && t == 0 && clear_on_success != nullptr) *clear_on_success = 0;
}

// One-sided Jacobi on the columns of X (n x n, FP32, n <= 64) without accumulating the rotations:
// at convergence X = U S, so U is read off by normalising the columns.  Same circle schedule and
// rotation rule as jacobi_svd_kernel; the sweeps run in four warps, a group of four lanes per pair
// (a two-step shuffle reduction of each product, a 128-thread barrier per round).  Eight lanes per
// pair over eight warps with a block barrier per round took 193 us for n = 60, one lane per pair
// in one warp (no reduction, issue-bound on one scheduler) 257 us.
// A round is a chain of dependent steps, so its length is what counts: multi-function-unit
// operations (reciprocal, square root) take ~40 cycles each against ~5 for an FMA on this part.
// The rotation of a pair with squared norms al, be and product g therefore needs two of them:
// with d = be - al, r = sqrt(d^2 + 4 g^2) and u = |d| + r, the angle of the classical rule
// (t = sign(d) 2 g / u, c = 1 / sqrt(1 + t^2), s = c t) has 1 + t^2 = 2 r / u, so
// c = u w, s = sign(d) 2 g w with w = 1 / sqrt(2 r u), and t g = sign(d) 4 g^2 r w^2 updates the
// squared norms (al - t g, be + t g) without a division.  The pair is rotated when
// g^2 > tol^2 al be (no square root on the way).  X is first scaled by a power of two so that
// its largest squared column norm lies in [1, 4) (d^2 + 4 g^2 cannot overflow); the singular
// values are scaled back at the end.  Products and rotations run on packed FP32 pairs.
// Sweeps end when one rotates nothing, or when the largest coupling it rotated was at most
// sqrt(tol / n) (the quadratic convergence of the cyclic Jacobi method then leaves every coupling
// of the next sweep below tol, so that sweep is not run).
// Afterwards the columns are normalised, sorted by decreasing norm and made orthonormal to FP32
// rounding by one polar correction U <- U (3 I - U^T U) / 2 (the Jacobi tolerance leaves
// |u_i^T u_j| <= tol).  Writes Ub (n x n, FP64) and sv = the column norms (FP64), sorted.
constexpr int kRowJacThreads = 256;

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

struct JacobiRowsOp {
  struct Args {
    const float* Xin;
    int n;
    double* Ub;
    double* sv;
    const int32_t* gate;
    int32_t* info_or;
    int32_t info_bits;
  };
  static constexpr int kThreads = kRowJacThreads, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void JacobiRowsOp::body(const Grid g, const Args& args) {
  const float* __restrict__ Xin = args.Xin;
  int n = args.n;
  double* __restrict__ Ub = args.Ub;
  double* __restrict__ sv = args.sv;
  const int32_t* __restrict__ gate = args.gate;
  int32_t* __restrict__ info_or = args.info_or;
  int32_t info_bits = args.info_bits;

  if (gate != nullptr && *gate != 0) return;
  if (info_or != nullptr && threadIdx.x == 0) *info_or |= info_bits;
  extern __shared__ __align__(16) float jsm[];
  const int np = (n + 1) & ~1;
  const int half = np / 2;
  // columns by position, rows padded to kLdb floats (320 bytes): the two pair groups of a 16-byte
  // access phase read two neighbouring columns at one offset and land on disjoint banks
  constexpr int kLdb = 80;
  float* buf0 = jsm;                    // [position][kLdb]
  float* buf1 = buf0 + 64 * kLdb;
  float* U = buf1 + 64 * kLdb;          // [64][65]: U(i, c) at i + 65 c
  float* E = U + 64 * 65;               // [64][65]
  __shared__ float nrm2[2][RH_MAX_ELL];
  __shared__ float sig[RH_MAX_ELL];
  __shared__ int rankof[RH_MAX_ELL];
  __shared__ int s_cur, s_exp;
  __shared__ unsigned s_red[2][4];      // per sweep-warp: any rotation, largest rotated coupling^2
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int e = t; e < 64 * 64; e += blockDim.x) {
    const int i = e & 63, q = e >> 6;
    buf0[kLdb * q + i] = (q < n && i < n) ? Xin[i + n * q] : 0.0f;
  }
  __syncthreads();
  // largest squared column norm -> the power-of-two scale 2^-s_exp applied to every entry
  {
    float mx = 0.0f;
    for (int q = w; q < np; q += blockDim.x >> 5) {
      const float x0 = buf0[kLdb * q + lane], x1 = buf0[kLdb * q + 32 + lane];
      float v = x0 * x0 + x1 * x1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      mx = fmaxf(mx, v);
    }
    if (lane == 0) sig[w] = mx;
    __syncthreads();
    if (t == 0) {
      float m = 0.0f;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, sig[k]);
      // 2^(2 e) <= m < 2^(2 e + 2); the entries are divided by 2^e
      s_exp = (m > 0.0f && isfinite(m)) ? (ilogbf(m) >> 1) : 0;
    }
    __syncthreads();
    const float sc = ldexpf(1.0f, -s_exp);
    for (int e = t; e < 64 * kLdb; e += blockDim.x) buf0[e] *= sc;
    __syncthreads();
  }
  const float tol = (float)(8 * (n > 8 ? n : 8)) * 5.9604645e-8f;
  const float tol2 = tol * tol;
  // Quadratic convergence: a sweep whose largest rotated coupling is c leaves couplings of order
  // c^2, so once c <= sqrt(tol / n) the next sweep would rotate nothing and is skipped.
  const float cstop2 = tol / (float)(n > 1 ? n : 1);
  // The sweeps run in warps 0..3 (one per scheduler) with a 128-thread barrier between rounds; a
  // group of four lanes rotates one pair, lane l holding entries 4l..4l+3 + 16m (m < 4) of both
  // columns.  The other warps wait for the epilogue.
  if (w < 4) {
    const int grp = lane >> 2, l = lane & 3;
    const int pr = 8 * w + grp;
    const bool active = pr < half;
    const int qa = active ? pr : 0, qb = active ? np - 1 - pr : 0;
    const int na = (qa == 0) ? 0 : (qa == np - 1 ? 1 : qa + 1);
    const int nb = (qb == 0) ? 0 : (qb == np - 1 ? 1 : qb + 1);
    int cur = 0;
    for (int sweep = 0; sweep < 40; ++sweep) {
      {
        const float* src = cur ? buf1 : buf0;
        for (int q = w; q < np; q += 4) {
          const float x0 = src[kLdb * q + lane], x1 = src[kLdb * q + 32 + lane];
          float v = x0 * x0 + x1 * x1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) nrm2[cur][q] = v;
        }
        named_bar_sync(1, 128);
      }
      int rotated = 0;
      float cmx2 = 0.0f;
      for (int rnd = 0; rnd < np - 1; ++rnd) {
        const float* src = cur ? buf1 : buf0;
        float* dst = cur ? buf0 : buf1;
        float2 a[8], b[8];   // a[2 m], a[2 m + 1]: entries 4 l + 16 m + {0, 1} and + {2, 3}
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float4 va = *reinterpret_cast<const float4*>(src + kLdb * qa + 4 * l + 16 * m);
          const float4 vb = *reinterpret_cast<const float4*>(src + kLdb * qb + 4 * l + 16 * m);
          a[2 * m] = make_float2(va.x, va.y);
          a[2 * m + 1] = make_float2(va.z, va.w);
          b[2 * m] = make_float2(vb.x, vb.y);
          b[2 * m + 1] = make_float2(vb.z, vb.w);
        }
        float al = nrm2[cur][qa], be = nrm2[cur][qb];
        float2 g0 = make_float2(0.0f, 0.0f), g1 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          g0 = f2_fma(a[2 * m], b[2 * m], g0);
          g1 = f2_fma(a[2 * m + 1], b[2 * m + 1], g1);
        }
        float gg = (g0.x + g0.y) + (g1.x + g1.y);
        gg += __shfl_xor_sync(0xffffffffu, gg, 1);
        gg += __shfl_xor_sync(0xffffffffu, gg, 2);
        const float g2 = gg * gg;
        const float albe = al * be;
        const float d = be - al;
        const float q = fmaf(d, d, 4.0f * g2);
        if (active && g2 > tol2 * albe && albe > 0.0f && q > 0.0f) {
          const float r = q * rsqrtf(q);
          const float u = fabsf(d) + r;
          const float wv = rsqrtf(2.0f * r * u);
          const float c = u * wv;
          const float sn = copysignf(2.0f, d) * gg * wv;   // sign(d) 2 g w, sign(0) = +
          const float tg = copysignf(4.0f, d) * g2 * r * wv * wv;
          const float2 c2 = make_float2(c, c), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const float2 x = a[m], y = b[m];
            a[m] = f2_fma(c2, x, f2_mul(ns2, y));
            b[m] = f2_fma(c2, y, f2_mul(s2, x));
          }
          al = al - tg;
          be = be + tg;
          rotated = 1;
          cmx2 = fmaxf(cmx2, __fdividef(g2, albe));
        }
        if (active) {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            *reinterpret_cast<float4*>(dst + kLdb * na + 4 * l + 16 * m) =
                make_float4(a[2 * m].x, a[2 * m].y, a[2 * m + 1].x, a[2 * m + 1].y);
            *reinterpret_cast<float4*>(dst + kLdb * nb + 4 * l + 16 * m) =
                make_float4(b[2 * m].x, b[2 * m].y, b[2 * m + 1].x, b[2 * m + 1].y);
          }
          if (l == 0) {
            nrm2[cur ^ 1][na] = al;
            nrm2[cur ^ 1][nb] = be;
          }
        }
        cur ^= 1;
        named_bar_sync(1, 128);
      }
      // squared couplings are >= 0 (or +inf when a norm underflowed): their FP32 bit patterns
      // order like the values
      const unsigned anyw = __any_sync(0xffffffffu, rotated);
      const unsigned mxw = __reduce_max_sync(0xffffffffu, (unsigned)__float_as_int(cmx2));
      if (lane == 0) {
        s_red[0][w] = anyw;
        s_red[1][w] = mxw;
      }
      named_bar_sync(1, 128);
      const unsigned any4 = s_red[0][0] | s_red[0][1] | s_red[0][2] | s_red[0][3];
      const unsigned mx4 = max(max(s_red[1][0], s_red[1][1]), max(s_red[1][2], s_red[1][3]));
      if (!any4 || __int_as_float((int)mx4) <= cstop2) break;
    }
    if (t == 0) s_cur = cur;
  }
  __syncthreads();
  const int cur = s_cur;
  // every sweep ends with player q at position q: columns are X's columns, rotated
  const float* fin = cur ? buf1 : buf0;
  for (int q = w; q < n; q += blockDim.x >> 5) {
    const float a = fin[kLdb * q + lane], b = fin[kLdb * q + 32 + lane];
    float v = a * a + b * b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sig[q] = sqrtf(v);
  }
  __syncthreads();
  const float unsc = ldexpf(1.0f, s_exp);   // exact
  for (int q = t; q < n; q += blockDim.x) {
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += (sig[k] > sig[q]) || (sig[k] == sig[q] && k < q);
    rankof[q] = rank;
    sv[rank] = (double)sig[q] * (double)unsc;
  }
  __syncthreads();
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e % n, q = e / n;
    const float s = sig[q];
    U[i + 65 * rankof[q]] = s > 0.0f ? fin[kLdb * q + i] / s : (i == q ? 1.0f : 0.0f);
  }
  __syncthreads();
  // polar correction: E = U^T U, U <- 1.5 U - 0.5 U E
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    float acc = 0.0f;
    for (int k = 0; k < n; ++k) acc = fmaf(U[k + 65 * i], U[k + 65 * j], acc);
    E[i + 65 * j] = acc;
  }
  __syncthreads();
  for (int e = t; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    float acc = 0.0f;
    for (int k = 0; k < n; ++k) acc = fmaf(U[i + 65 * k], E[k + 65 * j], acc);
    Ub[i + n * j] = (double)(1.5f * U[i + 65 * j] - 0.5f * acc);
  }
}

// dst (k x k) = the leading k x k block of the column-major n x n src
template <typename TS, typename TD>
__global__ void copy_leading_kernel(const TS* __restrict__ src, int n, int k, TD* __restrict__ dst) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x)
    dst[e] = (TD)src[(e % k) + n * (e / k)];
}
// d[c] = W[c, c]
__global__ void diag_kernel(const double* __restrict__ W, int n, double* __restrict__ d) {
  for (int c = threadIdx.x; c < n; c += blockDim.x) d[c] = W[c + n * c];
}
// d[c] = sum_i R[i, c]^2 (the squared norm of row c of B when B^T = Q_B R)
template <typename T>
__global__ void colnorm2_kernel(const T* __restrict__ R, int n, double* __restrict__ d) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) {
    const double v = (double)R[i + n * c];
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  if (threadIdx.x == 0) d[c] = s;
}

struct CastF2dGatedOp {
  struct Args {
    const float* src;
    double* dst;
    int64_t n;
    const int32_t* gate;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void CastF2dGatedOp::body(const Grid g, const Args& args) {
  const float* __restrict__ src = args.src;
  double* __restrict__ dst = args.dst;
  int64_t n = args.n;
  const int32_t* __restrict__ gate = args.gate;

  if (*gate) return;
  for (int64_t e = g.bx * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)g.gx * blockDim.x)
    dst[e] = (double)src[e];
}

// After the Gram route: fall back to the tall-skinny QR when the Cholesky factor broke down or
// when the truncation gap sigma_r^2 - sigma_{r+1}^2 is below 1e-5 sigma_1^2, where the FP32
// Gram cannot resolve the top-r subspace.
// Decides the first (FP32 Gram) route; arm[0] = 0 arms the second (double-float Gram) route exactly
// when the first is rejected, arm[0] = 1 keeps it off.
struct TruncDecideOp {
  struct Args {
    const int32_t* chol_flag;
    const double* sv;
    int ell;
    int r;
    int32_t* use_tsqr;
    int32_t* info;
    int32_t* arm;
  };
  static constexpr int kThreads = 32, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void TruncDecideOp::body(const Grid g, const Args& args) {
  const int32_t* __restrict__ chol_flag = args.chol_flag;
  const double* __restrict__ sv = args.sv;
  int ell = args.ell;
  int r = args.r;
  int32_t* __restrict__ use_tsqr = args.use_tsqr;
  int32_t* __restrict__ info = args.info;
  int32_t* __restrict__ arm = args.arm;

  if (threadIdx.x != 0 || g.bx != 0) return;
  if (*chol_flag) {
    *use_tsqr = 1;
    if (arm != nullptr) arm[0] = 0;
    return;
  }
  const double s1 = sv[0];
  const double sr = sv[r - 1];
  const double sr1 = (r < ell) ? sv[r] : 0.0;
  const bool ok = (r >= ell) || (s1 == 0.0) || (sr * sr - sr1 * sr1 >= 1e-5 * s1 * s1);
  *use_tsqr = ok ? 0 : 1;
  if (arm != nullptr) arm[0] = ok ? 1 : 0;
  if (ok && info != nullptr) *info |= 2;
}

template <typename T>
struct CastGatedOp {
  struct Args {
    const double* src;
    T* dst;
    int64_t n;
    const int32_t* gate;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T>
__device__ __forceinline__ void CastGatedOp<T>::body(const Grid g, const Args& args) {
  const double* __restrict__ src = args.src;
  T* __restrict__ dst = args.dst;
  int64_t n = args.n;
  const int32_t* __restrict__ gate = args.gate;

  if (gate != nullptr && *gate != 0) return;
  for (int64_t e = g.bx * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)g.gx * blockDim.x)
    dst[e] = (T)src[e];
}

}  // namespace

// ---------------------------------------------------------------------------------
// Orthonormal basis W of range(B^T) for a subspace-iteration step (Sec. 5, "Variants")
// ---------------------------------------------------------------------------------
// W = B^T R^{-1} in place, row by row (forward substitution w R = b), for B^T stored in the
// (L, n, R) view of a mode product's output: row p, column c at (p % L) + L (c + n (p / L)).  R is
// upper triangular (n x n, column-major, element type TR).  A diagonal entry with
// |R_cc| <= tiny max_k |R_kk| (a numerically dependent column of B^T) gets the reciprocal 0, so
// column c of W is zero instead of overflowing.  Runs when flag is NULL or *flag == 0.  One warp
// per row, lane l holding entries l and l + 32.
template <typename T, typename TR>
struct TrsmViewOp {
  struct Args {
    T* B;
    int64_t L;
    int64_t R;
    int n;
    const TR* Rm;
    const int32_t* flag;
    double tiny;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& args);
};
template <typename T, typename TR>
__device__ __forceinline__ void TrsmViewOp<T, TR>::body(const Grid g, const Args& args) {
  T* __restrict__ B = args.B;
  const int64_t L = args.L, M = args.L * args.R;
  const int n = args.n;
  if (args.flag != nullptr && *args.flag != 0) return;
  __shared__ T Rs[RH_MAX_ELL * (RH_MAX_ELL | 1)];
  __shared__ T rd[RH_MAX_ELL];
  __shared__ double dmax_s;
  const int ld = n | 1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Rs[(e % n) + ld * (e / n)] = (T)args.Rm[e];
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += 32) m = fmax(m, fabs((double)args.Rm[k + n * k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) dmax_s = m;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double d = (double)args.Rm[k + n * k];
    rd[k] = (fabs(d) > args.tiny * dmax_s && isfinite(d)) ? (T)(1.0 / d) : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)g.gx * (blockDim.x >> 5);
  for (int64_t row = (int64_t)g.bx * (blockDim.x >> 5) + (threadIdx.x >> 5); row < M; row += warps) {
    T* b = B + (L == 1 ? (int64_t)n * row : (row % L) + L * (int64_t)n * (row / L));
    T y0 = lane < n ? b[L * lane] : T(0);
    T y1 = lane + 32 < n ? b[L * (lane + 32)] : T(0);
    for (int c = 0; c < n; ++c) {
      const T xc = __shfl_sync(0xffffffffu, c < 32 ? y0 : y1, c & 31) * rd[c];
      if (lane == (c & 31)) {
        if (c < 32) y0 = xc; else y1 = xc;
      }
      if (lane > c && lane < n) y0 -= xc * Rs[c + ld * lane];
      if (lane + 32 > c && lane + 32 < n) y1 -= xc * Rs[c + ld * (lane + 32)];
    }
    if (lane < n) b[L * lane] = y0;
    if (lane + 32 < n) b[L * (lane + 32)] = y1;
  }
}

// Gram matrix of B^T (FP64 data, (L, n, R) view): per-CTA partials part[cta][j + n k] =
// sum over the CTA's rows p of B^T(p, j) B^T(p, k) for j <= k (summed by GramBReduceOp).  Tiles of
// 32 rows in shared memory; thread t owns the upper-triangle entries t, t + 256, ...  Runs when
// flag is NULL or *flag == 0.
struct GramViewF64Op {
  struct Args {
    const double* B;
    int64_t L;
    int64_t R;
    int n;
    double* part;
    const int32_t* flag;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static constexpr int kPer = (RH_MAX_ELL * (RH_MAX_ELL + 1) / 2 + kThreads - 1) / kThreads;
  __device__ static void body(const Grid g, const Args& args);
};
__device__ __forceinline__ void GramViewF64Op::body(const Grid g, const Args& args) {
  const double* __restrict__ B = args.B;
  const int64_t L = args.L, M = args.L * args.R;
  const int n = args.n;
  if (args.flag != nullptr && *args.flag != 0) return;
  __shared__ double As[32][RH_MAX_ELL + 1];
  const int npairs = n * (n + 1) / 2;
  int ja[kPer], ka[kPer];
  double acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    int e = threadIdx.x + kThreads * q, j = 0;
    while (e >= n - j && j < n) {   // row-by-row walk of the upper triangle
      e -= n - j;
      ++j;
    }
    ja[q] = j;
    ka[q] = j + e;
    acc[q] = 0.0;
  }
  const int64_t ntiles = (M + 31) / 32;
  for (int64_t t = g.bx; t < ntiles; t += g.gx) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * n; e += blockDim.x) {
      const int r = e / n, c = e % n;
      const int64_t p = t * 32 + r;
      double v = 0.0;
      if (p < M) v = B[(L == 1 ? (int64_t)n * p : (p % L) + L * (int64_t)n * (p / L)) + L * c];
      As[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (threadIdx.x + kThreads * q < npairs) {
        double a = acc[q];
        for (int r = 0; r < 32; ++r) a = fma(As[r][ja[q]], As[r][ka[q]], a);
        acc[q] = a;
      }
    }
  }
  double* o = args.part + (int64_t)g.bx * n * n;
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (threadIdx.x + kThreads * q < npairs) o[ja[q] + n * ka[q]] = acc[q];
}

// ---------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------
static int gram_rows(int64_t m) {
  const int64_t target = std::max<int64_t>(1, num_sms());
  return (int)std::max<int64_t>(8, std::min<int64_t>(96, ceil_div(m, target)));
}

size_t orth_workspace_elems(int64_t m, int n) {
  const int rb = gram_rows(m);
  const int64_t nb = ceil_div(m, rb);
  // Gpart | C | R | rdiag | Q1 | W (Householder copy) | beta | flag (as one double)
  return (size_t)(nb * n * n + n * n + n * n + n + m * n + m * n + n + 2) + 64;
}

rh_status launch_gram_f32(const float* B, int64_t L, int64_t R, int ell, double* part, double* W,
                          const int32_t* gate, cudaStream_t st, bool df = false, int site = SITE_OTHER);

rh_status launch_orthonormalize(int64_t m, int n, const double* Y, double* Q, int32_t* info, double* ws,
                                cudaStream_t st, bool f32) {
  const int rb = gram_rows(m);
  const int nb = (int)ceil_div(m, rb);
  double* Gpart = ws;
  double* C = Gpart + (size_t)nb * n * n;
  double* R = C + n * n;
  double* rdiag = R + n * n;
  double* Q1 = rdiag + n;
  double* W = Q1 + m * n;
  double* beta = W + m * n;
  int32_t* flag = reinterpret_cast<int32_t*>(beta + n);
  rh_status s = emit_memset(SITE_ORTH_ZERO, 0, flag, sizeof(int32_t), st);
  if (s != RH_OK) return s;
  if ((s = emit_memset(SITE_ORTH_ZERO, 1, C, sizeof(double) * n * n, st)) != RH_OK) return s;
  const size_t gsm = sizeof(double) * rb * n;
  const int rblocks = (int)ceil_div((int64_t)n * n, 32);
  const int tblocks = (int)std::min<int64_t>(ceil_div(m, 8), 4 * num_sms());
  if (f32) {
    // FP32 data: CholeskyQR2 whose first pass keeps what its stability needs -- the Gram matrix in
    // FP64, its Cholesky factor in double-float, the triangular solve in FP64 (Q_1 is then
    // orthonormal to ~u_64 kappa(Y)) -- and whose second pass, on the nearly orthonormal Q_1, runs
    // in FP32.  A breakdown hands over to the Householder branch below.  The FP32 copies live in
    // the W region (only the Householder branch uses W, and it reads Y).
    RH_EMIT(GramPartialOp, SITE_ORTH_GRAM, 0, nb, gsm, Y, m, n, rb, Gpart, flag);
    RH_EMIT(GramReduceOp, SITE_ORTH_GRAM_REDUCE, 0, rblocks, 0, Gpart, nb, n, C, flag);
    // the first pass writes Q itself: when Q_1^T Q_1 is within 1e-6 of I (u_64 kappa(Y)^2 small) the
    // FP32 second pass is skipped (flag 2) and Q_1 is the result
    RH_EMIT(CholOp<ArithDF>, SITE_ORTH_CHOL, 0, 1, chol_smem(n, sizeof(dfl::F2)), C, n, R, rdiag, flag, 0.0);
    RH_EMIT(TrsmRowsOp<double>, SITE_ORTH_TRSM, 0, tblocks, sizeof(double) * ((n | 1) * n + n), Y, m, n, R, rdiag, Q,
            flag);
    float* Q1f = reinterpret_cast<float*>(W);
    float* Q2f = Q1f + m * n;
    const int cblocks = (int)std::min<int64_t>(ceil_div(m * n, 256), 4 * num_sms());
    RH_EMIT(CastGatedOp<float>, SITE_ORTH_CAST, 0, cblocks, 0, Q, Q1f, m * n, flag);
    if ((s = launch_gram_f32(Q1f, m, 1, n, Gpart, C, flag, st, false, SITE_ORTH_GRAM2)) != RH_OK) return s;
    RH_EMIT(CholOp<ArithF32>, SITE_ORTH_CHOL2, 0, 1, chol_smem(n, sizeof(float)), C, n, R, rdiag, flag, 1e-6);
    RH_EMIT(TrsmRowsOp<float>, SITE_ORTH_TRSM2, 0, tblocks, sizeof(float) * ((n | 1) * n + n), Q1f, m, n, R, rdiag,
            Q2f, flag);
    RH_EMIT(CastF2dGatedOp, SITE_ORTH_CAST2, 0, cblocks, 0, Q2f, Q, m * n, flag);
  } else {
    const size_t tsm = sizeof(double) * ((n | 1) * n + n);
    const double* src = Y;
    double* dst = Q1;
    for (int pass = 0; pass < 2; ++pass) {
      const int so = pass == 0 ? 0 : SITE_ORTH_GRAM2 - SITE_ORTH_GRAM;   // the second pass's sites
      RH_EMIT(GramPartialOp, SITE_ORTH_GRAM + so, 0, nb, gsm, src, m, n, rb, Gpart, flag);
      RH_EMIT(GramReduceOp, SITE_ORTH_GRAM_REDUCE + so, 0, rblocks, 0, Gpart, nb, n, C, flag);
      RH_EMIT(CholOp<ArithF64>, SITE_ORTH_CHOL + so, 0, 1, chol_smem(n, sizeof(double)), C, n, R, rdiag, flag, 0.0);
      RH_EMIT(TrsmRowsOp<double>, SITE_ORTH_TRSM + so, 0, tblocks, tsm, src, m, n, R, rdiag, dst, flag);
      src = Q1;
      dst = Q;
    }
  }
  RH_EMIT(HouseholderQOp, SITE_ORTH_HOUSEHOLDER, 0, 1, 0, Y, m, n, W, beta, Q, flag, info);
  RH_EMIT(ColsignOp<double>, SITE_ORTH_SIGN, 0, n, 0, Q, m, n, nullptr, 0);
  return RH_OK;
}

static int smem_budget() { return 96 * 1024; }

TruncPlan plan_trunc(const ModeView& vb, int ell) {
  TruncPlan pl;
  pl.v = vb;
  pl.ell = ell;
  return pl;
}

constexpr int kTsqrThreads = 1024;

template <typename T>
static void trunc_dims(TruncPlan& pl) {
  const int n = pl.ell;
  if (sizeof(T) == 4) {
    // FP32: tsqr_rows_kernel, 256 rows per block, 256 / n triangles per merge
    pl.rows0 = kRowsQR;
    pl.fan = std::max(2, kRowsQR / n);
    pl.nblk0 = ceil_div(pl.v.M(), kRowsQR);
    return;
  }
  const int budget = smem_budget() - (int)sizeof(T) * (kTsqrThreads + 64);
  int rows0 = budget / (int)(sizeof(T) * n) - 1;
  rows0 = std::min(rows0, 512);
  rows0 = std::max(rows0, 2 * n);
  pl.rows0 = rows0;
  pl.fan = std::max(2, rows0 / n);
  pl.nblk0 = ceil_div(pl.v.M(), rows0);
}

static int odd_ld(int rows) { return rows | 1; }

// one wave of the ell <= 64 Gram kernel (3 CTAs per SM): fewer per-CTA partials (ell^2 doubles each)
// for the reduce to read, and no tail wave
int gram_ctas() { return 3 * num_sms(); }

// W = B B^T (ell x ell, FP64, full) of the FP32 (L, ell, R) tensor B: FP32 sums over 128 columns,
// FP64 across; part holds min(gram_ctas(), ceil(L R / 128)) ell^2 doubles.  Gated on *gate == 0.
rh_status launch_gram_f32(const float* B, int64_t L, int64_t R, int ell, double* part, double* W,
                          const int32_t* gate, cudaStream_t st, bool df, int site) {
  const int64_t ntiles = ceil_div(L * R, 128);
  // one CTA per SM at least (a single matrix fills the GPU), beyond that at least tune(min_tiles) per
  // CTA: a CTA's set-up and its ell^2 FP64 partial (written here, read by the reduce) would
  // otherwise outweigh its work on the many small matrices of a batch
  const int ctas = (int)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(gram_ctas(), ntiles),
                           std::max<int64_t>(num_sms(), ceil_div(ntiles, tune(TUNE_GRAM_MIN_TILES)))));
  if (!df) {
    using G32 = GramBOp<32, false>;
    using G64 = GramBOp<64, false>;
    if (ell <= 32)
      RH_EMIT(G32, site, 0, ctas, GramCfg<32>::SMEM, B, L, R, ell, part, gate);
    else
      RH_EMIT(G64, site, 0, ctas, GramCfg<64>::SMEM, B, L, R, ell, part, gate);
  } else {
    // the double-float sums are ALU-bound: blocks of 4 x 4 entries over the columns actually used
    switch ((ell + 7) / 8) {
#define RH_GDF(E) \
  case E / 8: {                                                           \
    using GE = GramBOp<E, true>;                                          \
    RH_EMIT(GE, site, 0, ctas, GramCfg<E>::SMEM, B, L, R, ell, part, gate); \
  } break
      RH_GDF(8); RH_GDF(16); RH_GDF(24); RH_GDF(32); RH_GDF(40); RH_GDF(48); RH_GDF(56); RH_GDF(64);
#undef RH_GDF
      default:
        set_error("Gram matrix: ell must be in [1, 64]");
        return RH_EUNSUPPORTED;
    }
  }
  RH_EMIT(GramBReduceOp, site == SITE_OTHER ? SITE_OTHER : site + 1, 0, (int)ceil_div((int64_t)ell * ell, 32), 0,
          part, ctas, ell, W, gate);
  return RH_OK;
}

template <typename T>
size_t trunc_workspace_elems(const TruncPlan& pl0) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int64_t nn = (int64_t)pl.ell * pl.ell;
  // two ping-pong buffers of R's
  size_t e = (size_t)(pl.nblk0 * nn + ceil_div(pl.nblk0, pl.fan) * nn + 2 * nn) + 64;
  if (sizeof(T) == 4) {
    // Gram route: CTA partials, W, R, rdiag, flags (in doubles), the FP32 copy of R
    const size_t dbl = (size_t)gram_ctas() * nn + 2 * nn + pl.ell + 8;
    e += 2 * dbl + nn + 64;
  }
  return e;
}

// R of B^T (M x n) by the FP64 tree: a Householder QR per block of rows0 rows, then merges of fan
// triangles per level; *out points at the final triangle (buf0 or buf1).
template <typename T>
static rh_status launch_tsqr_tree(const TruncPlan& pl, const T* B, T* buf0, T* buf1, const int32_t* gate, T** out,
                                  cudaStream_t st, int site) {
  const int n = pl.ell;
  const int ld0 = odd_ld(pl.rows0);
  const int ldm = odd_ld(pl.fan * n);
  const size_t sm0 = sizeof(T) * ((size_t)ld0 * n + kTsqrThreads + 64);
  const size_t smm = sizeof(T) * ((size_t)ldm * n + kTsqrThreads + 64);
  const int64_t cap = 8 * (int64_t)num_sms();
  RH_EMIT(TsqrLeafOp<T>, site, 0, (unsigned)std::min<int64_t>(pl.nblk0, cap), sm0, B, pl.v.L, pl.v.R, n, pl.rows0, ld0,
          buf0, gate);
  int64_t cnt = pl.nblk0;
  T* cur = buf0;
  T* nxt = buf1;
  for (int lv = 1; cnt > 1; ++lv) {
    const int64_t nout = ceil_div(cnt, pl.fan);
    RH_EMIT(TsqrMergeOp<T>, site, lv, (unsigned)std::min<int64_t>(nout, cap), smm, cur, cnt, n, pl.fan, ldm, nxt, gate);
    cnt = nout;
    T* t = cur;
    cur = nxt;
    nxt = t;
  }
  *out = cur;
  return RH_OK;
}

double* trunc_gram_part(const TruncPlan& pl0, float* ws) {
  TruncPlan pl = pl0;
  trunc_dims<float>(pl);
  const int64_t nn = (int64_t)pl.ell * pl.ell;
  const size_t tsqr_elems = (size_t)(pl.nblk0 * nn + ceil_div(pl.nblk0, pl.fan) * nn + 2 * nn) + 64;
  return reinterpret_cast<double*>(ws + ((tsqr_elems + 63) & ~size_t(63)));
}

template <typename T>
rh_status launch_trunc_svd(const TruncPlan& pl0, const T* B, T* ws, double* Ub, double* sv, cudaStream_t st, int r,
                           int32_t* info, int gram_nparts) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int n = pl.ell;
  const int64_t nn = (int64_t)n * n;
  T* buf0 = ws;
  T* buf1 = ws + pl.nblk0 * nn;
  const int np = (n + 1) & ~1;
  const size_t smj = sizeof(T) * 4 * (size_t)np * 32 * 2;
  int32_t* use_tsqr = nullptr;
  if (sizeof(T) == 4 && r >= 1 && r <= n) {
    // Gram route (FP32 data): W = B B^T, R = chol(W)^T-factor, Jacobi on R; gated fallback below
    const size_t tsqr_elems = (size_t)(pl.nblk0 * nn + ceil_div(pl.nblk0, pl.fan) * nn + 2 * nn) + 64;
    double* dbase = reinterpret_cast<double*>(ws + ((tsqr_elems + 63) & ~size_t(63)));
    const int ctas = gram_ctas();
    double* part = dbase;
    double* W = part + (size_t)ctas * nn;
    double* Rd = W + nn;
    double* rdiag = Rd + nn;
    int32_t* flags = reinterpret_cast<int32_t*>(rdiag + n);
    float* Rf = reinterpret_cast<float*>(flags + 16);
    use_tsqr = flags + 1;
    int32_t* flags2 = flags + 4;   // second route: [0] = skip / Cholesky failure
    (void)ctas;
    rh_status s = emit_memset(SITE_TRUNC_ZERO, 0, flags, 8 * sizeof(int32_t), st);
    if (s != RH_OK) return s;
    if (gram_nparts > 0) {
      // the partials came with B (tensor-core mode product): their fixed-order reduction only
      RH_EMIT(GramBReduceOp, SITE_TRUNC_GRAM_REDUCE, 0, (int)ceil_div((int64_t)n * n, 32), 0, part, gram_nparts, n,
              W, nullptr);
    } else if ((s = launch_gram_f32(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, part, W, nullptr, st, false,
                                    SITE_TRUNC_GRAM)) != RH_OK) {
      return s;
    }
    RH_EMIT(PivotedCholeskyOp, SITE_TRUNC_PCHOL, 0, 1, chol_smem(n, sizeof(dfl::F2)), W, n, Rf, flags, nullptr);
    const size_t smr = sizeof(float) * (2 * 64 * 80 + 2 * 64 * 65);
    {
      ProfileScope ps(PROF_JACOBI, 0, st);
      RH_EMIT(JacobiRowsOp, SITE_TRUNC_JACOBI, 0, 1, smr, Rf, n, Ub, sv, flags, nullptr, 0);
    }
    RH_EMIT(TruncDecideOp, SITE_TRUNC_DECIDE, 0, 1, 0, flags, sv, n, r, use_tsqr, info, flags2);
    // Second route when the first is rejected: the same factorization of a double-float Gram
    // matrix (no gap test: its error is ~2^-44 ||W||).  Its Cholesky clears use_tsqr when it
    // succeeds, so the tall-skinny QR below only runs when it breaks down too.
    if ((s = launch_gram_f32(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, part, W, flags2, st, true,
                             SITE_TRUNC_GRAM_DF)) != RH_OK)
      return s;
    RH_EMIT(PivotedCholeskyOp, SITE_TRUNC_PCHOL2, 0, 1, chol_smem(n, sizeof(dfl::F2)), W, n, Rf, flags2, use_tsqr);
    {
      ProfileScope ps(PROF_JACOBI, 2, st);
      RH_EMIT(JacobiRowsOp, SITE_TRUNC_JACOBI2, 0, 1, smr, Rf, n, Ub, sv, flags2, info, 8);
    }
  }
  T* cur = buf0;
  if constexpr (sizeof(T) == 4) {
    float* fin = nullptr;
    rh_status s = launch_tsqr_rows(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, reinterpret_cast<float*>(buf0),
                                   reinterpret_cast<float*>(buf1), use_tsqr, &fin, st, SITE_TRUNC_TSQR);
    if (s != RH_OK) return s;
    cur = reinterpret_cast<T*>(fin);
  } else {
    rh_status s = launch_tsqr_tree<T>(pl, B, buf0, buf1, use_tsqr, &cur, st, SITE_TRUNC_TSQR);
    if (s != RH_OK) return s;
  }
  // Preconditioning (Drmac and Veselic): the column-pivoted QR of the tall-skinny triangle,
  // R P = Q2 R2, makes B^T P = (Q_B Q2) R2 a pivoted QR of B^T, and the one-sided Jacobi on R2^T
  // then converges in a few sweeps and keeps the small singular values' vectors accurate, where the
  // Jacobi on the unpivoted R of a graded spectrum runs to its sweep cap.  R2 and the permutation
  // sit after the two triangle buffers.
  T* R2 = buf1 + ceil_div(pl.nblk0, pl.fan) * nn;
  int32_t* piv = reinterpret_cast<int32_t*>(R2 + nn);
  RH_EMIT(PivQrOp<T>, SITE_TRUNC_PIVQR, 0, 1, 0, cur, n, R2, piv, use_tsqr, 1);
  {
    ProfileScope ps(PROF_JACOBI, 1, st);
    RH_EMIT(JacobiSvdOp<T>, SITE_TRUNC_JACOBI_SVD, 0, 1, smj, R2, n, Ub, sv, use_tsqr, 1, piv);
  }
  return RH_OK;
}

// ---- basis of a subspace-iteration step ----------------------------------------------------
template <typename T>
size_t power_workspace_elems(const TruncPlan& pl0) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int64_t nn = (int64_t)pl.ell * pl.ell;
  const size_t tsqr = (size_t)(pl.nblk0 * nn + ceil_div(pl.nblk0, pl.fan) * nn + 2 * nn) + 64;
  const size_t dbl = (size_t)gram_ctas() * nn + 3 * nn + pl.ell + 16;   // partials, C, R, rdiag, flag
  return ((tsqr + 63) & ~size_t(63)) + (dbl * sizeof(double) + sizeof(T) - 1) / sizeof(T) + 64;
}

// W = orth(B^T) in place (Sec. 5, randomized subspace iteration: the basis of range(G_(n)^T Q)),
// for B in the (L, n, R) view: R_1 from the tall-skinny Householder QR of B^T (backward stable
// whatever the conditioning), W_1 = B^T R_1^{-1}, then one CholeskyQR pass on W_1 (Gram matrix
// with FP64 sums, FP64 Cholesky, W = W_1 R_2^{-1}), skipped when that Cholesky breaks down (W_1
// numerically rank deficient; its zero columns stay zero).
template <typename T>
rh_status launch_power_basis(const TruncPlan& pl0, T* B, T* ws, cudaStream_t st) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int n = pl.ell;
  const int64_t nn = (int64_t)n * n;
  T* buf0 = ws;
  T* buf1 = ws + pl.nblk0 * nn;
  const size_t tsqr = (size_t)(pl.nblk0 * nn + ceil_div(pl.nblk0, pl.fan) * nn + 2 * nn) + 64;
  double* part = reinterpret_cast<double*>(ws + ((tsqr + 63) & ~size_t(63)));
  double* C = part + (size_t)gram_ctas() * nn;
  double* R2 = C + nn;
  double* rdiag = R2 + nn;
  int32_t* flag = reinterpret_cast<int32_t*>(rdiag + n + 8);
  rh_status s = emit_memset(SITE_POWER_ZERO, 0, flag, sizeof(int32_t), st);
  if (s != RH_OK) return s;
  T* Rt = nullptr;
  if constexpr (sizeof(T) == 4) {
    float* fin = nullptr;
    s = launch_tsqr_rows(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, reinterpret_cast<float*>(buf0),
                         reinterpret_cast<float*>(buf1), nullptr, &fin, st, SITE_POWER_TSQR);
    Rt = reinterpret_cast<T*>(fin);
  } else {
    s = launch_tsqr_tree<T>(pl, B, buf0, buf1, nullptr, &Rt, st, SITE_POWER_TSQR);
  }
  if (s != RH_OK) return s;
  const double tiny = (sizeof(T) == 4 ? 64.0 * 5.9604645e-8 : 64.0 * 1.1102230246251565e-16);
  const int tblocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pl.v.L * pl.v.R, 8), 8 * num_sms()));
  using TrsmW1 = TrsmViewOp<T, T>;
  using TrsmW2 = TrsmViewOp<T, double>;
  RH_EMIT(TrsmW1, SITE_POWER_TRSM, 0, tblocks, 0, B, pl.v.L, pl.v.R, n, Rt, nullptr, tiny);
  // second pass: Gram matrix of W_1 (FP64 sums), Cholesky, W = W_1 R_2^{-1}
  if constexpr (sizeof(T) == 4) {
    if ((s = launch_gram_f32(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, part, C, nullptr, st, false,
                             SITE_POWER_GRAM)) != RH_OK)
      return s;
  } else {
    const int64_t ntiles = ceil_div(pl.v.L * pl.v.R, 32);
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>(gram_ctas(), ntiles));
    RH_EMIT(GramViewF64Op, SITE_POWER_GRAM, 0, ctas, 0, reinterpret_cast<const double*>(B), pl.v.L, pl.v.R, n, part,
            nullptr);
    RH_EMIT(GramBReduceOp, SITE_POWER_GRAM + 1, 0, (int)ceil_div(nn, 32), 0, part, ctas, n, C, nullptr);
  }
  RH_EMIT(CholOp<ArithF64>, SITE_POWER_CHOL, 0, 1, chol_smem(n, sizeof(double)), C, n, R2, rdiag, flag, 0.0);
  RH_EMIT(TrsmW2, SITE_POWER_TRSM2, 0, tblocks, 0, B, pl.v.L, pl.v.R, n, R2, flag, tiny);
  return RH_OK;
}

// R of the tall-skinny Householder QR of B^T (B: the (L, n, R) view of tr), as an n x n FP64 upper
// triangle (zeros below the diagonal); ws holds trunc_workspace_elems(tr) elements of T.
__global__ void triangle_to_f64_kernel(const float* __restrict__ Rf, const double* __restrict__ Rd, int n,
                                       double* __restrict__ R) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int j = e % n, k = e / n;
    R[e] = j <= k ? (Rf ? (double)Rf[e] : Rd[e]) : 0.0;
  }
}

template <typename T>
rh_status launch_tall_skinny_r(const TruncPlan& pl0, const T* B, T* ws, double* R, cudaStream_t st) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int n = pl.ell;
  const int64_t nn = (int64_t)n * n;
  T* buf0 = ws;
  T* buf1 = ws + pl.nblk0 * nn;
  T* fin = nullptr;
  rh_status s;
  if constexpr (sizeof(T) == 4) {
    float* f = nullptr;
    s = launch_tsqr_rows(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, reinterpret_cast<float*>(buf0),
                         reinterpret_cast<float*>(buf1), nullptr, &f, st, SITE_OTHER);
    fin = reinterpret_cast<T*>(f);
  } else {
    s = launch_tsqr_tree<T>(pl, B, buf0, buf1, nullptr, &fin, st, SITE_OTHER);
  }
  if (s != RH_OK) return s;
  triangle_to_f64_kernel<<<(unsigned)std::max<int64_t>(1, ceil_div(nn, 256)), 256, 0, st>>>(
      sizeof(T) == 4 ? reinterpret_cast<const float*>(fin) : nullptr,
      sizeof(T) == 8 ? reinterpret_cast<const double*>(fin) : nullptr, n, R);
  RH_LAUNCH_CHECK();
  return RH_OK;
}
template rh_status launch_tall_skinny_r<float>(const TruncPlan&, const float*, float*, double*, cudaStream_t);
template rh_status launch_tall_skinny_r<double>(const TruncPlan&, const double*, double*, double*, cudaStream_t);

// ---- staged truncation (adaptive variants) ----------------------------------------------
template <typename T>
rh_status launch_trunc_factor(const TruncPlan& pl0, const T* B, T* ws, bool gram, double* part, double* W, T** R,
                              double* rownorm2, cudaStream_t st, bool df) {
  TruncPlan pl = pl0;
  trunc_dims<T>(pl);
  const int n = pl.ell;
  const int64_t nn = (int64_t)n * n;
  if (gram) {
    rh_status s = launch_gram_f32(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, part, W, nullptr, st, df,
                                  SITE_OTHER);
    if (s != RH_OK) return s;
    diag_kernel<<<1, 64, 0, st>>>(W, n, rownorm2);
    RH_LAUNCH_CHECK();
    return RH_OK;
  }
  T* buf0 = ws;
  T* buf1 = ws + pl.nblk0 * nn;
  T* cur = buf0;
  if constexpr (sizeof(T) == 4) {
    float* fin = nullptr;
    rh_status s = launch_tsqr_rows(reinterpret_cast<const float*>(B), pl.v.L, pl.v.R, n, reinterpret_cast<float*>(buf0),
                                   reinterpret_cast<float*>(buf1), nullptr, &fin, st, SITE_OTHER);
    if (s != RH_OK) return s;
    cur = reinterpret_cast<T*>(fin);
  } else {
    rh_status s = launch_tsqr_tree<T>(pl, B, buf0, buf1, nullptr, &cur, st, SITE_OTHER);
    if (s != RH_OK) return s;
  }
  *R = cur;
  colnorm2_kernel<T><<<n, 32, 0, st>>>(cur, n, rownorm2);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template <typename T>
rh_status launch_trunc_leading_svd(int n, int k, bool gram, const double* W, const T* R, double* Wk, float* Xf,
                                   T* Rk, double* Ub, double* sv, int32_t* flag, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, ceil_div((int64_t)k * k, 256));
  if (gram) {
    RH_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), st));
    copy_leading_kernel<double, double><<<blocks, 256, 0, st>>>(W, n, k, Wk);
    RH_LAUNCH_CHECK();
    RH_EMIT(PivotedCholeskyOp, SITE_OTHER, 0, 1, chol_smem(k, sizeof(dfl::F2)), Wk, k, Xf, flag, nullptr);
    const size_t smr = sizeof(float) * (2 * 64 * 80 + 2 * 64 * 65);
    RH_EMIT(JacobiRowsOp, SITE_OTHER, 0, 1, smr, Xf, k, Ub, sv, flag, nullptr, 0);
    return RH_OK;
  }
  copy_leading_kernel<T, T><<<blocks, 256, 0, st>>>(R, n, k, Rk);
  RH_LAUNCH_CHECK();
  const int np = (k + 1) & ~1;
  const size_t smj = sizeof(T) * 4 * (size_t)np * 32 * 2;
  RH_EMIT(JacobiSvdOp<T>, SITE_OTHER, 0, 1, smj, Rk, k, Ub, sv, nullptr, 0, nullptr);
  return RH_OK;
}

template <typename T>
rh_status launch_factor_and_cast(int64_t I, int ell, int r, const double* Q, const double* Ub, double* A, T* Uc,
                                 cudaStream_t st) {
  const int64_t total = std::max<int64_t>(I * r, (int64_t)ell * r);
  const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 8 * num_sms());
  RH_EMIT(FactorCastOp<T>, SITE_FACTOR, 0, blocks, 0, I, ell, r, Q, Ub, A, Uc);
  RH_EMIT(ColsignOp<T>, SITE_FACTOR_SIGN, 0, r, 0, A, I, r, Uc, ell);
  return RH_OK;
}

template <typename T>
rh_status launch_cast(const double* src, T* dst, int64_t n, cudaStream_t st, int site) {
  const int blocks = (int)std::min<int64_t>(ceil_div(n, 256), 8 * num_sms());
  RH_EMIT(CastOp<T>, site, 0, std::max(blocks, 1), 0, src, dst, n);
  return RH_OK;
}

rh_status launch_sumsq(const double* x, int64_t n, double* out, cudaStream_t st, double* part, size_t part_elems) {
  if (part != nullptr && part_elems >= 2 && n > 16384) {
    const int64_t G = std::min<int64_t>(std::min<int64_t>((int64_t)part_elems, 256), ceil_div(n, 4096));
    const int64_t chunk = ceil_div(n, G);
    const int64_t gg = ceil_div(n, chunk);
    RH_EMIT(SumsqPartOp, SITE_FINAL, 0, (int)gg, 0, x, n, chunk, part);
    RH_EMIT(SumPartsOp, SITE_FINAL, 1, 1, 0, part, (int)gg, out);
    return RH_OK;
  }
  RH_EMIT(SumsqOp, SITE_FINAL, 0, 1, 0, x, n, out);
  return RH_OK;
}

template size_t trunc_workspace_elems<float>(const TruncPlan&);
template size_t trunc_workspace_elems<double>(const TruncPlan&);
template rh_status launch_trunc_svd<float>(const TruncPlan&, const float*, float*, double*, double*, cudaStream_t, int,
                                           int32_t*, int);
template rh_status launch_trunc_svd<double>(const TruncPlan&, const double*, double*, double*, double*, cudaStream_t,
                                            int, int32_t*, int);
template rh_status launch_trunc_factor<float>(const TruncPlan&, const float*, float*, bool, double*, double*, float**,
                                             double*, cudaStream_t, bool);
template rh_status launch_trunc_factor<double>(const TruncPlan&, const double*, double*, bool, double*, double*,
                                              double**, double*, cudaStream_t, bool);
template rh_status launch_trunc_leading_svd<float>(int, int, bool, const double*, const float*, double*, float*, float*,
                                                  double*, double*, int32_t*, cudaStream_t);
template rh_status launch_trunc_leading_svd<double>(int, int, bool, const double*, const double*, double*, float*,
                                                   double*, double*, double*, int32_t*, cudaStream_t);
template rh_status launch_factor_and_cast<float>(int64_t, int, int, const double*, const double*, double*, float*,
                                                 cudaStream_t);
template rh_status launch_factor_and_cast<double>(int64_t, int, int, const double*, const double*, double*, double*,
                                                  cudaStream_t);
template rh_status launch_cast<float>(const double*, float*, int64_t, cudaStream_t, int);
template rh_status launch_cast<double>(const double*, double*, int64_t, cudaStream_t, int);
template size_t power_workspace_elems<float>(const TruncPlan&);
template size_t power_workspace_elems<double>(const TruncPlan&);
template rh_status launch_power_basis<float>(const TruncPlan&, float*, float*, cudaStream_t);
template rh_status launch_power_basis<double>(const TruncPlan&, double*, double*, cudaStream_t);

}  // namespace rh
