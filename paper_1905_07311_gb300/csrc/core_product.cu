// Truncated core of one R-STHOSVD mode (Alg. 1 step 6 inside Alg. 3): G_(n) <- U_r^T B with
// B = Q^T G_(n) the ell x M mode product (column p at B + ell p) and U_r the leading r columns of
// U_B (ell x r, column-major).  The output order is a CoreOut: the usual column-major core, or the
// core with the next mode m first and the other modes in increasing order, so that the next
// unfolding is read with unit stride and its Kolda column order (Omega's rows) is unchanged.
//
// A CTA takes 128 consecutive columns: the 128 x ell slice of B is read with 16-byte loads and
// stored transposed in shared memory, U_r stays in shared memory, and each of the 256 threads
// accumulates a 4 (c) x 8 (p) register tile in FP32 (sums over ell <= 64 terms).
#include "common.cuh"
#include "kernels.cuh"

namespace rh {
namespace {

constexpr int kCpTile = 128;   // columns per CTA
constexpr int kCpLd = kCpTile + 4;

template <typename TO>
__global__ void __launch_bounds__(256) core_product_kernel(const float* __restrict__ B, int ell, int ko, int64_t M,
                                                           CoreOut co, const float* __restrict__ U,
                                                           TO* __restrict__ out) {
  extern __shared__ __align__(16) float cp_smem[];
  float* Bt = cp_smem;                      // [64][kCpLd]: Bt[k][p]
  float* Us = Bt + 64 * kCpLd;              // [64][64]:   Us[k][c]
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * 64; e += 256) {
    const int k = e >> 6, c = e & 63;
    Us[e] = (k < ell && c < ko) ? U[k + ell * c] : 0.0f;
  }
  const int cg = tid >> 4;           // c = 4 cg .. 4 cg + 3
  const int pl = tid & 15;           // p = 4 pl + {0..3} and 64 + 4 pl + {0..3}
  const int64_t ntiles = (M + kCpTile - 1) / kCpTile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t p0 = t * kCpTile;
    const int valid = (int)(M - p0 < kCpTile ? M - p0 : kCpTile);
    __syncthreads();
    {
      // the slice is valid * ell contiguous values starting at B + ell p0
      const float* src = B + (int64_t)ell * p0;
      const int n = valid * ell;
      const bool vec = ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
      for (int e = 4 * tid; e < kCpTile * ell; e += 4 * 256) {
        float v[4];
        if (vec && e + 3 < n) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(src + e));
          v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) v[j] = (e + j < n) ? src[e + j] : 0.0f;
        }
        int p = e / ell, k = e - p * ell;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (p < kCpTile) Bt[k * kCpLd + p] = v[j];
          if (++k == ell) {
            k = 0;
            ++p;
          }
        }
      }
      // rows k >= ell stay zero
      for (int e = tid; e < (64 - ell) * kCpTile; e += 256) Bt[(ell + e / kCpTile) * kCpLd + e % kCpTile] = 0.0f;
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
    for (int k = 0; k < ell; ++k) {
      const float4 u = *reinterpret_cast<const float4*>(&Us[k * 64 + 4 * cg]);
      const float4 x0 = *reinterpret_cast<const float4*>(&Bt[k * kCpLd + 4 * pl]);
      const float4 x1 = *reinterpret_cast<const float4*>(&Bt[k * kCpLd + 64 + 4 * pl]);
      const float uu[4] = {u.x, u.y, u.z, u.w};
      const float xx[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(uu[a], xx[b], acc[a][b]);
    }
    const int64_t cs = co.cstride();
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int pp = (b < 4 ? 4 * pl + b : 64 + 4 * pl + (b - 4));
      if (pp >= valid) continue;
      const int64_t base = co.base(p0 + pp, ko);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int c = 4 * cg + a;
        if (c < ko) out[base + cs * c] = (TO)acc[a][b];
      }
    }
  }
}

}  // namespace

size_t core_product_smem() { return sizeof(float) * (64 * kCpLd + 64 * 64); }

template <typename TO>
rh_status launch_core_product(const float* B, int ell, int ko, int64_t M, CoreOut co, const float* U, TO* out,
                              cudaStream_t st) {
  if (ell < 1 || ell > 64 || ko < 1 || ko > 64 || co.S < 1 || co.I < 1 || co.Ln < 1 || M % (co.S * co.I) != 0) {
    set_error("core product: bad shape");
    return RH_EINVAL;
  }
  const size_t smem = core_product_smem();
  RH_CUDA_TRY(cudaFuncSetAttribute(core_product_kernel<TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ntiles = ceil_div(M, kCpTile);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, 3 * (int64_t)num_sms()));
  core_product_kernel<TO><<<grid, 256, smem, st>>>(B, ell, ko, M, co, U, out);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template rh_status launch_core_product<float>(const float*, int, int, int64_t, CoreOut, const float*, float*,
                                              cudaStream_t);
template rh_status launch_core_product<double>(const float*, int, int, int64_t, CoreOut, const float*, double*,
                                               cudaStream_t);

}  // namespace rh
