// Structure-preserving STHOSVD on a COO tensor (Alg. 6, SP-STHOSVD, Sec. 5).
//
// Per mode n in the processing order, on the current sparse core G (COO, 0-based, deduplicated):
//   Y = G_(n) Omega_n       sketch straight from the nonzeros (step 4): nonzero (i_1..i_d, v)
//                           adds v Omega_n(p, :) to row i_n, p its Kolda column index
//   Y = Q R                 thin QR (step 5, CholeskyQR2 / Householder)
//   P_n = sRRQR(Q^T)        ell_n rows of Q, max |A_ij| <= eta = 2 (step 6)
//   A_n = Q (P_n^T Q)^{-1}  (step 7)
//   G_(n) <- P_n^T G_(n)    keep the nonzeros whose mode-n index is selected and renumber it to
//                           its position in the sorted selection (step 8): G stays sparse
// and finally the dense ell_1 x ... x ell_d core of the surviving entries.
//
// The sketch is deterministic: the nonzeros are stably sorted by i_n (CUB radix sort), each row's
// run is cut into work items of at most kItem nonzeros, a warp turns an item into a partial row
// (FP32 sums of products; ceil(ell / 4) lanes per nonzero, lane q handling Omega columns
// 4q..4q+3, 32 / ceil(ell / 4) nonzeros per pass, the groups combined in a fixed order), and the
// partials of a row are added in FP64 in item order.
// Omega rows are shared: a row p of Omega_n (a Kolda column of the unfolding) is needed by every
// nonzero with the same other-mode coordinates, and a count tensor repeats them often (a Zipf
// tensor needs 0.17 to 0.27 distinct rows per nonzero).  When the unfolding has fewer than 2^31
// columns the nonzeros are also sorted by p, each distinct row is generated once into a table
// (FP32, or BF16 in the BF16-Omega form) and the work items read it from there; otherwise every
// nonzero generates its row.  Both give the same normals, so the same sums.  The item list is built on the host from the row counts, and the selection
// (strong RRQR: column-pivoted QR of Q^T, then swaps while some |A_ij| > eta, the largest entry first,
// lowest (i, j) on ties) runs on the host in FP64, so the call synchronises its stream per mode.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "philox.cuh"
#include "tc.cuh"

namespace rh {
namespace {

constexpr int kItem = 512;   // nonzeros per work item of the sketch

__global__ void iota_kernel(int32_t* __restrict__ a, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    a[e] = (int32_t)e;
}

// Keys outside [0, I) are counted in *bad (one atomic per block; the host turns a nonzero count
// into RH_EINVAL before any kernel uses a key as an address).
__global__ void __launch_bounds__(256) bad_keys_kernel(const int32_t* __restrict__ key, int64_t n, int64_t I,
                                                       int32_t* __restrict__ bad) {
  __shared__ int32_t cnt_s;
  if (threadIdx.x == 0) cnt_s = 0;
  __syncthreads();
  int32_t c = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = key[e];
    c += (k < 0 || k >= I) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt_s, c);
  __syncthreads();
  if (threadIdx.x == 0 && cnt_s) atomicAdd(bad, cnt_s);
}

// Row runs of the sorted keys: begin[r] and end[r] of row r's run; rows without entries keep their
// zero fill.  No atomics, so a heavy row (a Zipf index) costs nothing extra.  Keys outside [0, I)
// are skipped (never used as addresses; bad_keys_kernel reports them).
__global__ void run_bounds_kernel(const int32_t* __restrict__ ks, int64_t n, int64_t I, int32_t* __restrict__ begin,
                                  int32_t* __restrict__ end) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = ks[k];
    if (r < 0 || r >= I) continue;
    if (k == 0 || ks[k - 1] != r) begin[r] = (int32_t)k;
    if (k == n - 1 || ks[k + 1] != r) end[r] = (int32_t)(k + 1);
  }
}

// cnt[r] = end[r] - begin[r] for r < I (cnt holds the ends on entry)
__global__ void run_counts_kernel(const int32_t* __restrict__ begin, int64_t I, int32_t* __restrict__ cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < I; r += (int64_t)gridDim.x * blockDim.x)
    cnt[r] -= begin[r];
}

struct SpIdx {
  const int32_t* idx[RH_MAX_ORDER];
  int64_t stride[RH_MAX_ORDER];   // Kolda stride of each mode in the mode-n unfolding (0 for n)
};

// Kolda column index p of every nonzero in the mode-n unfolding (stride 0 for mode n), < 2^31
__global__ void kolda_key_kernel(SpIdx ix, int d, int64_t n, int32_t* __restrict__ key) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = 0;
    for (int k = 0; k < d; ++k) p += (int64_t)ix.idx[k][e] * ix.stride[k];
    key[e] = (int32_t)p;
  }
}

// head[k] = 1 where the sorted key changes (a new distinct Omega row)
__global__ void run_heads_kernel(const int32_t* __restrict__ ks, int64_t n, int32_t* __restrict__ head) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    head[k] = (k == 0 || ks[k] != ks[k - 1]) ? 1 : 0;
}

// u1 = inclusive sum of the heads: nonzero es[k] uses distinct row u1[k] - 1, whose Omega row is
// pd[u] = ks[k]
__global__ void distinct_rows_kernel(const int32_t* __restrict__ ks, const int32_t* __restrict__ es,
                                     const int32_t* __restrict__ head, const int32_t* __restrict__ u1, int64_t n,
                                     int32_t* __restrict__ uid, int32_t* __restrict__ pd) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = u1[k] - 1;
    uid[es[k]] = u;
    if (head[k]) pd[u] = ks[k];
  }
}

// Table of the distinct Omega rows: row u (of *count) holds Omega_n(pd[u], 0 .. 4 nq - 1) at
// tab[u ldo ...], FP32 or rounded to BF16 (ties to even).
template <bool BF16>
__global__ void omega_table_kernel(const int32_t* __restrict__ pd, const int32_t* __restrict__ count, int nq, int ldo,
                                   uint32_t k0, uint32_t k1, uint32_t sid, void* __restrict__ tab) {
  const int64_t total = (int64_t)(*count) * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / nq;
    const int q = (int)(t - u * nq);
    const float4 w = rng::omega4(k0, k1, sid, pd[u], (uint32_t)q);
    if constexpr (BF16) {
      const uint32_t a = (uint32_t)tc::bf16_rne(w.x) | ((uint32_t)tc::bf16_rne(w.y) << 16);
      const uint32_t b = (uint32_t)tc::bf16_rne(w.z) | ((uint32_t)tc::bf16_rne(w.w) << 16);
      reinterpret_cast<uint2*>(tab)[(u * ldo + 4 * q) / 4] = make_uint2(a, b);
    } else {
      reinterpret_cast<float4*>(tab)[(u * ldo + 4 * q) / 4] = w;
    }
  }
}

// Source of the Omega columns 4q..4q+3 of a nonzero: generated (SRC 0), generated and rounded to
// BF16 (1), or read from the table of distinct rows, FP32 (2) or BF16 (3).
template <int SRC>
__device__ __forceinline__ float4 omega_quad(const SpIdx& ix, int d, int e, int q, uint32_t k0, uint32_t k1,
                                             uint32_t sid, const int32_t* __restrict__ uid, const void* __restrict__ tab,
                                             int ldo) {
  if constexpr (SRC <= 1) {
    int64_t p = 0;
    for (int k = 0; k < d; ++k) p += (int64_t)ix.idx[k][e] * ix.stride[k];
    float4 w = rng::omega4(k0, k1, sid, p, (uint32_t)q);
    if constexpr (SRC == 1) {
      w.x = tc::bf16_to_f(tc::bf16_rne(w.x));
      w.y = tc::bf16_to_f(tc::bf16_rne(w.y));
      w.z = tc::bf16_to_f(tc::bf16_rne(w.z));
      w.w = tc::bf16_to_f(tc::bf16_rne(w.w));
    }
    return w;
  } else if constexpr (SRC == 2) {
    return __ldg(reinterpret_cast<const float4*>(tab) + ((int64_t)uid[e] * ldo + 4 * q) / 4);
  } else {
    const uint2 r = __ldg(reinterpret_cast<const uint2*>(tab) + ((int64_t)uid[e] * ldo + 4 * q) / 4);
    return make_float4(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u), __uint_as_float(r.y << 16),
                       __uint_as_float(r.y & 0xFFFF0000u));
  }
}

// Warp per work item (row, [begin, end) of the sorted nonzeros): partial row of Y in FP64.
template <int SRC>
__global__ void __launch_bounds__(256) sp_sketch_items_kernel(SpIdx ix, int d, const float* __restrict__ vals,
                                                              const int32_t* __restrict__ perm,
                                                              const int3* __restrict__ items, int nitems, int ell,
                                                              uint32_t k0, uint32_t k1, uint32_t sid,
                                                              const int32_t* __restrict__ uid,
                                                              const void* __restrict__ tab, int ldo,
                                                              double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  // nq lanes per nonzero (lane q generates Omega columns 4q..4q+3), npass = 32 / nq nonzeros
  // per pass of the warp: ell = 40 keeps 30 of 32 lanes busy
  const int nq = (ell + 3) >> 2;
  const int npass = 32 / nq;
  const int g = lane / nq, q = lane - g * nq;
  const bool active = g < npass;
  for (int it = warp; it < nitems; it += nwarps) {
    const int3 item = items[it];   // x: row (unused here), y: begin, z: end
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (active) {
      for (int j = item.y + g; j < item.z; j += npass) {
        const int e = perm[j];
        const float v = vals[e];
        const float4 w = omega_quad<SRC>(ix, d, e, q, k0, k1, sid, uid, tab, ldo);
        acc[0] = fmaf(v, w.x, acc[0]);
        acc[1] = fmaf(v, w.y, acc[1]);
        acc[2] = fmaf(v, w.z, acc[2]);
        acc[3] = fmaf(v, w.w, acc[3]);
      }
    }
    // group 0 adds the other groups' sums in a fixed order
    for (int s = 1; s < npass; ++s) {
      const int src = (lane + s * nq) & 31;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float o = __shfl_sync(0xffffffffu, acc[c], src);
        if (g == 0) acc[c] += o;
      }
    }
    if (g == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (4 * q + c < ell) part[(int64_t)it * ell + 4 * q + c] = (double)acc[c];
    }
  }
}

// Y[r, c] = sum of the partials of row r's items (rows without items: 0).  CTA per row: lane l of
// warp w owns columns l and l + 32 and sums the items w, w + 8, w + 16, ... of the row in four
// interleaved chains (independent loads in flight), then warp 0 adds the eight warp sums in order:
// a fixed summation order, so the result is deterministic, and a heavy row (a Zipf index can hold
// thousands of items) is spread over 256 threads instead of one serial chain per column.
constexpr int kRedRowWarps = 8;
__global__ void __launch_bounds__(32 * kRedRowWarps) sp_sketch_reduce_kernel(const double* __restrict__ part,
                                                                             const int32_t* __restrict__ row_items,
                                                                             int64_t I, int ell,
                                                                             double* __restrict__ Y) {
  __shared__ double red[kRedRowWarps][2][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t r = blockIdx.x; r < I; r += gridDim.x) {
    const int b = row_items[r], e = row_items[r + 1];
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      double ch[4] = {0.0, 0.0, 0.0, 0.0};
      if (c < ell) {
        int it = b + w;
        for (; it + 3 * kRedRowWarps < e; it += 4 * kRedRowWarps) {
#pragma unroll
          for (int j = 0; j < 4; ++j) ch[j] += part[(int64_t)(it + j * kRedRowWarps) * ell + c];
        }
        for (; it < e; it += kRedRowWarps) ch[0] += part[(int64_t)it * ell + c];
      }
      red[w][h][lane] = (ch[0] + ch[1]) + (ch[2] + ch[3]);
    }
    __syncthreads();
    if (w == 0) {
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        double t = red[0][h][lane];
#pragma unroll
        for (int k = 1; k < kRedRowWarps; ++k) t += red[k][h][lane];
        if (c < ell) Y[r + I * c] = t;
      }
    }
    __syncthreads();
  }
}

__global__ void keep_flags_kernel(const int32_t* __restrict__ key, int64_t n, const int32_t* __restrict__ pos,
                                  int32_t* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = pos[key[e]] >= 0 ? 1 : 0;
}

// stable compaction of the kept nonzeros; mode n's index is renumbered through pos
__global__ void compact_kernel(SpIdx in, int d, int n, const float* __restrict__ vals, int64_t nnz,
                               const int32_t* __restrict__ flag, const int32_t* __restrict__ dest,
                               const int32_t* __restrict__ pos, SpIdx out, float* __restrict__ out_vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[e]) continue;
    const int64_t t = dest[e];
    for (int k = 0; k < d; ++k) {
      const int32_t v = in.idx[k][e];
      const_cast<int32_t*>(out.idx[k])[t] = (k == n) ? pos[v] : v;
    }
    out_vals[t] = vals[e];
  }
}

struct PosTabs {
  const int32_t* pos[RH_MAX_ORDER];   // position of each index in its mode's sorted selection, or -1
};

// SP-HOSVD: keep the nonzeros whose every index is selected
__global__ void keep_all_kernel(SpIdx in, int d, int64_t n, PosTabs pt, int32_t* __restrict__ flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int keep = 1;
    for (int k = 0; k < d; ++k) keep &= pt.pos[k][in.idx[k][e]] >= 0 ? 1 : 0;
    flag[e] = keep;
  }
}

// stable compaction of the kept nonzeros with every index renumbered through its mode's table
__global__ void compact_all_kernel(SpIdx in, int d, const float* __restrict__ vals, int64_t nnz,
                                   const int32_t* __restrict__ flag, const int32_t* __restrict__ dest, PosTabs pt,
                                   SpIdx out, float* __restrict__ out_vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[e]) continue;
    const int64_t t = dest[e];
    for (int k = 0; k < d; ++k) const_cast<int32_t*>(out.idx[k])[t] = pt.pos[k][in.idx[k][e]];
    out_vals[t] = vals[e];
  }
}

__global__ void scatter_core_kernel(SpIdx ix, int d, const float* __restrict__ vals, int64_t nnz,
                                    double* __restrict__ core) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t off = 0;
    for (int k = 0; k < d; ++k) off += (int64_t)ix.idx[k][e] * ix.stride[k];
    core[off] = (double)vals[e];
  }
}

__global__ void sumsq_f32_kernel(const float* __restrict__ v, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)v[e], (double)v[e], s);
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

__global__ void sum_parts_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t += part[k];
    *out = t;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 8 * num_sms())); }

// ---- host: subset selection on Q (FP64): strong RRQR, column-pivoted QR, DEIM ------------------
// inv (ell x ell, column-major) of the rows sel of Q (I x ell, column-major); false if singular
bool invert_rows(const std::vector<double>& Q, int64_t I, int ell, const std::vector<int>& sel,
                 std::vector<double>& inv) {
  std::vector<double> M((size_t)ell * ell);
  for (int a = 0; a < ell; ++a)
    for (int c = 0; c < ell; ++c) M[a + (size_t)ell * c] = Q[sel[a] + I * c];
  inv.assign((size_t)ell * ell, 0.0);
  for (int a = 0; a < ell; ++a) inv[a + (size_t)ell * a] = 1.0;
  for (int c = 0; c < ell; ++c) {   // Gauss-Jordan, partial pivoting
    int pr = c;
    for (int a = c + 1; a < ell; ++a)
      if (std::fabs(M[a + (size_t)ell * c]) > std::fabs(M[pr + (size_t)ell * c])) pr = a;
    if (M[pr + (size_t)ell * c] == 0.0) return false;
    if (pr != c)
      for (int k = 0; k < ell; ++k) {
        std::swap(M[c + (size_t)ell * k], M[pr + (size_t)ell * k]);
        std::swap(inv[c + (size_t)ell * k], inv[pr + (size_t)ell * k]);
      }
    const double piv = 1.0 / M[c + (size_t)ell * c];
    for (int k = 0; k < ell; ++k) {
      M[c + (size_t)ell * k] *= piv;
      inv[c + (size_t)ell * k] *= piv;
    }
    for (int a = 0; a < ell; ++a) {
      if (a == c) continue;
      const double f = M[a + (size_t)ell * c];
      if (f == 0.0) continue;
      for (int k = 0; k < ell; ++k) {
        M[a + (size_t)ell * k] -= f * M[c + (size_t)ell * k];
        inv[a + (size_t)ell * k] -= f * inv[c + (size_t)ell * k];
      }
    }
  }
  return true;
}

// A = Q inv (I x ell)
void apply_inv(const std::vector<double>& Q, int64_t I, int ell, const std::vector<double>& inv,
               std::vector<double>& A) {
  A.assign((size_t)I * ell, 0.0);
  for (int c = 0; c < ell; ++c)
    for (int k = 0; k < ell; ++k) {
      const double f = inv[k + (size_t)ell * c];
      if (f == 0.0) continue;
      const double* q = &Q[(size_t)I * k];
      double* a = &A[(size_t)I * c];
      for (int64_t i = 0; i < I; ++i) a[i] += q[i] * f;
    }
}

// Column-pivoted Householder QR of Q^T (ell x I; column i is row i of Q): the ell pivots, in order
// (largest remaining column norm, lowest index on ties).
rh_status cpqr_rows_host(const std::vector<double>& Q, int64_t I, int ell, std::vector<int>& sel) {
  std::vector<double> W((size_t)ell * I);
  for (int64_t i = 0; i < I; ++i)
    for (int c = 0; c < ell; ++c) W[c + (size_t)ell * i] = Q[i + I * c];
  std::vector<char> taken(I, 0);
  sel.clear();
  std::vector<double> v(ell);
  for (int s = 0; s < ell; ++s) {
    int64_t best = -1;
    double bn = -1.0;
    for (int64_t i = 0; i < I; ++i) {
      if (taken[i]) continue;
      double nrm = 0.0;
      for (int a = s; a < ell; ++a) nrm += W[a + (size_t)ell * i] * W[a + (size_t)ell * i];
      if (nrm > bn) {
        bn = nrm;
        best = i;
      }
    }
    if (best < 0) {   // every remaining norm is NaN
      set_error("subset selection: Q holds non-finite values");
      return RH_ENUMERIC;
    }
    taken[best] = 1;
    sel.push_back((int)best);
    // Householder reflector of W[s:, best], applied to every column
    double alpha = 0.0;
    for (int a = s; a < ell; ++a) alpha += W[a + (size_t)ell * best] * W[a + (size_t)ell * best];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = W[s + (size_t)ell * best];
    const double beta = x0 >= 0 ? -alpha : alpha;
    for (int a = s; a < ell; ++a) v[a] = W[a + (size_t)ell * best];
    v[s] -= beta;
    double vv = 0.0;
    for (int a = s; a < ell; ++a) vv += v[a] * v[a];
    if (vv == 0.0) continue;
    for (int64_t i = 0; i < I; ++i) {
      double dot = 0.0;
      for (int a = s; a < ell; ++a) dot += v[a] * W[a + (size_t)ell * i];
      const double f = 2.0 * dot / vv;
      for (int a = s; a < ell; ++a) W[a + (size_t)ell * i] -= f * v[a];
    }
  }
  return RH_OK;
}

// Solves the j x j system M c = b in place (M column-major, Gaussian elimination with partial
// pivoting); false if a pivot is zero or not finite.
bool solve_small(std::vector<double>& M, int j, std::vector<double>& b) {
  for (int c = 0; c < j; ++c) {
    int pr = c;
    for (int a = c + 1; a < j; ++a)
      if (std::fabs(M[a + (size_t)j * c]) > std::fabs(M[pr + (size_t)j * c])) pr = a;
    const double pv = M[pr + (size_t)j * c];
    if (pv == 0.0 || !std::isfinite(pv)) return false;
    if (pr != c) {
      for (int k = 0; k < j; ++k) std::swap(M[c + (size_t)j * k], M[pr + (size_t)j * k]);
      std::swap(b[c], b[pr]);
    }
    for (int a = c + 1; a < j; ++a) {
      const double f = M[a + (size_t)j * c] / pv;
      if (f == 0.0) continue;
      for (int k = c; k < j; ++k) M[a + (size_t)j * k] -= f * M[c + (size_t)j * k];
      b[a] -= f * b[c];
    }
  }
  for (int c = j - 1; c >= 0; --c) {
    double t = b[c];
    for (int k = c + 1; k < j; ++k) t -= M[c + (size_t)j * k] * b[k];
    b[c] = t / M[c + (size_t)j * c];
  }
  return true;
}

// DEIM (Chaturantabut and Sorensen 2010; Sorensen and Embree 2016): the first index is the largest
// |Q(i, 0)|; index j is the largest |r| of the residual r = Q(:, j) - Q(:, 0:j) c of interpolating
// column j at the indices chosen so far, Q(P, 0:j) c = Q(P, j) (lowest index on ties).
rh_status deim_rows_host(const std::vector<double>& Q, int64_t I, int ell, std::vector<int>& sel) {
  sel.clear();
  std::vector<double> M, c;
  for (int j = 0; j < ell; ++j) {
    const double* qj = &Q[(size_t)I * j];
    std::vector<double> r(qj, qj + I);
    if (j > 0) {
      M.assign((size_t)j * j, 0.0);
      c.assign(j, 0.0);
      for (int a = 0; a < j; ++a) {
        for (int k = 0; k < j; ++k) M[a + (size_t)j * k] = Q[sel[a] + (size_t)I * k];
        c[a] = qj[sel[a]];
      }
      if (!solve_small(M, j, c)) {
        set_error("subset selection: DEIM met a singular interpolation matrix (Q is rank deficient)");
        return RH_ENUMERIC;
      }
      for (int k = 0; k < j; ++k) {
        const double f = c[k];
        const double* qk = &Q[(size_t)I * k];
        for (int64_t i = 0; i < I; ++i) r[i] -= qk[i] * f;
      }
    }
    int64_t best = -1;
    double bm = -1.0;
    for (int64_t i = 0; i < I; ++i)
      if (std::fabs(r[i]) > bm) {
        bm = std::fabs(r[i]);
        best = i;
      }
    if (best < 0 || bm == 0.0) {
      set_error(best < 0 ? "subset selection: Q holds non-finite values"
                         : "subset selection: DEIM residual vanished (Q is rank deficient)");
      return RH_ENUMERIC;
    }
    sel.push_back((int)best);
  }
  return RH_OK;
}

// sRRQR swaps on a start selection: while some |A_ij| > eta on an unselected row, row i replaces
// selected row j for the largest |A_ij| (lowest (i, j) on ties); at most 100000 swaps.
rh_status srrqr_swaps_host(const std::vector<double>& Q, int64_t I, int ell, double eta, std::vector<int>& sel) {
  std::vector<double> inv, A;
  for (int sw = 0; sw < 100000; ++sw) {
    if (!invert_rows(Q, I, ell, sel, inv)) {
      set_error("subset selection: the selected rows of Q are singular");
      return RH_ENUMERIC;
    }
    apply_inv(Q, I, ell, inv, A);
    std::vector<char> in(I, 0);
    for (int x : sel) in[x] = 1;
    double amax = 0.0;
    int64_t bi = -1;
    int bj = -1;
    for (int64_t i = 0; i < I; ++i) {
      if (in[i]) continue;
      for (int j = 0; j < ell; ++j) {
        const double a = std::fabs(A[i + (size_t)I * j]);
        if (a > amax) {
          amax = a;
          bi = i;
          bj = j;
        }
      }
    }
    if (amax <= eta) break;
    sel[bj] = (int)bi;
  }
  return RH_OK;
}

// Sorts the selection and forms A = Q (P^T Q)^{-1}, storing A(P, :) as the exact identity (it is one in
// exact arithmetic), so that a decomposition with this factor reproduces the selected entries.
rh_status interp_factor_host(const std::vector<double>& Q, int64_t I, int ell, std::vector<int>& sel,
                             std::vector<double>& A) {
  std::sort(sel.begin(), sel.end());
  std::vector<double> inv;
  if (!invert_rows(Q, I, ell, sel, inv)) {
    set_error("subset selection: the selected rows of Q are singular");
    return RH_ENUMERIC;
  }
  apply_inv(Q, I, ell, inv, A);
  for (int a = 0; a < ell; ++a)
    for (int c = 0; c < ell; ++c) A[sel[a] + (size_t)I * c] = (a == c) ? 1.0 : 0.0;
  return RH_OK;
}

// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) on the host: ten rounds of two 32 x 32 -> 64-bit
// multiplications by 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl constants 0x9E3779B9 and
// 0xBB67AE85 between rounds.
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Sampling selections (uniform or leverage-score weights): ell rows without replacement, draw k taking
// the first untaken row whose running weight sum exceeds u_k times the untaken total (sums in FP64,
// increasing row order); u_k = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 from Philox4x32-10 with counter
// (k, stream, 0, 0x53454C45) and key (seed lo, seed hi).
rh_status sample_rows_host(const std::vector<double>& Q, int64_t I, int ell, bool leverage, uint64_t seed,
                           uint32_t stream, std::vector<int>& sel) {
  std::vector<double> w(I, 1.0);
  if (leverage)
    for (int64_t i = 0; i < I; ++i) {
      double s = 0.0;
      for (int c = 0; c < ell; ++c) {
        const double q = Q[i + (size_t)I * c];
        s = s + q * q;
      }
      w[i] = s;
    }
  std::vector<char> taken(I, 0);
  sel.clear();
  for (int k = 0; k < ell; ++k) {
    uint32_t ctr[4] = {(uint32_t)k, stream, 0u, 0x53454C45u};
    philox_host(ctr, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    const double u = ((double)(ctr[0] >> 5) * 67108864.0 + (double)(ctr[1] >> 6)) * 0x1p-53;
    double T = 0.0;
    for (int64_t i = 0; i < I; ++i)
      if (!taken[i]) T = T + w[i];
    if (!(T > 0.0)) {
      set_error("subset selection: no sampling weight left (Q has too few nonzero rows or non-finite values)");
      return RH_ENUMERIC;
    }
    const double t = u * T;
    int64_t pick = -1, last = -1;
    double c = 0.0;
    for (int64_t i = 0; i < I; ++i) {
      if (taken[i]) continue;
      c = c + w[i];
      if (w[i] > 0.0) last = i;
      if (c > t) {
        pick = i;
        break;
      }
    }
    if (pick < 0) pick = last;   // t rounded up to the total
    taken[pick] = 1;
    sel.push_back((int)pick);
  }
  return RH_OK;
}

// Row selection P and A = Q (P^T Q)^{-1} of Alg. 6 steps 6-7 (method: RH_SELECT_*).
rh_status subset_select_host(const std::vector<double>& Q, int64_t I, int ell, int method, double eta,
                             std::vector<int>& sel, std::vector<double>& A, uint64_t seed = 0, uint32_t stream = 0) {
  rh_status s;
  if (method == RH_SELECT_UNIFORM || method == RH_SELECT_LEVERAGE)
    s = sample_rows_host(Q, I, ell, method == RH_SELECT_LEVERAGE, seed, stream, sel);
  else
    s = method == RH_SELECT_DEIM ? deim_rows_host(Q, I, ell, sel) : cpqr_rows_host(Q, I, ell, sel);
  if (s != RH_OK) return s;
  if (method == RH_SELECT_SRRQR && (s = srrqr_swaps_host(Q, I, ell, eta, sel)) != RH_OK) return s;
  return interp_factor_host(Q, I, ell, sel, A);
}

struct SpBufs {
  int32_t *keys_in, *keys_out, *perm_in, *perm_out, *cnt, *flag, *dest, *pos, *row_items;
  int32_t *uid, *pd;   // distinct Omega row of each nonzero, Kolda index of each distinct row
  void* omtab;         // table of the distinct Omega rows (nnz rows of ldo entries at most)
  int3* items;
  double *part, *Y, *Q, *orth, *norm_part;
  int32_t* idx[2][RH_MAX_ORDER];
  float* vals[2];
  void* cub_tmp;
  size_t cub_bytes;
  int32_t* info;
  int32_t* pos_all;   // SP-HOSVD position tables, mode after mode
};

struct SpSizes {
  int64_t nnz, I_max, items_max;
  int ell_max;
  size_t orth, cub_bytes;
  int64_t pos_elems = 0;   // SP-HOSVD: one position table per mode (sum of I_n)
  int om_esize = 4;        // bytes per entry of the Omega table (4 FP32, 2 BF16)
};

size_t cub_bytes_for(int64_t nnz) {
  size_t a = 0, b = 0, c = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, a, (const int32_t*)nullptr, (int32_t*)nullptr, (const int32_t*)nullptr,
                                  (int32_t*)nullptr, (int)std::max<int64_t>(nnz, 1), 0, 31, (cudaStream_t)0);
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const int32_t*)nullptr, (int32_t*)nullptr,
                                (int)std::max<int64_t>(nnz, 1), (cudaStream_t)0);
  cub::DeviceScan::InclusiveSum(nullptr, c, (const int32_t*)nullptr, (int32_t*)nullptr,
                                (int)std::max<int64_t>(nnz, 1), (cudaStream_t)0);
  return std::max(a, std::max(b, c));
}

// entries per row of the Omega table: ell rounded up to a whole number of quads
int omega_ldo(int ell) { return 4 * ((ell + 3) / 4); }

SpBufs carve_sp(Arena& ar, int d, const SpSizes& z) {
  SpBufs b;
  const size_t n = (size_t)std::max<int64_t>(z.nnz, 1);
  b.keys_in = ar.take<int32_t>(n);
  b.keys_out = ar.take<int32_t>(n);
  b.perm_in = ar.take<int32_t>(n);
  b.perm_out = ar.take<int32_t>(n);
  b.flag = ar.take<int32_t>(n);
  b.dest = ar.take<int32_t>(n);
  b.cnt = ar.take<int32_t>((size_t)z.I_max + 1);
  b.pos = ar.take<int32_t>((size_t)z.I_max + 1);
  b.row_items = ar.take<int32_t>((size_t)z.I_max + 1);
  b.uid = ar.take<int32_t>(n);
  b.pd = ar.take<int32_t>(n);
  b.omtab = ar.take<char>(n * (size_t)omega_ldo(z.ell_max) * (size_t)z.om_esize);
  b.items = ar.take<int3>((size_t)z.items_max);
  b.part = ar.take<double>((size_t)z.items_max * z.ell_max);
  b.Y = ar.take<double>((size_t)z.I_max * z.ell_max);
  b.Q = ar.take<double>((size_t)z.I_max * z.ell_max);
  b.orth = ar.take<double>(z.orth);
  b.norm_part = ar.take<double>(1024);
  for (int s = 0; s < 2; ++s) {
    for (int k = 0; k < d; ++k) b.idx[s][k] = ar.take<int32_t>(n);
    b.vals[s] = ar.take<float>(n);
  }
  b.cub_bytes = z.cub_bytes;
  b.cub_tmp = ar.take<char>(z.cub_bytes);
  b.info = ar.take<int32_t>(4);
  b.pos_all = z.pos_elems ? ar.take<int32_t>((size_t)z.pos_elems) : nullptr;
  return b;
}

int bits_for(int64_t v) {
  int b = 1;
  while (b < 31 && (int64_t(1) << b) < v) ++b;
  return b;
}

// Y = G_(n) Omega_n (I x ell, FP64, column-major) from the COO nonzeros (Alg. 6 step 4): stable sort
// by i_n, work items of at most kItem nonzeros per row, warp partials, FP64 sums in item order.
rh_status sp_sketch_mode(const SpIdx& ix, int order, int n, int64_t I, int64_t M, int ell, int64_t cnnz,
                         const int32_t* key, const float* vals, uint64_t seed, int32_t tensor_id, bool om_bf16,
                         int64_t items_max, const SpBufs& b, double* Y, cudaStream_t st) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  const uint32_t sid = ((uint32_t)tensor_id << 4) | (uint32_t)n;
  const int ldo = omega_ldo(ell), nq = ldo / 4;
  const bool table = cnnz > 0 && M < (int64_t(1) << 31);
  size_t tb = b.cub_bytes;
  if (cnnz > 0) {
    iota_kernel<<<grid_for(cnnz), 256, 0, st>>>(b.perm_in, cnnz);
    RH_LAUNCH_CHECK();
  }
  if (table) {
    // (0) the distinct Omega rows: sort the nonzeros' Kolda indices, number the distinct ones, and
    // generate each row once into the table
    ProfileScope ps(PROF_SP_TABLE, n, st);
    kolda_key_kernel<<<grid_for(cnnz), 256, 0, st>>>(ix, order, cnnz, b.keys_in);
    RH_LAUNCH_CHECK();
    RH_CUDA_TRY(cub::DeviceRadixSort::SortPairs(b.cub_tmp, tb, b.keys_in, b.keys_out, b.perm_in, b.perm_out,
                                                (int)cnnz, 0, bits_for(M), st));
    run_heads_kernel<<<grid_for(cnnz), 256, 0, st>>>(b.keys_out, cnnz, b.flag);
    RH_LAUNCH_CHECK();
    tb = b.cub_bytes;
    RH_CUDA_TRY(cub::DeviceScan::InclusiveSum(b.cub_tmp, tb, b.flag, b.dest, (int)cnnz, st));
    distinct_rows_kernel<<<grid_for(cnnz), 256, 0, st>>>(b.keys_out, b.perm_out, b.flag, b.dest, cnnz, b.uid, b.pd);
    RH_LAUNCH_CHECK();
    const int tgrid = grid_for(cnnz * (int64_t)nq);
    if (om_bf16)
      omega_table_kernel<true><<<tgrid, 256, 0, st>>>(b.pd, b.dest + cnnz - 1, nq, ldo, k0, k1, sid, b.omtab);
    else
      omega_table_kernel<false><<<tgrid, 256, 0, st>>>(b.pd, b.dest + cnnz - 1, nq, ldo, k0, k1, sid, b.omtab);
    RH_LAUNCH_CHECK();
  }
  // (a) stable sort of the nonzeros by i_n; row counts (an empty tensor has no items: Y = 0)
  tb = b.cub_bytes;
  RH_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * (I + 1), st));
  if (cnnz > 0) {
    ProfileScope ps(PROF_SP_SORT, n, st);
    RH_CUDA_TRY(cub::DeviceRadixSort::SortPairs(b.cub_tmp, tb, key, b.keys_out, b.perm_in, b.perm_out,
                                                (int)cnnz, 0, bits_for(I), st));
    // row counts from the runs of the sorted keys; keys outside [0, I) counted in cnt[I]
    bad_keys_kernel<<<grid_for(cnnz), 256, 0, st>>>(key, cnnz, I, b.cnt + I);
    RH_LAUNCH_CHECK();
    RH_CUDA_TRY(cudaMemsetAsync(b.pos, 0, sizeof(int32_t) * I, st));
    run_bounds_kernel<<<grid_for(cnnz), 256, 0, st>>>(b.keys_out, cnnz, I, b.pos, b.cnt);
    RH_LAUNCH_CHECK();
    run_counts_kernel<<<grid_for(I), 256, 0, st>>>(b.pos, I, b.cnt);
    RH_LAUNCH_CHECK();
  }
  std::vector<int32_t> cnt(I + 1);
  RH_CUDA_TRY(cudaMemcpyAsync(cnt.data(), b.cnt, sizeof(int32_t) * (I + 1), cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  if (cnt[I] != 0) {
    set_error("invalid argument: " + std::to_string(cnt[I]) + " indices of mode " + std::to_string(n) +
              " lie outside [0, " + std::to_string(I) + ")");
    return RH_EINVAL;
  }
  // (b) work items: each row's run cut into pieces of at most kItem nonzeros
  std::vector<int3> items;
  std::vector<int32_t> row_items(I + 1, 0);
  int64_t off = 0;
  for (int64_t r = 0; r < I; ++r) {
    row_items[r] = (int32_t)items.size();
    for (int64_t a = 0; a < cnt[r]; a += kItem)
      items.push_back(make_int3((int)r, (int)(off + a), (int)(off + std::min<int64_t>(cnt[r], a + kItem))));
    off += cnt[r];
  }
  row_items[I] = (int32_t)items.size();
  if ((int64_t)items.size() > items_max) {
    set_error("SP-STHOSVD: internal item count exceeds the plan");
    return RH_ENUMERIC;
  }
  if (!items.empty())
    RH_CUDA_TRY(cudaMemcpyAsync(b.items, items.data(), sizeof(int3) * items.size(), cudaMemcpyHostToDevice, st));
  RH_CUDA_TRY(cudaMemcpyAsync(b.row_items, row_items.data(), sizeof(int32_t) * (I + 1), cudaMemcpyHostToDevice, st));
  // (c) sketch Y = G_(n) Omega_n (step 4)
  if (!items.empty()) {
    ProfileScope ps(PROF_SP_ITEMS, n, st);
    const int nwarps = (int)std::min<int64_t>((int64_t)items.size(), 64LL * num_sms());
    const dim3 grid((unsigned)ceil_div(nwarps, 8));
    const int nit = (int)items.size();
    if (table && om_bf16)
      sp_sketch_items_kernel<3><<<grid, 256, 0, st>>>(ix, order, vals, b.perm_out, b.items, nit, ell, k0, k1, sid,
                                                        b.uid, b.omtab, ldo, b.part);
    else if (table)
      sp_sketch_items_kernel<2><<<grid, 256, 0, st>>>(ix, order, vals, b.perm_out, b.items, nit, ell, k0, k1, sid,
                                                        b.uid, b.omtab, ldo, b.part);
    else if (om_bf16)
      sp_sketch_items_kernel<1><<<grid, 256, 0, st>>>(ix, order, vals, b.perm_out, b.items, nit, ell, k0, k1, sid,
                                                        nullptr, nullptr, ldo, b.part);
    else
      sp_sketch_items_kernel<0><<<grid, 256, 0, st>>>(ix, order, vals, b.perm_out, b.items, nit, ell, k0, k1, sid,
                                                        nullptr, nullptr, ldo, b.part);
    RH_LAUNCH_CHECK();
  }
  ProfileScope psr(PROF_SP_REDUCE, n, st);
  sp_sketch_reduce_kernel<<<(unsigned)std::min<int64_t>(I, 64LL * num_sms()), 32 * kRedRowWarps, 0, st>>>(
      b.part, b.row_items, I, ell, Y);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

// independent: SP-HOSVD (every mode on the input sizes, modes in increasing order, one position
// table per mode); otherwise Alg. 6 (the size rule on the current core, order rho).
rh_status sp_plan(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* ranks, const rh_options& o,
                  std::vector<int>& rho, std::vector<int>& ells, SpSizes& z, bool independent = false) {
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
  RH_CHECK_ARG(ranks != nullptr, "ranks is NULL");
  RH_CHECK_ARG(nnz >= 1 && nnz < (int64_t(1) << 31), "nnz must be in [1, 2^31)");
  RH_CHECK_ARG(o.p >= 0, "oversampling p must be >= 0");
  RH_CHECK_ARG(o.tensor_id >= 0 && o.tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(o.power_iters == 0, "the sparse range finder runs without subspace iteration (power_iters must be 0)");
  RH_CHECK_ARG(o.select >= RH_SELECT_SRRQR && o.select <= RH_SELECT_LEVERAGE,
               "select must be one of RH_SELECT_SRRQR, _CPQR, _DEIM, _UNIFORM, _LEVERAGE");
  RH_CHECK_ARG(o.omega_prec == RH_F64 || o.omega_prec == RH_F32 || o.omega_prec == RH_BF16,
               "omega_prec must be RH_F32 (or RH_F64: the same FP32 normals) or RH_BF16");
  for (int k = 0; k < order; ++k) {
    RH_CHECK_ARG(dims[k] >= 1 && dims[k] < (int64_t(1) << 31), "every dimension must be in [1, 2^31)");
    RH_CHECK_ARG(ranks[k] >= 1, "every rank must be >= 1");
  }
  rho.resize(order);
  if (independent) {
    std::iota(rho.begin(), rho.end(), 0);
  } else if (o.rho[0] < 0) {
    std::iota(rho.begin(), rho.end(), 0);
    std::stable_sort(rho.begin(), rho.end(), [&](int a, int c) { return dims[a] > dims[c]; });
  } else {
    std::vector<int> seen(order, 0);
    for (int k = 0; k < order; ++k) {
      RH_CHECK_ARG(o.rho[k] >= 0 && o.rho[k] < order && !seen[o.rho[k]], "rho must be a permutation of 0..order-1");
      seen[o.rho[k]] = 1;
      rho[k] = o.rho[k];
    }
  }
  std::vector<int64_t> cur(dims, dims + order);
  ells.assign(order, 0);
  z.nnz = nnz;
  z.I_max = 1;
  z.ell_max = 1;
  z.orth = 1;
  for (int j = 0; j < order; ++j) {
    const int n = rho[j];
    int64_t M = 1;
    for (int k = 0; k < order; ++k)
      if (k != n) M *= cur[k];
    int64_t ell = (int64_t)ranks[n] + o.p;
    const int64_t lim = std::min<int64_t>(cur[n], M);
    if (ell >= lim) {   // Alg. 6 requires r + p < min(I_n, prod of the other sizes)
      if (!o.clamp) {
        set_error("invalid argument: r_n + p = " + std::to_string(ell) + " must be < min(I_n, prod of the other " +
                  "sizes) = " + std::to_string(lim) + " for mode " + std::to_string(n));
        return RH_EINVAL;
      }
      ell = lim - 1;
    }
    if (ell < 1) {
      set_error("invalid argument: mode " + std::to_string(n) + " is too small for SP-STHOSVD");
      return RH_EINVAL;
    }
    if (ell > RH_MAX_ELL) {
      set_error("unsupported: r_n + p exceeds RH_MAX_ELL (64)");
      return RH_EUNSUPPORTED;
    }
    ells[n] = (int)ell;
    z.I_max = std::max(z.I_max, cur[n]);
    z.ell_max = std::max(z.ell_max, (int)ell);
    z.orth = std::max(z.orth, orth_workspace_elems(cur[n], (int)ell));
    if (independent)
      z.pos_elems += cur[n];
    else
      cur[n] = ell;
  }
  z.items_max = nnz / kItem + z.I_max + 1;
  z.cub_bytes = cub_bytes_for(nnz);
  z.om_esize = o.omega_prec == RH_BF16 ? 2 : 4;
  return RH_OK;
}

// Alg. 6 steps 5-7 for one mode: Y = QR (device), the row selection P (host, FP64, method of
// Sec. 5; sampling with stream (tensor_id << 4) | n), A_n = Q (P^T Q)^{-1} into factors_n, P into
// selected_n (optional); sel receives P (sorted).
rh_status sp_select_mode(int64_t I, int ell, int n, const rh_options& o, const SpBufs& b, double* factor_n,
                         int32_t* selected_n, std::vector<int>& sel, cudaStream_t st) {
  rh_status s;
  RH_CUDA_TRY(cudaMemsetAsync(b.info, 0, sizeof(int32_t), st));
  if ((s = launch_orthonormalize(I, ell, b.Y, b.Q, b.info, b.orth, st, false)) != RH_OK) return s;
  std::vector<double> Qh((size_t)I * ell);
  RH_CUDA_TRY(cudaMemcpyAsync(Qh.data(), b.Q, sizeof(double) * I * ell, cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> A;
  if ((s = subset_select_host(Qh, I, ell, o.select, 2.0, sel, A, o.seed, ((uint32_t)o.tensor_id << 4) | (uint32_t)n)) !=
      RH_OK)
    return s;
  std::sort(sel.begin(), sel.end());
  RH_CUDA_TRY(cudaMemcpyAsync(factor_n, A.data(), sizeof(double) * I * ell, cudaMemcpyHostToDevice, st));
  if (selected_n) RH_CUDA_TRY(cudaMemcpyAsync(selected_n, sel.data(), sizeof(int32_t) * ell, cudaMemcpyHostToDevice, st));
  // the host vectors are read by the copies above: wait for them before they go out of scope
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  return RH_OK;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" {

size_t sp_sthosvd_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* ranks,
                                     const rh_options* opts) {
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  std::vector<int> rho, ells;
  SpSizes z;
  if (sp_plan(order, dims, nnz, ranks, o, rho, ells, z) != RH_OK) return 0;
  Arena ar(nullptr);
  carve_sp(ar, order, z);
  return ar.used;
}

rh_status sp_sthosvd_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                         const float* vals, const int32_t* ranks, const rh_options* opts, double* const* factors,
                         int32_t* const* selected, double* core, double* norms, void* workspace,
                         size_t workspace_bytes, void* stream) {
  clear_error();
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  std::vector<int> rho, ells;
  SpSizes z;
  rh_status s = sp_plan(order, dims, nnz, ranks, o, rho, ells, z);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(idx != nullptr && vals != nullptr && factors != nullptr && core != nullptr,
               "idx, vals, factors and core must be non-NULL");
  for (int k = 0; k < order; ++k) {
    RH_CHECK_ARG(idx[k] != nullptr && factors[k] != nullptr, "every idx[n] and factors[n] must be non-NULL");
  }
  Arena meas(nullptr);
  carve_sp(meas, order, z);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  SpBufs b = carve_sp(ar, order, z);
  cudaStream_t st = (cudaStream_t)stream;

  // the working copy of the tensor (set 0) and ||X||^2
  for (int k = 0; k < order; ++k)
    RH_CUDA_TRY(cudaMemcpyAsync(b.idx[0][k], idx[k], sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
  RH_CUDA_TRY(cudaMemcpyAsync(b.vals[0], vals, sizeof(float) * nnz, cudaMemcpyDeviceToDevice, st));
  if (norms) {
    const int nb = (int)std::min<int64_t>(ceil_div(nnz, 256), 1024);
    sumsq_f32_kernel<<<nb, 256, 0, st>>>(b.vals[0], nnz, b.norm_part);
    RH_LAUNCH_CHECK();
    sum_parts_kernel<<<1, 32, 0, st>>>(b.norm_part, nb, norms);
    RH_LAUNCH_CHECK();
  }
  std::vector<int64_t> cur(dims, dims + order);
  int set = 0;
  int64_t cnnz = nnz;
  for (int j = 0; j < order; ++j) {
    const int n = rho[j];
    const int ell = ells[n];
    const int64_t I = cur[n];
    SpIdx ix;
    int64_t stride = 1;
    for (int k = 0; k < order; ++k) {
      ix.idx[k] = b.idx[set][k];
      if (k == n) {
        ix.stride[k] = 0;
      } else {
        ix.stride[k] = stride;
        stride *= cur[k];
      }
    }
    for (int k = order; k < RH_MAX_ORDER; ++k) {
      ix.idx[k] = nullptr;
      ix.stride[k] = 0;
    }
    if ((s = sp_sketch_mode(ix, order, n, I, stride, ell, cnnz, b.idx[set][n], b.vals[set], o.seed, o.tensor_id,
                            o.omega_prec == RH_BF16, z.items_max, b, b.Y, st)) != RH_OK)
      return s;
    // (d)-(e) thin QR (step 5), the row selection (step 6, strong RRQR by default) and
    // A_n = Q (P^T Q)^{-1} (step 7)
    std::vector<int> sel;
    if ((s = sp_select_mode(I, ell, n, o, b, factors[n], selected ? selected[n] : nullptr, sel, st)) != RH_OK)
      return s;
    // (f) G_(n) <- P^T G_(n): keep the selected slices, renumber mode n (step 8)
    std::vector<int32_t> pos(I, -1);
    for (int a = 0; a < ell; ++a) pos[sel[a]] = a;
    RH_CUDA_TRY(cudaMemcpyAsync(b.pos, pos.data(), sizeof(int32_t) * I, cudaMemcpyHostToDevice, st));
    if (cnnz > 0) {
      keep_flags_kernel<<<grid_for(cnnz), 256, 0, st>>>(b.idx[set][n], cnnz, b.pos, b.flag);
      RH_LAUNCH_CHECK();
      size_t tb = b.cub_bytes;
      RH_CUDA_TRY(cub::DeviceScan::ExclusiveSum(b.cub_tmp, tb, b.flag, b.dest, (int)cnnz, st));
      int32_t last_dest = 0, last_flag = 0;
      RH_CUDA_TRY(cudaMemcpyAsync(&last_dest, b.dest + cnnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      RH_CUDA_TRY(cudaMemcpyAsync(&last_flag, b.flag + cnnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      SpIdx out;
      for (int k = 0; k < RH_MAX_ORDER; ++k) {
        out.idx[k] = k < order ? b.idx[1 - set][k] : nullptr;
        out.stride[k] = 0;
      }
      compact_kernel<<<grid_for(cnnz), 256, 0, st>>>(ix, order, n, b.vals[set], cnnz, b.flag, b.dest, b.pos, out,
                                                      b.vals[1 - set]);
      RH_LAUNCH_CHECK();
      RH_CUDA_TRY(cudaStreamSynchronize(st));
      cnnz = (int64_t)last_dest + last_flag;
    }
    set = 1 - set;
    cur[n] = ell;
  }
  // dense ell_1 x ... x ell_d core of the surviving entries
  int64_t ncore = 1;
  for (int k = 0; k < order; ++k) ncore *= cur[k];
  RH_CUDA_TRY(cudaMemsetAsync(core, 0, sizeof(double) * ncore, st));
  if (cnnz > 0) {
    SpIdx ix;
    int64_t stride = 1;
    for (int k = 0; k < RH_MAX_ORDER; ++k) {
      ix.idx[k] = k < order ? b.idx[set][k] : nullptr;
      ix.stride[k] = k < order ? stride : 0;
      if (k < order) stride *= cur[k];
    }
    scatter_core_kernel<<<grid_for(cnnz), 256, 0, st>>>(ix, order, b.vals[set], cnnz, core);
    RH_LAUNCH_CHECK();
  }
  if (norms) {
    if ((s = launch_sumsq(core, ncore, norms + 1, st)) != RH_OK) return s;
  }
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  return RH_OK;
}

size_t sp_hosvd_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* ranks,
                                   const rh_options* opts) {
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  std::vector<int> rho, ells;
  SpSizes z;
  if (sp_plan(order, dims, nnz, ranks, o, rho, ells, z, true) != RH_OK) return 0;
  Arena ar(nullptr);
  carve_sp(ar, order, z);
  return ar.used;
}

rh_status sp_hosvd_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx, const float* vals,
                       const int32_t* ranks, const rh_options* opts, double* const* factors, int32_t* const* selected,
                       double* core, double* norms, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  std::vector<int> rho, ells;
  SpSizes z;
  rh_status s = sp_plan(order, dims, nnz, ranks, o, rho, ells, z, true);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(idx != nullptr && vals != nullptr && factors != nullptr && core != nullptr,
               "idx, vals, factors and core must be non-NULL");
  for (int k = 0; k < order; ++k)
    RH_CHECK_ARG(idx[k] != nullptr && factors[k] != nullptr, "every idx[n] and factors[n] must be non-NULL");
  Arena meas(nullptr);
  carve_sp(meas, order, z);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  SpBufs b = carve_sp(ar, order, z);
  cudaStream_t st = (cudaStream_t)stream;
  if (norms) {
    const int nb = (int)std::min<int64_t>(ceil_div(nnz, 256), 1024);
    sumsq_f32_kernel<<<nb, 256, 0, st>>>(vals, nnz, b.norm_part);
    RH_LAUNCH_CHECK();
    sum_parts_kernel<<<1, 32, 0, st>>>(b.norm_part, nb, norms);
    RH_LAUNCH_CHECK();
  }
  // every mode of the input on its own (Sec. 5, SP-HOSVD): sketch, QR, selection, A_n
  SpIdx in;
  PosTabs pt;
  int64_t pos_off = 0;
  for (int k = 0; k < RH_MAX_ORDER; ++k) {
    in.idx[k] = k < order ? idx[k] : nullptr;
    in.stride[k] = 0;
    pt.pos[k] = nullptr;
  }
  for (int n = 0; n < order; ++n) {
    const int ell = ells[n];
    const int64_t I = dims[n];
    SpIdx ix = in;
    int64_t stride = 1;
    for (int k = 0; k < order; ++k) {
      ix.stride[k] = 0;
      if (k != n) {
        ix.stride[k] = stride;
        stride *= dims[k];
      }
    }
    if ((s = sp_sketch_mode(ix, order, n, I, stride, ell, nnz, idx[n], vals, o.seed, o.tensor_id,
                            o.omega_prec == RH_BF16, z.items_max, b, b.Y, st)) != RH_OK)
      return s;
    std::vector<int> sel;
    if ((s = sp_select_mode(I, ell, n, o, b, factors[n], selected ? selected[n] : nullptr, sel, st)) != RH_OK)
      return s;
    std::vector<int32_t> pos(I, -1);
    for (int a = 0; a < ell; ++a) pos[sel[a]] = a;
    int32_t* pn = b.pos_all + pos_off;
    RH_CUDA_TRY(cudaMemcpyAsync(pn, pos.data(), sizeof(int32_t) * I, cudaMemcpyHostToDevice, st));
    RH_CUDA_TRY(cudaStreamSynchronize(st));   // pos is read by the copy
    pt.pos[n] = pn;
    pos_off += I;
  }
  // the core: the nonzeros whose every index is selected, renumbered (X at the selected coordinates)
  keep_all_kernel<<<grid_for(nnz), 256, 0, st>>>(in, order, nnz, pt, b.flag);
  RH_LAUNCH_CHECK();
  size_t tb = b.cub_bytes;
  RH_CUDA_TRY(cub::DeviceScan::ExclusiveSum(b.cub_tmp, tb, b.flag, b.dest, (int)nnz, st));
  int32_t last_dest = 0, last_flag = 0;
  RH_CUDA_TRY(cudaMemcpyAsync(&last_dest, b.dest + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaMemcpyAsync(&last_flag, b.flag + nnz - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SpIdx out;
  for (int k = 0; k < RH_MAX_ORDER; ++k) {
    out.idx[k] = k < order ? b.idx[0][k] : nullptr;
    out.stride[k] = 0;
  }
  compact_all_kernel<<<grid_for(nnz), 256, 0, st>>>(in, order, vals, nnz, b.flag, b.dest, pt, out, b.vals[0]);
  RH_LAUNCH_CHECK();
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  const int64_t kept = (int64_t)last_dest + last_flag;
  int64_t ncore = 1;
  SpIdx cx;
  for (int k = 0; k < RH_MAX_ORDER; ++k) {
    cx.idx[k] = k < order ? b.idx[0][k] : nullptr;
    cx.stride[k] = k < order ? ncore : 0;
    if (k < order) ncore *= ells[k];
  }
  RH_CUDA_TRY(cudaMemsetAsync(core, 0, sizeof(double) * ncore, st));
  if (kept > 0) {
    scatter_core_kernel<<<grid_for(kept), 256, 0, st>>>(cx, order, b.vals[0], kept, core);
    RH_LAUNCH_CHECK();
  }
  if (norms && (s = launch_sumsq(core, ncore, norms + 1, st)) != RH_OK) return s;
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  return RH_OK;
}

rh_status rh_subset_select(int64_t I, int32_t ell, const double* Q, int32_t method, double eta, uint64_t seed,
                           uint32_t stream, int32_t* selected, double* A) {
  clear_error();
  RH_CHECK_ARG(I >= 1 && ell >= 1 && ell <= I, "need 1 <= ell <= I");
  RH_CHECK_ARG(I <= (int64_t(1) << 31) - 1 && (uint64_t)I * (uint64_t)ell <= (uint64_t(1) << 40),
               "I x ell too large for the host selection");
  RH_CHECK_ARG(method >= RH_SELECT_SRRQR && method <= RH_SELECT_LEVERAGE,
               "method must be one of RH_SELECT_SRRQR, _CPQR, _DEIM, _UNIFORM, _LEVERAGE");
  RH_CHECK_ARG(method != RH_SELECT_SRRQR || eta >= 1.0, "eta must be >= 1");
  RH_CHECK_ARG(Q != nullptr && selected != nullptr && A != nullptr, "Q, selected and A must be non-NULL");
  const std::vector<double> Qh(Q, Q + (size_t)I * ell);
  std::vector<int> sel;
  std::vector<double> Ah;
  const rh_status s = subset_select_host(Qh, I, ell, method, eta, sel, Ah, seed, stream);
  if (s != RH_OK) return s;
  for (int a = 0; a < ell; ++a) selected[a] = sel[a];
  std::copy(Ah.begin(), Ah.end(), A);
  return RH_OK;
}

size_t rhosvd_sketch_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, int32_t mode, int32_t ell) {
  if (order < 1 || order > RH_MAX_ORDER || dims == nullptr || mode < 0 || mode >= order || mode >= 16) return 0;
  if (nnz < 0 || nnz >= (int64_t(1) << 31) || ell < 1 || ell > RH_MAX_ELL) return 0;
  for (int k = 0; k < order; ++k)
    if (dims[k] < 1 || dims[k] >= (int64_t(1) << 31)) return 0;
  SpSizes z;
  z.nnz = nnz;
  z.I_max = dims[mode];
  z.ell_max = ell;
  z.orth = 1;
  z.items_max = nnz / kItem + z.I_max + 1;
  z.cub_bytes = cub_bytes_for(nnz);
  Arena ar(nullptr);
  carve_sp(ar, order, z);
  return ar.used;
}

rh_status rhosvd_sketch_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                            const float* vals, int32_t mode, int32_t ell, uint64_t seed, int32_t tensor_id,
                            int32_t omega_prec, double* Y, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const size_t need = rhosvd_sketch_coo_workspace_size(order, dims, nnz, mode, ell);
  RH_CHECK_ARG(need > 0, "bad order, dims, nnz, mode or ell");
  RH_CHECK_ARG(tensor_id >= 0 && tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(omega_prec == RH_F64 || omega_prec == RH_F32 || omega_prec == RH_BF16,
               "omega_prec must be RH_F32 (or RH_F64: the same FP32 normals) or RH_BF16");
  RH_CHECK_ARG(idx != nullptr && Y != nullptr && (nnz == 0 || vals != nullptr), "idx, vals and Y must be non-NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(nnz == 0 || idx[k] != nullptr, "every idx[n] must be non-NULL");
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  SpSizes z;
  z.nnz = nnz;
  z.I_max = dims[mode];
  z.ell_max = ell;
  z.orth = 1;
  z.items_max = nnz / kItem + z.I_max + 1;
  z.cub_bytes = cub_bytes_for(nnz);
  Arena ar(workspace);
  const SpBufs b = carve_sp(ar, order, z);
  SpIdx ix;
  int64_t stride = 1;
  for (int k = 0; k < RH_MAX_ORDER; ++k) {
    ix.idx[k] = k < order ? idx[k] : nullptr;
    ix.stride[k] = 0;
    if (k < order && k != mode) {
      ix.stride[k] = stride;
      stride *= dims[k];
    }
  }
  return sp_sketch_mode(ix, order, mode, dims[mode], stride, ell, nnz, nnz ? idx[mode] : nullptr, vals, seed, tensor_id,
                        omega_prec == RH_BF16, z.items_max, b, Y, (cudaStream_t)stream);
}

}  // extern "C"
