// C-ABI drivers of R-HOSVD (Alg. 2), of the core formation G = X x_1 A_1^T ... x_d A_d^T
// (Alg. 2 step 6) and of the direct reconstruction error ||X - X_hat||_F (validation).
// Host code sequences kernels on the caller's stream; every arithmetic step runs on the device.
#include <algorithm>
#include <string>
#include <vector>

#include "driver.cuh"

namespace rh {
namespace {

// ---- casts and norms ---------------------------------------------------------------
template <typename T>
__global__ void cast_strided_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (T)src[e];
}

template <typename T>
__global__ void sumsq_parts_kernel(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[e];
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

__global__ void sum_fixed_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < n; ++k) t += part[k];
    *out = t;
  }
}

constexpr int kNormBlocks = 1024;

template <typename T>
rh_status cast_to(const double* src, T* dst, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4096));
  cast_strided_kernel<T><<<blocks, 256, 0, st>>>(src, dst, n);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

template <typename T>
rh_status sumsq_big(const T* x, int64_t n, double* part, double* out, cudaStream_t st) {
  sumsq_parts_kernel<T><<<kNormBlocks, 256, 0, st>>>(x, n, part);
  RH_LAUNCH_CHECK();
  sum_fixed_kernel<<<1, 32, 0, st>>>(part, kNormBlocks, out);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

// ---- G = X x_n A_n^T over all modes ---------------------------------------------------
struct CorePlan {
  std::vector<int> order;       // modes in processing order
  size_t max_inter = 0;         // elements of the largest intermediate (excluding X and G)
  size_t fac_elems = 0;         // sum I_n k_n
};

CorePlan plan_core(int d, const int64_t* dims, const int32_t* ks) {
  CorePlan pl;
  std::vector<int64_t> cur(dims, dims + d);
  std::vector<int> left;
  for (int n = 0; n < d; ++n) {
    left.push_back(n);
    pl.fac_elems += (size_t)dims[n] * ks[n];
  }
  while (!left.empty()) {
    // the mode that shrinks the current tensor most (ties: lower mode)
    auto best = std::max_element(left.begin(), left.end(), [&](int a, int b) {
      const double ra = (double)cur[a] / ks[a], rb = (double)cur[b] / ks[b];
      return ra < rb || (ra == rb && a > b);
    });
    const int n = *best;
    left.erase(best);
    cur[n] = ks[n];
    pl.order.push_back(n);
    if (!left.empty()) pl.max_inter = std::max(pl.max_inter, (size_t)prod(cur));
  }
  return pl;
}

// split_tc (FP32 data, the RH_F32_BF16X2 form): every product but the last whose shape the
// tensor-core mode product covers runs there (the FP32 input split into BF16 head and tail on the
// fly -- pieces = 3: exactly, into three -- the factor into two pieces in qa); the others, and the
// last (FP64 output), on the CUDA cores.
template <typename T>
rh_status run_core(int d, const int64_t* dims, const T* X, const double* const* factors, const int32_t* ks,
                   double* G, const CorePlan& pl, T* fac, T* W0, T* W1, cudaStream_t st, bool split_tc = false,
                   uint16_t* qa = nullptr, int32_t* err = nullptr, int pieces = 2) {
  std::vector<const T*> fc(d);
  size_t off = 0;
  rh_status s;
  for (int n = 0; n < d; ++n) {
    if ((s = cast_to<T>(factors[n], fac + off, dims[n] * (int64_t)ks[n], st)) != RH_OK) return s;
    fc[n] = fac + off;
    off += (size_t)dims[n] * ks[n];
  }
  std::vector<int64_t> cur(dims, dims + d);
  const T* in = X;
  T* bufs[2] = {W0, W1};
  int nb = 0;
  for (size_t j = 0; j < pl.order.size(); ++j) {
    const int n = pl.order[j];
    const ModeView v = mode_view(d, cur.data(), n);
    const bool last = (j + 1 == pl.order.size());
    if (last) {
      if ((s = launch_ttm_strided<T, double>(v, in, fc[n], 1, dims[n], ks[n], G, st)) != RH_OK) return s;
    } else {
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (split_tc && qa != nullptr) {
          const float* xin = reinterpret_cast<const float*>(in);
          float* out = reinterpret_cast<float*>(bufs[nb]);
          if (v.L == 1 && ttm_tc_supported(v, ks[n])) {
            if ((s = launch_ttm_tc_f32(v, ks[n], xin, factors[n], qa, out, err, st, pieces)) != RH_OK) return s;
            done = true;
          } else if (ttm_tc_strided_supported(v, ks[n])) {
            if ((s = launch_ttm_tc_f32s(v, ks[n], xin, factors[n], qa, out, err, st, pieces)) != RH_OK) return s;
            done = true;
          }
        }
      }
      if (!done && (s = launch_ttm_strided<T, T>(v, in, fc[n], 1, dims[n], ks[n], bufs[nb], st)) != RH_OK) return s;
      in = bufs[nb];
      nb ^= 1;
    }
    cur[n] = ks[n];
  }
  return RH_OK;
}

size_t esize(int32_t dtype) { return dtype == RH_F64 ? sizeof(double) : sizeof(float); }

}  // namespace

size_t core_chain_elems(int d, const int64_t* dims, const int32_t* ks, size_t* fac_elems) {
  const CorePlan pl = plan_core(d, dims, ks);
  if (fac_elems) *fac_elems = pl.fac_elems;
  return std::max<size_t>(pl.max_inter, 1);
}

template <typename T>
rh_status launch_core_ttm(int d, const int64_t* dims, const T* X, const double* const* factors, const int32_t* ks,
                          double* G, T* fac, T* W0, T* W1, cudaStream_t st, bool split_tc, uint16_t* qa,
                          int32_t* err, int pieces) {
  return run_core<T>(d, dims, X, factors, ks, G, plan_core(d, dims, ks), fac, W0, W1, st, split_tc, qa, err, pieces);
}
template rh_status launch_core_ttm<float>(int, const int64_t*, const float*, const double* const*, const int32_t*,
                                          double*, float*, float*, float*, cudaStream_t, bool, uint16_t*, int32_t*, int);
template rh_status launch_core_ttm<double>(int, const int64_t*, const double*, const double* const*, const int32_t*,
                                           double*, double*, double*, double*, cudaStream_t, bool, uint16_t*, int32_t*, int);

}  // namespace rh

using namespace rh;

extern "C" {

size_t core_ttm_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ks) {
  if (check_tensor_args(order, dims, dtype) != RH_OK || ks == nullptr) return 0;
  for (int n = 0; n < order; ++n)
    if (ks[n] < 1) return 0;
  const CorePlan pl = plan_core(order, dims, ks);
  Arena ar(nullptr);
  ar.take<char>(pl.fac_elems * esize(dtype));
  ar.take<char>(std::max<size_t>(pl.max_inter, 1) * esize(dtype));
  ar.take<char>(std::max<size_t>(pl.max_inter, 1) * esize(dtype));
  return ar.used;
}

rh_status core_ttm(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const double* const* factors,
                   const int32_t* ks, double* G, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_status s = check_tensor_args(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(ks != nullptr && factors != nullptr && X != nullptr && G != nullptr,
               "X, factors, ks and G must be non-NULL");
  for (int n = 0; n < order; ++n) {
    RH_CHECK_ARG(ks[n] >= 1, "every k_n must be >= 1");
    RH_CHECK_ARG(factors[n] != nullptr, "every factors[n] must be non-NULL");
  }
  const size_t need = core_ttm_workspace_size(order, dims, dtype, ks);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  const CorePlan pl = plan_core(order, dims, ks);
  Arena ar(workspace);
  const size_t es = esize(dtype);
  char* fac = ar.take<char>(pl.fac_elems * es);
  char* w0 = ar.take<char>(std::max<size_t>(pl.max_inter, 1) * es);
  char* w1 = ar.take<char>(std::max<size_t>(pl.max_inter, 1) * es);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == RH_F64)
    return run_core<double>(order, dims, static_cast<const double*>(X), factors, ks, G, pl,
                            reinterpret_cast<double*>(fac), reinterpret_cast<double*>(w0),
                            reinterpret_cast<double*>(w1), st);
  return run_core<float>(order, dims, static_cast<const float*>(X), factors, ks, G, pl, reinterpret_cast<float*>(fac),
                         reinterpret_cast<float*>(w0), reinterpret_cast<float*>(w1), st);
}

// ---- ||X - G x_1 A_1 ... x_d A_d||_F^2 and ||X||_F^2 ----------------------------------------
static void resid_plan(int d, const int64_t* dims, const int32_t* ks, int& fused, std::vector<int>& pre,
                       size_t& max_inter, size_t& fac_elems, int64_t& parts) {
  fused = 0;
  double best = -1;
  fac_elems = (size_t)1;
  for (int n = 0; n < d; ++n) {
    const double r = (double)dims[n] / ks[n];
    if (r > best) {
      best = r;
      fused = n;
    }
  }
  std::vector<int> others;
  for (int n = 0; n < d; ++n)
    if (n != fused) others.push_back(n);
  std::stable_sort(others.begin(), others.end(),
                   [&](int a, int b) { return (double)dims[a] / ks[a] < (double)dims[b] / ks[b]; });
  pre = others;
  std::vector<int64_t> cur(ks, ks + d);
  max_inter = (size_t)prod(cur);
  fac_elems = (size_t)prod(cur);
  for (int n = 0; n < d; ++n) fac_elems += (size_t)dims[n] * ks[n];
  for (int n : pre) {
    cur[n] = dims[n];
    max_inter = std::max(max_inter, (size_t)prod(cur));
  }
  parts = ttm_resid_parts(mode_view(d, cur.data(), fused), (int)dims[fused]);
}

size_t rh_tucker_residual_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ks) {
  if (check_tensor_args(order, dims, dtype) != RH_OK || ks == nullptr) return 0;
  for (int n = 0; n < order; ++n)
    if (ks[n] < 1) return 0;
  int fused;
  std::vector<int> pre;
  size_t mi, fe;
  int64_t parts;
  resid_plan(order, dims, ks, fused, pre, mi, fe, parts);
  Arena ar(nullptr);
  ar.take<char>(fe * esize(dtype));
  ar.take<char>(mi * esize(dtype));
  ar.take<char>(mi * esize(dtype));
  ar.take<double>((size_t)std::max<int64_t>(parts, kNormBlocks));
  return ar.used;
}

// ---- orthonormalising post-processing (Sec. 5) ---------------------------------------------
static rh_status ortho_tucker_check(int32_t order, const int64_t* dims, const int32_t* ks) {
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr && ks != nullptr, "bad order, dims or ks");
  for (int n = 0; n < order; ++n) {
    RH_CHECK_ARG(dims[n] >= 1, "every dimension must be >= 1");
    RH_CHECK_ARG(ks[n] >= 1 && ks[n] <= dims[n] && ks[n] <= RH_MAX_ELL, "need 1 <= k_n <= min(I_n, 64)");
  }
  return RH_OK;
}

size_t rh_orthonormalize_tucker_workspace_size(int32_t order, const int64_t* dims, const int32_t* ks) {
  if (ortho_tucker_check(order, dims, ks) != RH_OK) return 0;
  size_t orth = 1, q = 1, ncore = 1;
  for (int n = 0; n < order; ++n) {
    orth = std::max(orth, orth_workspace_elems(dims[n], ks[n]));
    q = std::max(q, (size_t)dims[n] * ks[n]);
    ncore *= (size_t)ks[n];
  }
  Arena ar(nullptr);
  ar.take<double>(orth);
  ar.take<double>(q);
  ar.take<double>((size_t)RH_MAX_ELL * RH_MAX_ELL);
  ar.take<double>(ncore);
  ar.take<double>(ncore);
  return ar.used;
}

rh_status rh_orthonormalize_tucker(int32_t order, const int64_t* dims, const int32_t* ks, double* const* factors,
                                   double* core, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_status s = ortho_tucker_check(order, dims, ks);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(factors != nullptr && core != nullptr, "factors and core must be non-NULL");
  for (int n = 0; n < order; ++n) RH_CHECK_ARG(factors[n] != nullptr, "every factors[n] must be non-NULL");
  const size_t need = rh_orthonormalize_tucker_workspace_size(order, dims, ks);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  size_t orth = 1, q = 1;
  int64_t ncore = 1;
  for (int n = 0; n < order; ++n) {
    orth = std::max(orth, orth_workspace_elems(dims[n], ks[n]));
    q = std::max(q, (size_t)dims[n] * ks[n]);
    ncore *= ks[n];
  }
  Arena ar(workspace);
  double* ows = ar.take<double>(orth);
  double* Q = ar.take<double>(q);
  double* R = ar.take<double>((size_t)RH_MAX_ELL * RH_MAX_ELL);
  double* bufs[2] = {ar.take<double>((size_t)ncore), ar.take<double>((size_t)ncore)};
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> kd(ks, ks + order);
  const double* in = core;
  int nb = 0;
  for (int n = 0; n < order; ++n) {
    const int64_t I = dims[n];
    const int k = ks[n];
    // A_n = Q_n R_n: Q_n by the thin QR of Alg. 1 step 2 (column signs: largest entry positive),
    // R_n = Q_n^T A_n (k x k, the mode-0 product of the I x k matrix A_n)
    if ((s = launch_orthonormalize(I, k, factors[n], Q, nullptr, ows, st, false)) != RH_OK) return s;
    if ((s = launch_ttm<double, double>(ModeView{1, I, (int64_t)k}, factors[n], Q, k, R, st)) != RH_OK) return s;
    // G <- G x_n R_n (G_(n) <- R_n G_(n)); R_n(c, i) = R[c + k i]
    if ((s = launch_ttm_strided<double, double>(mode_view(order, kd.data(), n), in, R, k, 1, k, bufs[nb], st)) !=
        RH_OK)
      return s;
    in = bufs[nb];
    nb ^= 1;
    RH_CUDA_TRY(cudaMemcpyAsync(factors[n], Q, sizeof(double) * I * k, cudaMemcpyDeviceToDevice, st));
  }
  RH_CUDA_TRY(cudaMemcpyAsync(core, in, sizeof(double) * ncore, cudaMemcpyDeviceToDevice, st));
  return RH_OK;
}

rh_status rh_tucker_residual(int32_t order, const int64_t* dims, int32_t dtype, const void* X,
                             const double* const* factors, const int32_t* ks, const double* core, double* out,
                             void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_status s = check_tensor_args(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(ks != nullptr && factors != nullptr && X != nullptr && core != nullptr && out != nullptr,
               "X, factors, ks, core and out must be non-NULL");
  for (int n = 0; n < order; ++n) {
    RH_CHECK_ARG(ks[n] >= 1, "every k_n must be >= 1");
    RH_CHECK_ARG(factors[n] != nullptr, "every factors[n] must be non-NULL");
  }
  const size_t need = rh_tucker_residual_workspace_size(order, dims, dtype, ks);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  int fused;
  std::vector<int> pre;
  size_t mi, fe;
  int64_t parts;
  resid_plan(order, dims, ks, fused, pre, mi, fe, parts);
  Arena ar(workspace);
  const size_t es = esize(dtype);
  char* fac = ar.take<char>(fe * es);
  char* w0 = ar.take<char>(mi * es);
  char* w1 = ar.take<char>(mi * es);
  double* part = ar.take<double>((size_t)std::max<int64_t>(parts, kNormBlocks));
  cudaStream_t st = (cudaStream_t)stream;
  auto run = [&](auto tag) -> rh_status {
    using T = decltype(tag);
    T* f = reinterpret_cast<T*>(fac);
    std::vector<int64_t> cur(ks, ks + order);
    const int64_t ncore = prod(cur);
    rh_status s2;
    if ((s2 = cast_to<T>(core, f, ncore, st)) != RH_OK) return s2;
    const T* in = f;
    std::vector<const T*> fc(order);
    size_t off = (size_t)ncore;
    for (int n = 0; n < order; ++n) {
      if ((s2 = cast_to<T>(factors[n], f + off, dims[n] * (int64_t)ks[n], st)) != RH_OK) return s2;
      fc[n] = f + off;
      off += (size_t)dims[n] * ks[n];
    }
    T* bufs[2] = {reinterpret_cast<T*>(w0), reinterpret_cast<T*>(w1)};
    int nb = 0;
    for (int n : pre) {
      // expand mode n: Y(.., i, ..) = sum_c A_n(i, c) T(.., c, ..), A_n column-major I_n x k_n
      const ModeView v = mode_view(order, cur.data(), n);
      if ((s2 = launch_ttm_strided<T, T>(v, in, fc[n], dims[n], 1, (int)dims[n], bufs[nb], st)) != RH_OK) return s2;
      in = bufs[nb];
      nb ^= 1;
      cur[n] = dims[n];
    }
    const ModeView v = mode_view(order, cur.data(), fused);
    if ((s2 = launch_ttm_residual<T>(v, in, fc[fused], dims[fused], 1, (int)dims[fused], static_cast<const T*>(X),
                                     part, out, st)) != RH_OK)
      return s2;
    int64_t n = 1;
    for (int k = 0; k < order; ++k) n *= dims[k];
    return sumsq_big<T>(static_cast<const T*>(X), n, part, out + 1, st);
  };
  if (dtype == RH_F64) return run(double());
  return run(float());
}

}  // extern "C"
