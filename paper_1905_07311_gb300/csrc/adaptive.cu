// Adaptive-rank randomized HOSVD and STHOSVD (Sec. 4: Alg. 4 and Alg. 5 with the adaptive range
// finder).  The paper names a blocked randomized QB without listing it; the reading used here
// (and by the oracle): grow Q by blocks of b columns of one Gaussian stream until
// ||G - Q Q^T G||_F <= tau, tau = eps ||X||_F / sqrt(d) (absolute, norm of the input), add p more
// columns of the same stream, then take the SVD of B = Q^T G and keep the smallest r whose discarded
// energy sum_{i>r} sigma_i^2 + ||G - Q B||^2 is <= tau^2.
//
// Without power iteration the span of the first k columns of that Q is the span of G Omega(:, 1:k),
// and the thin QR of the whole sketch is column-prefix consistent, so one sketch of width
// ell = cap + p gives every candidate at once: with B = Q^T G (ell rows),
//   ||G - Q_k Q_k^T G||^2 = ||G||^2 - sum_{i<=k} ||B(i,:)||^2,
// and the SVD of the leading k + p rows of B comes from the leading (k+p) x (k+p) block of the
// triangle R of B^T (B B^T = R^T R) or of the Gram matrix W = B B^T.  The row norms are the column
// norms of R (the diagonal of W).  The chosen sizes drive the next launches, so the call
// synchronises its stream once per mode (twice when a Gram factorization falls back).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rh {
namespace {

// Ucpad (ell x r) = [Uc (k x r); 0]
template <typename T>
__global__ void pad_rows_kernel(const T* __restrict__ Uc, int k, int r, int ell, T* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ell * r; e += gridDim.x * blockDim.x) {
    const int i = e % ell, c = e / ell;
    out[e] = i < k ? Uc[i + k * c] : T(0);
  }
}

struct AdaptSizes {
  size_t part = 0, pnorm = 0, I_ell = 0, orth = 0, tensor = 0, trunc = 0, fac = 0, chain = 0;
  size_t tc_part = 0, qa = 0, tc_norm = 0;   // tensor-core first mode (low-precision input forms)
};

// The stored input of a low-precision form, read by the tensor-core kernels on the first mode.
struct TcInput {
  int32_t form = -1;   // RH_BF16, RH_BF16X2, RH_F32_BF16X2 or RH_FP8_E4M3; -1: none
  const void* X = nullptr;
};

struct AdaptBufs {
  void* part;
  double* pnorm;
  double *Y, *Q, *orth;
  void* Qc;
  void* G[2];
  void* B;
  void* trunc;
  double *gpart, *W, *Wk, *d, *Ub, *sv, *norm2, *normx;
  float* Xf;
  void *Rk, *Uc, *Ucpad, *fac, *chain[2];
  int32_t* flag;
  float* tc_part;
  uint16_t* qa;
  double* tc_norm;
  int32_t* err;
};

size_t tsize(int32_t dtype) { return dtype == RH_F64 ? sizeof(double) : sizeof(float); }

// upper bounds for every buffer: every mode planned on the input sizes with ell = cap + p
rh_status adapt_sizes(int32_t order, const int64_t* dims, int32_t dtype, int32_t variant, const int32_t* caps,
                      int p, AdaptSizes& z) {
  std::vector<int32_t> ells(order);
  for (int n = 0; n < order; ++n) {
    const ModeView v = mode_view(order, dims, n);
    const int64_t ell = std::min<int64_t>((int64_t)caps[n] + p, std::min<int64_t>(v.I, v.M()));
    ells[n] = (int32_t)ell;
    if (ell > RH_MAX_ELL) {
      set_error("unsupported: max_ranks[n] + p exceeds RH_MAX_ELL (64) for mode " + std::to_string(n));
      return RH_EUNSUPPORTED;
    }
    const SketchPlan sk = plan_sketch(v, (int)ell);
    z.part = std::max(z.part, sk.part_elems());
    z.pnorm = std::max(z.pnorm, sk.norm_elems());
    z.I_ell = std::max(z.I_ell, (size_t)(v.I * ell));
    z.orth = std::max(z.orth, orth_workspace_elems(v.I, (int)ell));
    z.tensor = std::max(z.tensor, (size_t)(v.M() * ell));
    const TruncPlan tp = plan_trunc(ModeView{v.L, (int64_t)ell, v.R}, (int)ell);
    z.trunc = std::max(z.trunc, dtype == RH_F64 ? trunc_workspace_elems<double>(tp) : trunc_workspace_elems<float>(tp));
  }
  z.tensor = std::max<size_t>(z.tensor, (size_t)std::accumulate(dims, dims + order, int64_t(1), std::multiplies<int64_t>()));
  if (dtype != RH_F64 && dtype != RH_F32) {
    const ModeView v0 = mode_view(order, dims, 0);
    z.tc_part = (size_t)sketch_tc_ctas(v0) * ells[0] * v0.I;
    z.qa = (size_t)128 * v0.I;
    z.tc_norm = (size_t)sketch_tc_ctas(v0);
    z.pnorm = std::max<size_t>(z.pnorm, 1024);   // partial sums of the norm of BF16 pieces
  }
  if (variant == 0) {
    size_t fe = 0;
    z.chain = core_chain_elems(order, dims, ells.data(), &fe);   // the kept ranks are at most ell_n
    z.fac = fe;
  }
  return RH_OK;
}

AdaptBufs carve_adapt(Arena& ar, const AdaptSizes& z, int32_t dtype, int32_t variant) {
  dtype = dtype == RH_F64 ? RH_F64 : RH_F32;   // intermediates of the low-precision forms are FP32
  const size_t ts = tsize(dtype);
  auto takeT = [&](size_t n) -> void* { return (void*)ar.take<char>(n * ts); };
  AdaptBufs b;
  b.part = takeT(z.part);
  b.pnorm = ar.take<double>(z.pnorm);
  b.Y = ar.take<double>(z.I_ell);
  b.Q = ar.take<double>(z.I_ell);
  b.orth = ar.take<double>(z.orth);
  b.Qc = takeT(z.I_ell);
  b.G[0] = takeT(z.tensor);
  b.G[1] = variant == 1 ? takeT(z.tensor) : nullptr;
  b.B = takeT(z.tensor);
  b.trunc = takeT(z.trunc);
  b.gpart = ar.take<double>((size_t)gram_ctas() * RH_MAX_ELL * RH_MAX_ELL);
  b.W = ar.take<double>(RH_MAX_ELL * RH_MAX_ELL);
  b.Wk = ar.take<double>(RH_MAX_ELL * RH_MAX_ELL);
  b.d = ar.take<double>(RH_MAX_ELL);
  b.Ub = ar.take<double>(RH_MAX_ELL * RH_MAX_ELL);
  b.sv = ar.take<double>(RH_MAX_ELL);
  b.norm2 = ar.take<double>(1);
  b.normx = ar.take<double>(1);
  b.Xf = ar.take<float>(RH_MAX_ELL * RH_MAX_ELL);
  b.Rk = takeT(RH_MAX_ELL * RH_MAX_ELL);
  b.Uc = takeT(RH_MAX_ELL * RH_MAX_ELL);
  b.Ucpad = takeT(RH_MAX_ELL * RH_MAX_ELL);
  b.fac = variant == 0 ? takeT(std::max<size_t>(z.fac, 1)) : nullptr;
  b.chain[0] = variant == 0 ? takeT(z.chain) : nullptr;
  b.chain[1] = variant == 0 ? takeT(z.chain) : nullptr;
  b.flag = ar.take<int32_t>(4);
  b.tc_part = z.tc_part ? ar.take<float>(z.tc_part) : nullptr;
  b.qa = z.qa ? ar.take<uint16_t>(z.qa) : nullptr;
  b.tc_norm = z.tc_norm ? ar.take<double>(z.tc_norm) : nullptr;
  b.err = ar.take<int32_t>(4);
  return b;
}

// smallest r >= 1 with sum_{i>r} sv_i^2 + res2 <= tau2 (r = k when none)
int trim_rank(const std::vector<double>& sv, double res2, double tau2) {
  const int k = (int)sv.size();
  std::vector<double> tail(k + 1, 0.0);
  for (int i = k - 1; i >= 0; --i) tail[i] = tail[i + 1] + sv[i] * sv[i];
  for (int r = 1; r <= k; ++r)
    if (tail[r] + res2 <= tau2) return r;
  return k;
}

// One adaptive RandSVD of the mode-n unfolding of G (view v).  *tau2 < 0 on the first call: it is
// then set to eps^2 ||G||^2 / d from this pass's norm (G = X on the first mode of either variant).
// Writes A_n (I x r) into factor; leaves B (ell x M in the view (L, ell, R)) and U_r padded to ell
// rows (Ucpad) for the caller's core update.
// Sketch of the first mode (with ||X||^2) on the tensor cores, straight from the stored form.
rh_status tc_sketch(const ModeView& v, int ell, const TcInput& in, uint64_t seed, uint32_t sid, const AdaptBufs& bf,
                    cudaStream_t st) {
  rh_status s;
  const int S = sketch_tc_ctas(v);
  RH_CUDA_TRY(cudaMemsetAsync(bf.err, 0, sizeof(int32_t), st));
  const uint16_t* p0 = static_cast<const uint16_t*>(in.X);
  const uint16_t* p1 = in.form == RH_BF16X2 ? p0 + v.I * v.M() : nullptr;
  if (in.form == RH_F32_BF16X2) {
    s = launch_sketch_tc_f32(v, ell, static_cast<const float*>(in.X), seed, sid, bf.tc_part, bf.tc_norm, bf.err, st);
  } else if (in.form == RH_FP8_E4M3) {
    const int64_t dims2[2] = {v.I, v.M()};
    const Fp8Layout f8 = fp8_layout(2, dims2);
    const uint8_t* x8 = static_cast<const uint8_t*>(in.X);
    s = launch_sketch_tc_fp8(v, ell, x8, reinterpret_cast<const float*>(x8 + f8.scale_off), f8.ld, seed, sid,
                             bf.tc_part, bf.tc_norm, bf.err, st);
  } else {
    s = launch_sketch_tc(v, ell, p0, p1, seed, sid, bf.tc_part, bf.err, st);
  }
  if (s != RH_OK) return s;
  SketchPlan rp = plan_sketch(v, ell);
  rp.S = S;
  if ((s = launch_sketch_reduce<float>(rp, bf.tc_part, nullptr, bf.Y, nullptr, st)) != RH_OK) return s;
  if (in.form == RH_F32_BF16X2 || in.form == RH_FP8_E4M3) return launch_sum_n(bf.tc_norm, S, bf.norm2, st);
  return launch_pieces_sumsq(p0, p1, v.I * v.M(), bf.pnorm, bf.norm2, st);
}

rh_status tc_mode_product(const ModeView& v, int ell, const TcInput& in, const AdaptBufs& bf, float* B,
                          cudaStream_t st) {
  if (in.form == RH_F32_BF16X2)
    return launch_ttm_tc_f32(v, ell, static_cast<const float*>(in.X), bf.Q, bf.qa, B, bf.err, st);
  if (in.form == RH_FP8_E4M3) {
    const int64_t dims2[2] = {v.I, v.M()};
    const Fp8Layout f8 = fp8_layout(2, dims2);
    const uint8_t* x8 = static_cast<const uint8_t*>(in.X);
    return launch_ttm_tc_fp8(v, ell, x8, reinterpret_cast<const float*>(x8 + f8.scale_off), f8.ld, bf.Q, bf.qa, B,
                             bf.err, st);
  }
  const uint16_t* p0 = static_cast<const uint16_t*>(in.X);
  const uint16_t* p1 = in.form == RH_BF16X2 ? p0 + v.I * v.M() : nullptr;
  return launch_ttm_tc(v, ell, p0, p1, bf.Q, bf.qa, B, bf.err, st);
}

template <typename T>
rh_status adapt_mode(const ModeView& v, const T* G, const TcInput* tci, int cap, int p, int b_blk, double eps, int d,
                     double* tau2, uint64_t seed, uint32_t sid, const AdaptBufs& bf, double* factor, int* r_out,
                     int* ell_out, double* g2_out, cudaStream_t st, bool qr_only) {
  rh_status s;
  const int ell = (int)std::min<int64_t>((int64_t)cap + p, std::min<int64_t>(v.I, v.M()));
  const int kmax = (int)std::min<int64_t>(cap, std::min<int64_t>(v.I, v.M()));
  // sketch (with ||G||^2), thin QR, mode product B = Q^T G_(n); the first mode of a low-precision
  // form reads the stored tensor on the tensor cores (Omega in BF16, B in FP32)
  T* B = static_cast<T*>(bf.B);
  if (tci) {
    if ((s = tc_sketch(v, ell, *tci, seed, sid, bf, st)) != RH_OK) return s;
    if ((s = launch_orthonormalize(v.I, ell, bf.Y, bf.Q, nullptr, bf.orth, st, true)) != RH_OK) return s;
    if ((s = tc_mode_product(v, ell, *tci, bf, reinterpret_cast<float*>(B), st)) != RH_OK) return s;
  } else {
    const SketchPlan sk = plan_sketch(v, ell);
    if ((s = launch_sketch<T>(sk, G, seed, sid, static_cast<T*>(bf.part), bf.pnorm, st)) != RH_OK) return s;
    if ((s = launch_sketch_reduce<T>(sk, static_cast<const T*>(bf.part), bf.pnorm, bf.Y, bf.norm2, st)) != RH_OK)
      return s;
    if ((s = launch_orthonormalize(v.I, ell, bf.Y, bf.Q, nullptr, bf.orth, st, sizeof(T) == 4)) != RH_OK) return s;
    if ((s = launch_cast<T>(bf.Q, static_cast<T*>(bf.Qc), v.I * ell, st)) != RH_OK) return s;
    if ((s = launch_ttm<T, T>(v, G, static_cast<const T*>(bf.Qc), ell, B, st)) != RH_OK) return s;
  }
  // factor of the whole B: Gram matrix (FP32 data) or the tall-skinny QR triangle; row norms of B
  const TruncPlan tp = plan_trunc(ModeView{v.L, (int64_t)ell, v.R}, ell);
  bool gram = sizeof(T) == 4 && !qr_only;
  T* R = nullptr;
  if ((s = launch_trunc_factor<T>(tp, B, static_cast<T*>(bf.trunc), gram, bf.gpart, bf.W, &R, bf.d, st)) != RH_OK)
    return s;
  std::vector<double> d2(ell);
  double g2 = 0.0;
  RH_CUDA_TRY(cudaMemcpyAsync(d2.data(), bf.d, sizeof(double) * ell, cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaMemcpyAsync(&g2, bf.norm2, sizeof(double), cudaMemcpyDeviceToHost, st));
  int32_t tc_err = 0;
  if (tci) RH_CUDA_TRY(cudaMemcpyAsync(&tc_err, bf.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  if (tc_err != 0) {
    set_error("a tensor-core kernel gave up waiting (code " + std::to_string(tc_err) + ")");
    return RH_ETIMEOUT;
  }
  if (*tau2 < 0.0) *tau2 = eps * eps * g2 / d;
  const double t2 = *tau2;
  // blocked growth: k = b, 2b, ... (the last block capped at kmax) until ||G - Q_k B_k||^2 <= tau^2
  int k = 0;
  double pref = 0.0;
  while (k < kmax) {
    const int nk = std::min(k + b_blk, kmax);
    for (int i = k; i < nk; ++i) pref += d2[i];
    k = nk;
    if (g2 - pref <= t2) break;
  }
  // p more columns of the same stream, then the SVD of the leading kp rows of B and the trim
  const int kp = std::min(k + p, ell);
  double pk = 0.0;
  for (int i = 0; i < kp; ++i) pk += d2[i];
  const double res2 = std::max(0.0, g2 - pk);
  std::vector<double> sv(kp);
  // routes for FP32 data: FP32 Gram (kept when its Cholesky succeeds and the truncation gap is
  // resolved), double-float Gram (kept when its Cholesky succeeds), tall-skinny QR of B^T
  bool df = false;
  for (int attempt = 0; attempt < 3; ++attempt) {
    if ((s = launch_trunc_leading_svd<T>(ell, kp, gram, bf.W, R, bf.Wk, bf.Xf, static_cast<T*>(bf.Rk), bf.Ub, bf.sv,
                                         bf.flag, st)) != RH_OK)
      return s;
    int32_t flag = 0;
    RH_CUDA_TRY(cudaMemcpyAsync(sv.data(), bf.sv, sizeof(double) * kp, cudaMemcpyDeviceToHost, st));
    if (gram) RH_CUDA_TRY(cudaMemcpyAsync(&flag, bf.flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RH_CUDA_TRY(cudaStreamSynchronize(st));
    if (!gram) break;
    const int r = trim_rank(sv, res2, t2);
    const bool gap_ok = r >= kp || sv[0] == 0.0 || (sv[r - 1] * sv[r - 1] - sv[r] * sv[r] >= 1e-5 * sv[0] * sv[0]);
    if (!flag && (gap_ok || df)) break;
    if (!df)
      df = true;       // the FP32 Gram matrix cannot resolve this truncation: the double-float one can
    else
      gram = false;    // the double-float Cholesky broke down: tall-skinny QR of B^T
    if ((s = launch_trunc_factor<T>(tp, B, static_cast<T*>(bf.trunc), gram, bf.gpart, bf.W, &R, bf.d, st, df)) !=
        RH_OK)
      return s;
  }
  const int r = trim_rank(sv, res2, t2);
  if ((s = launch_factor_and_cast<T>(v.I, kp, r, bf.Q, bf.Ub, factor, static_cast<T*>(bf.Uc), st)) != RH_OK) return s;
  pad_rows_kernel<T><<<(int)std::max<int64_t>(1, ceil_div((int64_t)ell * r, 256)), 256, 0, st>>>(
      static_cast<const T*>(bf.Uc), kp, r, ell, static_cast<T*>(bf.Ucpad));
  RH_LAUNCH_CHECK();
  *r_out = r;
  *ell_out = ell;
  *g2_out = g2;
  return RH_OK;
}

template <typename T>
rh_status run_adaptive(int32_t order, const int64_t* dims, const T* X, const TcInput* tci, double eps,
                       int32_t variant, int32_t b_blk, const int32_t* caps, const rh_options& o,
                       double* const* factors, double* core, int32_t* ranks, double* norms, const AdaptBufs& bf,
                       cudaStream_t st) {
  rh_status s;
  std::vector<int> rho(order);
  if (variant == 1 && o.rho[0] >= 0) {
    for (int k = 0; k < order; ++k) rho[k] = o.rho[k];
  } else {
    std::iota(rho.begin(), rho.end(), 0);
    if (variant == 1) std::stable_sort(rho.begin(), rho.end(), [&](int a, int c) { return dims[a] > dims[c]; });
  }
  std::vector<int64_t> cur(dims, dims + order);
  double tau2 = -1.0, nx2 = 0.0;
  const T* G = X;
  int gbuf = -1;
  for (int j = 0; j < order; ++j) {
    const int n = rho[j];
    const ModeView v = variant == 1 ? mode_view(order, cur.data(), n) : mode_view(order, dims, n);
    const uint32_t sid = ((uint32_t)o.tensor_id << 4) | (uint32_t)n;
    int r = 0, ell = 0;
    double g2 = 0.0;
    if ((s = adapt_mode<T>(v, variant == 1 ? G : X, j == 0 ? tci : nullptr, caps[n], o.p, b_blk, eps, order, &tau2,
                           o.seed, sid, bf, factors[n], &r, &ell, &g2, st, o.svd_route != 0)) != RH_OK)
      return s;
    if (j == 0) nx2 = g2;
    ranks[n] = r;
    if (variant == 1) {
      // G <- U_r^T B (Alg. 5: G <- A^T G_(n) = U_r^T Q^T G_(n)), in the usual column-major order
      const ModeView vb{v.L, (int64_t)ell, v.R};
      const bool last = (j == order - 1);
      if (last) {
        if ((s = launch_ttm<T, double>(vb, static_cast<const T*>(bf.B), static_cast<const T*>(bf.Ucpad), r, core,
                                       st)) != RH_OK)
          return s;
      } else {
        const int wg = gbuf == 0 ? 1 : 0;
        if ((s = launch_ttm<T, T>(vb, static_cast<const T*>(bf.B), static_cast<const T*>(bf.Ucpad), r,
                                  static_cast<T*>(bf.G[wg]), st)) != RH_OK)
          return s;
        G = static_cast<const T*>(bf.G[wg]);
        gbuf = wg;
      }
      cur[n] = r;
    }
  }
  if (variant == 0) {
    // Alg. 4 step 6: G = X x_1 A_1^T ... x_d A_d^T
    if ((s = launch_core_ttm<T>(order, dims, X, factors, ranks, core, static_cast<T*>(bf.fac),
                                static_cast<T*>(bf.chain[0]), static_cast<T*>(bf.chain[1]), st)) != RH_OK)
      return s;
  }
  int64_t ncore = 1;
  for (int k = 0; k < order; ++k) ncore *= ranks[k];
  if (norms) {
    RH_CUDA_TRY(cudaMemcpyAsync(norms, &nx2, sizeof(double), cudaMemcpyHostToDevice, st));
    if ((s = launch_sumsq(core, ncore, norms + 1, st)) != RH_OK) return s;
  }
  RH_CUDA_TRY(cudaStreamSynchronize(st));
  return RH_OK;
}

}  // namespace
}  // namespace rh

namespace rh {
namespace {

bool lowp_form(int32_t dtype) {
  return dtype == RH_BF16 || dtype == RH_BF16X2 || dtype == RH_F32_BF16X2 || dtype == RH_FP8_E4M3;
}

// How a low-precision form runs: its first mode on the tensor cores (*tc = true) when mode 0 is
// processed first and the tensor-core kernels cover it; an FP32-split input may instead run as
// plain FP32 (*as_f32 = true); anything else is unsupported.
rh_status lowp_plan(int32_t order, const int64_t* dims, int32_t dtype, int32_t variant, const int32_t* caps,
                    const rh_options& o, bool* tc, bool* as_f32) {
  *tc = false;
  *as_f32 = false;
  if (!lowp_form(dtype)) return RH_OK;
  if (variant != 1) {
    set_error("unsupported: the BF16 and E4M3 forms take the sequential variant (Alg. 5) only");
    return RH_EUNSUPPORTED;
  }
  int first = 0;
  if (o.rho[0] >= 0) {
    first = o.rho[0];
  } else {
    for (int k = 1; k < order; ++k)
      if (dims[k] > dims[first]) first = k;
  }
  const ModeView v0 = mode_view(order, dims, 0);
  const int ell0 = (int)std::min<int64_t>((int64_t)caps[0] + o.p, std::min<int64_t>(v0.I, v0.M()));
  if (first == 0 && sketch_tc_supported(v0, ell0) && ttm_tc_supported(v0, ell0)) {
    *tc = true;
    return RH_OK;
  }
  if (dtype == RH_F32_BF16X2) {
    *as_f32 = true;
    return RH_OK;
  }
  set_error("unsupported: the BF16 and E4M3 forms need mode 0 processed first, I_0 % 8 == 0, I_0 <= 1024 and "
            "max_ranks[0] + p <= 64");
  return RH_EUNSUPPORTED;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" {

size_t adaptive_rank_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t variant,
                                    const int32_t* max_ranks, const rh_options* opts) {
  if (order < 1 || order > RH_MAX_ORDER || dims == nullptr || max_ranks == nullptr) return 0;
  if (dtype != RH_F64 && dtype != RH_F32 && !lowp_form(dtype)) return 0;
  if (variant != 0 && variant != 1) return 0;
  for (int k = 0; k < order; ++k)
    if (dims[k] < 1 || max_ranks[k] < 1) return 0;
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  if (o.power_iters != 0) return 0;
  bool tc = false, as_f32 = false;
  if (lowp_plan(order, dims, dtype, variant, max_ranks, o, &tc, &as_f32) != RH_OK) return 0;
  if (as_f32) dtype = RH_F32;
  AdaptSizes z;
  if (adapt_sizes(order, dims, dtype, variant, max_ranks, o.p, z) != RH_OK) return 0;
  Arena ar(nullptr);
  carve_adapt(ar, z, dtype, variant);
  return ar.used;
}

rh_status adaptive_rank(int32_t order, const int64_t* dims, int32_t dtype, const void* X, double eps,
                        int32_t variant, int32_t block, const int32_t* max_ranks, const rh_options* opts,
                        double* const* factors, double* core, int32_t* ranks, double* norms, void* workspace,
                        size_t workspace_bytes, void* stream) {
  clear_error();
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(dims[k] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(dtype == RH_F64 || dtype == RH_F32 || lowp_form(dtype), "dtype must be a dense input form");
  RH_CHECK_ARG(variant == 0 || variant == 1, "variant must be 0 (Alg. 4) or 1 (Alg. 5)");
  RH_CHECK_ARG(eps > 0.0 && std::isfinite(eps), "eps must be positive");
  RH_CHECK_ARG(block >= 1, "block must be >= 1");
  RH_CHECK_ARG(X != nullptr && factors != nullptr && core != nullptr && ranks != nullptr,
               "X, factors, core and ranks must be non-NULL");
  RH_CHECK_ARG(max_ranks != nullptr, "max_ranks is NULL");
  for (int k = 0; k < order; ++k) {
    RH_CHECK_ARG(max_ranks[k] >= 1, "every max_ranks[n] must be >= 1");
    RH_CHECK_ARG(factors[k] != nullptr, "every factors[n] must be non-NULL");
  }
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  if (o.power_iters != 0) {
    set_error("unsupported: the adaptive range finder runs without subspace iteration (power_iters must be 0)");
    return RH_EUNSUPPORTED;
  }
  RH_CHECK_ARG(o.p >= 0, "oversampling p must be >= 0");
  RH_CHECK_ARG(o.svd_route == 0 || o.svd_route == 1, "svd_route must be 0 or 1");
  RH_CHECK_ARG(o.tensor_id >= 0 && o.tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  if (variant == 1 && o.rho[0] >= 0) {
    std::vector<int> seen(order, 0);
    for (int k = 0; k < order; ++k) {
      RH_CHECK_ARG(o.rho[k] >= 0 && o.rho[k] < order && !seen[o.rho[k]], "rho must be a permutation of 0..order-1");
      seen[o.rho[k]] = 1;
    }
  }
  bool tc = false, as_f32 = false;
  rh_status s = lowp_plan(order, dims, dtype, variant, max_ranks, o, &tc, &as_f32);
  if (s != RH_OK) return s;
  if (as_f32) dtype = RH_F32;
  AdaptSizes z;
  s = adapt_sizes(order, dims, dtype, variant, max_ranks, o.p, z);
  if (s != RH_OK) return s;
  Arena meas(nullptr);
  carve_adapt(meas, z, dtype, variant);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  const AdaptBufs bf = carve_adapt(ar, z, dtype, variant);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == RH_F64)
    return run_adaptive<double>(order, dims, static_cast<const double*>(X), nullptr, eps, variant, block, max_ranks, o,
                                factors, core, ranks, norms, bf, st);
  TcInput tin;
  tin.form = dtype;
  tin.X = X;
  return run_adaptive<float>(order, dims, static_cast<const float*>(X), tc ? &tin : nullptr, eps, variant, block,
                             max_ranks, o, factors, core, ranks, norms, bf, st);
}

}  // extern "C"
