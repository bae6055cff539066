// Launchers shared between the translation units of the library (host side).
#pragma once

#include "common.cuh"

namespace rh {

// ---- sketch Y = G_(n) Omega_n  (sketch.cu) -----------------------------------------
struct SketchPlan {
  ModeView v;
  int ell, ellp;      // ellp: Omega columns computed (padded ell)
  int gx, S;
  int64_t chunk;
  int ti = 0;         // small-row kernel (I <= 128, ell <= 32): rows per CTA; 0 = the general kernel
  int64_t row0 = 0;   // Omega row of Kolda column 0 (a slab of a larger tensor: its global offset)
  size_t part_elems() const { return (size_t)S * ell * v.I; }
  size_t norm_elems() const { return (size_t)S * gx; }
};
SketchPlan plan_sketch(const ModeView& v, int ell);

template <typename T>
rh_status launch_sketch(const SketchPlan& pl, const T* G, uint64_t seed, uint32_t sid, T* part, double* part_norm,
                        cudaStream_t st);
template <typename T>
rh_status launch_sketch_reduce(const SketchPlan& pl, const T* part, const double* part_norm, double* Y,
                               double* norm2, cudaStream_t st, int site = SITE_SKETCH_REDUCE, int accumulate = 0);
// Y = G_(n) W with a dense M x ell operand W stored like a mode product's output, (L, ell, R):
// element (p, c) at (p % L) + L (c + ell (p / L)) -- the sketch of a subspace-iteration step.
// split (FP32): every element of G enters as the sum of its exact BF16 head and tail.  Partial
// sketches in part (pl.part_elems()), summed by launch_sketch_reduce (no norm).
SketchPlan plan_sketch_dense(const ModeView& v, int ell);
template <typename T>
rh_status launch_sketch_dense(const SketchPlan& pl, const T* G, const T* W, bool split, T* part, cudaStream_t st,
                              int site);

// ---- tensor-core sketch over BF16 pieces (sketch_tc.cu) --------------------------------
bool sketch_tc_supported(const ModeView& v, int ell);
int sketch_tc_ctas(const ModeView& v);
rh_status launch_sketch_tc(const ModeView& v, int ell, const uint16_t* piece0, const uint16_t* piece1, uint64_t seed,
                           uint32_t sid, float* part, int32_t* err, cudaStream_t st, int64_t row0 = 0);
// FP32 input split on the fly into the same two pieces (pieces = 3: an exact three-piece split);
// norm_part (sketch_tc_ctas doubles, may be NULL) receives per-CTA sums of squares of the split
// values
rh_status launch_sketch_tc_f32(const ModeView& v, int ell, const float* X, uint64_t seed, uint32_t sid, float* part,
                               double* norm_part, int32_t* err, cudaStream_t st, int64_t row0 = 0, int pieces = 2);
// E4M3 input (leading dimension ld, one FP32 scale per 128 bytes of storage), dequantized and
// split on the fly into the same two pieces as FP32 input
rh_status launch_sketch_tc_fp8(const ModeView& v, int ell, const uint8_t* X, const float* scales, int64_t ld,
                               uint64_t seed, uint32_t sid, float* part, double* norm_part, int32_t* err,
                               cudaStream_t st, int64_t row0 = 0);
// A mode with L > 1 (L % 64 == 0) on the tensor cores: the FP32 tensor read through its 3-D view
// (l, i, r), split on the fly, K-major pieces (rows i, K = l); same partial sketches as launch_sketch_tc_f32
bool sketch_tc_strided_supported(const ModeView& v, int ell);
rh_status launch_sketch_tc_f32s(const ModeView& v, int ell, const float* X, uint64_t seed, uint32_t sid, float* part,
                                double* norm_part, int32_t* err, cudaStream_t st, int64_t row0 = 0, int pieces = 2);
// A first mode with few rows (L = 1, I <= 128, ell <= 32) on the tensor cores as grouped operations
// (small_tc.cu).  The input in one of the BF16 forms: RH_F32_BF16X2 (FP32, split on the fly into
// head + tail), RH_BF16, RH_BF16X2 (the two pieces) or RH_FP8_E4M3 (bytes at stride ld, scales).
// The sketch writes the partial sketches of plan_sketch_small_tc (part [S][ell][I], FP32; part_norm
// [S] or NULL), summed by launch_sketch_reduce<float>; the mode product writes B[c + ell p] (FP32)
// from the FP64 Q (I x ell) split into two BF16 pieces.
struct SmallInput {
  const void* X;
  int32_t form;
  int64_t ld = 0;                 // RH_FP8_E4M3
  const float* scales = nullptr;  // RH_FP8_E4M3
};
bool small_tc_supported(const ModeView& v, int ell);
SketchPlan plan_sketch_small_tc(const ModeView& v, int ell);
rh_status launch_sketch_small_tc(const SketchPlan& pl, const SmallInput& in, uint64_t seed, uint32_t sid, float* part,
                                 double* part_norm, int32_t* err, cudaStream_t st, int site = SITE_SKETCH);
rh_status launch_ttm_small_tc(const ModeView& v, const SmallInput& in, const double* Q, int ell, float* B, int32_t* err,
                              cudaStream_t st, int site = SITE_MODE_PRODUCT);
rh_status launch_sum_n(const double* part, int n, double* out, cudaStream_t st, int accumulate = 0);
rh_status launch_split_bf16x2(const float* x, int64_t n, uint16_t* hi, uint16_t* lo, cudaStream_t st);
// ||X_1 + X_2||^2 of BF16 pieces (piece1 may be NULL); part holds 1024 doubles
rh_status launch_pieces_sumsq(const uint16_t* piece0, const uint16_t* piece1, int64_t n, double* part, double* out,
                              cudaStream_t st);

// ---- tensor-core mode product of the first mode (ttm_tc.cu) ---------------------------
bool ttm_tc_supported(const ModeView& v, int ell);
int ttm_tc_ctas(const ModeView& v);
// qa: 128 x I BF16 scratch for the split Q; B: ell x M FP32 (layout c + ell p)
rh_status launch_ttm_tc(const ModeView& v, int ell, const uint16_t* piece0, const uint16_t* piece1, const double* Q,
                        uint16_t* qa, float* B, int32_t* err, cudaStream_t st, double* gram_part = nullptr);
// FP32 X split on the fly into two BF16 pieces (pieces = 3: exactly, into three).  gram_part
// (ell <= 60, ttm_tc_gram_supported): also the FP32 Gram route's per-CTA partials of W = B B^T
// (ttm_tc_ctas(v) upper triangles of ell^2 doubles), see launch_trunc_svd.
bool ttm_tc_gram_supported(int ell);
rh_status launch_ttm_tc_f32(const ModeView& v, int ell, const float* X, const double* Q, uint16_t* qa, float* B,
                            int32_t* err, cudaStream_t st, int pieces = 2, double* gram_part = nullptr);
// a mode with L > 1 (L % 128 == 0): B in the (L, ell, R) layout, qa 128 x ceil8(I) BF16
bool ttm_tc_strided_supported(const ModeView& v, int ell);
rh_status launch_ttm_tc_f32s(const ModeView& v, int ell, const float* X, const double* Q, uint16_t* qa, float* B,
                             int32_t* err, cudaStream_t st, int pieces = 2, double* gram_part = nullptr);
// G <- U^T B on the tensor cores for a truncated core (Alg. 1 step 6): B ell x M FP32 (layout
// c + ell p, split on the fly), U ell x ko FP32 (split into two BF16 pieces in qa, 128 x ceil8(ell)),
// out[co.base(p) + c co.cstride()] FP32 (see CoreOut).  Needs ell % 4 == 0, ell, ko <= 64.
bool core_product_tc_supported(int ell, int ko, int64_t M);
rh_status launch_core_product_tc(const float* B, int ell, int ko, int64_t M, CoreOut co, const float* U, uint16_t* qa,
                                 float* out, int32_t* err, cudaStream_t st, int pieces = 2);
rh_status launch_ttm_tc_fp8(const ModeView& v, int ell, const uint8_t* X, const float* scales, int64_t ld,
                            const double* Q, uint16_t* qa, float* B, int32_t* err, cudaStream_t st,
                            double* gram_part = nullptr);

// ---- mode-n product B = G x_n Q^T  (ttm.cu) ------------------------------------------
// B[(p%L) + L*ko*(p/L) + L*c] = sum_i Q[i + I*c] G[(p%L) + L*I*(p/L) + L*i],  c < ko.
template <typename T, typename TO>
rh_status launch_ttm(const ModeView& v, const T* G, const T* Q, int ko, TO* B, cudaStream_t st, int site = SITE_OTHER);
// general factor layout: Q(i, c) = Q[i qsi + c qsc]; any ko >= 1
template <typename T, typename TO>
rh_status launch_ttm_strided(const ModeView& v, const T* G, const T* Q, int64_t qsi, int64_t qsc, int ko, TO* B,
                             cudaStream_t st);
// *out = sum (Xref - G x_n Q^T)^2 with Xref laid out like the product; part holds
// ttm_resid_parts(v, ko) doubles
int64_t ttm_resid_parts(const ModeView& v, int ko);
template <typename T>
rh_status launch_ttm_residual(const ModeView& v, const T* G, const T* Q, int64_t qsi, int64_t qsc, int ko,
                              const T* Xref, double* part, double* out, cudaStream_t st);

// ---- truncated core of one mode (core_product.cu) ---------------------------------------
// out[co.base(p) + c co.cstride()] = sum_k U[k + ell c] B[k + ell p], p < M, c < ko
// (B: ell x M FP32 with c fastest; ell, ko <= 64; M % (co.S co.I) == 0).
template <typename TO>
rh_status launch_core_product(const float* B, int ell, int ko, int64_t M, CoreOut co, const float* U, TO* out,
                              cudaStream_t st);

// ---- core G = X x_1 A_1^T ... x_d A_d^T (tucker.cu) ----------------------------------------
// returns the elements of each of the two ping-pong buffers; *fac_elems = sum I_n k_n
size_t core_chain_elems(int d, const int64_t* dims, const int32_t* ks, size_t* fac_elems);
// split_tc: FP32 data in the RH_F32_BF16X2 form, the products the tensor-core mode product covers run
// there (qa: 128 x ceil8(max I_n) BF16 scratch, err: wait status; pieces = 3: the exact split)
template <typename T>
rh_status launch_core_ttm(int d, const int64_t* dims, const T* X, const double* const* factors, const int32_t* ks,
                          double* G, T* fac, T* W0, T* W1, cudaStream_t st, bool split_tc = false,
                          uint16_t* qa = nullptr, int32_t* err = nullptr, int pieces = 2);

// ---- small dense linear algebra (smallla.cu) --------------------------------------------
size_t orth_workspace_elems(int64_t m, int n);   // doubles
// f32: FP32 data -- the second CholeskyQR pass (on the nearly orthonormal Q_1) in FP32 and the first
// pass's Cholesky factor in double-float (the Householder branch still takes over on a breakdown)
rh_status launch_orthonormalize(int64_t m, int n, const double* Y, double* Q, int32_t* info, double* ws,
                                cudaStream_t st, bool f32 = false);

// Truncation of B (mode-n unfolding of a L x ell x R tensor, entries of type T):
// TSQR of B_(n)^T, one-sided Jacobi SVD of the ell x ell triangle -> U_B (ell x ell, FP64,
// columns sorted by decreasing singular value) and the singular values.
struct TruncPlan {
  ModeView v;         // view of B: (L, ell, R)
  int ell;
  int rows0;          // rows per first-level block
  int fan;            // blocks merged per higher level
  int64_t nblk0;      // first-level blocks
};
TruncPlan plan_trunc(const ModeView& vb, int ell);
template <typename T>
size_t trunc_workspace_elems(const TruncPlan& pl);   // elements of T
// FP32 data with a truncation rank r (1..ell) first try the Gram route: W = B B^T (FP64 sums of
// FP32 tile sums), Cholesky W = R^T R, Jacobi on R.  It is kept when the Cholesky succeeds and
// sigma_r^2 - sigma_{r+1}^2 >= 1e-5 sigma_1^2 (then *info |= 2, if info is given); otherwise
// device-side flags run the tall-skinny QR route.  r = 0 (and FP64) take the QR route only.
// gram_nparts > 0: the FP32 Gram route's per-CTA partials of W = B B^T were already written (by the
// tensor-core mode product that produced B) into trunc_gram_part(pl, ws), gram_nparts of them, so
// only their reduction runs here.
template <typename T>
rh_status launch_trunc_svd(const TruncPlan& pl, const T* B, T* ws, double* Ub, double* sv, cudaStream_t st, int r,
                           int32_t* info, int gram_nparts = 0);
// Where launch_trunc_svd<float> keeps the per-CTA partials of its Gram route (gram_ctas() ell^2
// doubles) inside its workspace ws.
double* trunc_gram_part(const TruncPlan& pl, float* ws);
int gram_ctas();

// Staged truncation (adaptive variants).  Stage 1, the factor of the whole ell x M matrix B:
// gram (FP32 data) -> W = B B^T in W (part: gram partials, see launch_gram_f32); otherwise the
// tall-skinny QR triangle R of B^T (inside ws, *R points at it).  rownorm2[c] = ||row c of B||^2.
// Stage 2, the SVD of the leading k rows of B from that factor: U_B (k x k) and sv (k), through
// the pivoted Cholesky of W[0:k, 0:k] and the row Jacobi (flag <- 1 on a Cholesky breakdown), or
// through the Jacobi SVD of R[0:k, 0:k] (Wk, Xf, Rk: k x k scratch).
template <typename T>
rh_status launch_trunc_factor(const TruncPlan& pl, const T* B, T* ws, bool gram, double* part, double* W, T** R,
                              double* rownorm2, cudaStream_t st, bool df = false);
template <typename T>
rh_status launch_trunc_leading_svd(int n, int k, bool gram, const double* W, const T* R, double* Wk, float* Xf,
                                   T* Rk, double* Ub, double* sv, int32_t* flag, cudaStream_t st);
int gram_ctas();

// A = Q * Ub(:, 0:r)  (I x r, FP64);  Uc = (T) Ub(:, 0:r) (ell x r)
template <typename T>
rh_status launch_factor_and_cast(int64_t I, int ell, int r, const double* Q, const double* Ub, double* A, T* Uc,
                                 cudaStream_t st);
template <typename T>
rh_status launch_cast(const double* src, T* dst, int64_t n, cudaStream_t st, int site = SITE_CAST_Q);

// Basis of a subspace-iteration step: B (the (L, ell, R) view of tr, entries T) is replaced by W, an
// orthonormal basis of range(B^T) stored in the same layout (tall-skinny Householder R, W = B^T R^{-1},
// one CholeskyQR pass).  ws holds power_workspace_elems(tr) elements of T.
// R (n x n FP64, upper) of the tall-skinny Householder QR of B^T; ws: trunc_workspace_elems(tr) of T
template <typename T>
rh_status launch_tall_skinny_r(const TruncPlan& tr, const T* B, T* ws, double* R, cudaStream_t st);
template <typename T>
size_t power_workspace_elems(const TruncPlan& tr);
template <typename T>
rh_status launch_power_basis(const TruncPlan& tr, T* B, T* ws, cudaStream_t st);
// ||x||^2 (FP64); with a scratch part of part_elems >= 2 doubles a large x is summed over many CTAs
rh_status launch_sumsq(const double* x, int64_t n, double* out, cudaStream_t st, double* part = nullptr,
                       size_t part_elems = 0);

}  // namespace rh
