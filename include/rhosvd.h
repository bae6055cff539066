/*
 * rhosvd.h -- C ABI of the GB300 (sm_103a) randomized Tucker compression library.
 *
 * Method: Minster, Saibaba, Kilmer, "Randomized algorithms for low-rank tensor
 * decompositions in the Tucker format".  The library computes, on one GPU:
 *   - the randomized range finder on a mode-n unfolding, Y_n = X_(n) Omega_n with a
 *     Gaussian Omega_n of ell = r_n + p columns generated on the fly (Alg. 1 step 1,
 *     Sec. 3.1), followed by a thin QR (Alg. 1 step 2);
 *   - the mode-n products that form the core (Alg. 1 step 3, Alg. 2 step 6,
 *     Alg. 3 step 6) and the truncation of Alg. 1 steps 4-6.
 *
 * Conventions shared by every entry point
 *   Layout     Dense tensors are column-major: X(i_1,...,i_d) lives at
 *              i_1 + I_1 (i_2 + I_2 (i_3 + ...)), 0-based.  The mode-n unfolding
 *              X_(n) (Sec. 2.1) has columns indexed by the remaining indices with the
 *              earliest mode fastest (the order of Eq. kron).  Matrices are
 *              column-major with leading dimension equal to their row count.
 *   Memory     Every data pointer is a DEVICE pointer on the current CUDA device,
 *              owned by the caller.  Inputs are read only.  The library allocates no
 *              device memory: scratch space is the caller's ``workspace`` buffer of
 *              ``workspace_bytes`` bytes (256-byte aligned), sized by the matching
 *              ``*_workspace_size`` query.  Host arrays (dims, ranks, rho, the
 *              arrays of factor pointers) are read during the call only.
 *   Streams    ``stream`` is a cudaStream_t (NULL = legacy default stream).  Calls
 *              enqueue kernels and return without synchronising; results are ready
 *              when the stream reaches that point.  A call never waits on the device.
 *   Omega      Omega_n(row, col) ~ N(0,1) from Philox4x32-10 (key = seed,
 *              counter = (col/4, row lo, row hi, (tensor_id << 4) | mode)) and a
 *              Box-Muller transform in FP32 with the library's own log / sin / cos.
 *              ``row`` is the Kolda column index of the unfolding being sketched.
 *              The FP64 paths use these FP32 normals promoted exactly.
 *   Errors     Every call returns an rh_status.  Argument errors return RH_EINVAL
 *              before anything is enqueued; a failed launch returns RH_ECUDA.  The
 *              message of the last failure on the calling thread is rh_last_error().
 *              No C++ exception crosses this boundary.
 *   Dtypes     RH_F64: FP64 storage, FP64 arithmetic.  RH_F32: FP32 storage, FP32
 *              products with FP32 accumulation inside a tile and FP64 accumulation
 *              across tiles; the small dense factorizations run in FP64 (QR) or in
 *              the storage precision (truncation SVD).
 */
#ifndef RHOSVD_H
#define RHOSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RH_MAX_ORDER 8
#define RH_MAX_ELL 64

typedef int32_t rh_status;
enum {
  RH_OK = 0,
  RH_EINVAL = 1,        /* bad argument (size rule, null pointer, unsupported combination) */
  RH_ENOMEM = 2,        /* workspace_bytes smaller than the *_workspace_size query        */
  RH_ECUDA = 3,         /* a CUDA launch or runtime call failed                           */
  RH_ENUMERIC = 4,      /* numerical failure detected on the host side                    */
  RH_ETIMEOUT = 5,      /* a bounded device wait gave up                                  */
  RH_EUNSUPPORTED = 6   /* valid request that this build does not implement               */
};

/* Element types of an input tensor.
 *   RH_F64, RH_F32  plain arrays.
 *   RH_BF16         one BF16 array (a tensor stored in BF16).
 *   RH_BF16X2       an FP32 tensor held as two BF16 arrays, head h = bf16(x) and tail
 *                   t = bf16(x - h) (16 significant bits, |x - h - t| <= 2^-16 |x|), stored one after
 *                   the other in a single buffer of 2 N BF16 values (see rh_split_bf16x2).
 *   RH_F32_BF16X2   a plain FP32 array, read as RH_BF16X2: the kernels of the first mode split
 *                   each tile into head and tail in shared memory as they load it, so the results
 *                   are bit-identical to RH_BF16X2 of rh_split_bf16x2(X) without the split pass.
 *                   In rsthosvd a first mode that the tensor-core kernels do not cover (not mode 0,
 *                   or I_0 % 8 != 0, I_0 > 1024) runs in FP32 on the CUDA cores instead of being
 *                   rejected, so the form accepts any FP32 tensor (info bit 4 shows which modes
 *                   ran on the tensor cores).
 *   RH_F32_BF16X3   a plain FP32 array read exactly: every tensor-core kernel of rsthosvd and
 *                   rhosvd (sketches, mode products, core products) splits each FP32 tile into
 *                   three BF16 pieces h = bf16(x), m = bf16(x - h), t = bf16(x - h - m) with
 *                   h + m + t = x (24 significant bits), so every product with a BF16 operand is
 *                   the exact product with x; the factor Q of a mode product and U of a core
 *                   product keep two pieces (16 significant bits).  ||X||^2 is that of the FP32
 *                   values.  Shapes the tensor-core kernels do not cover (and first modes with few
 *                   rows) run in FP32 on the CUDA cores.  Not with subspace iteration
 *                   (power_iters > 0), and not on the grouped engine of rsthosvd_batched (its
 *                   stream engine runs it).
 *   RH_FP8_E4M3     a tensor stored in FP8 E4M3 (OCP FP8: bias 7, max 448, no infinities) with one
 *                   FP32 scale per 128 bytes of storage.  Buffer layout (see rh_fp8_layout): the
 *                   E4M3 bytes column-major with the mode-1 fibres at a stride of ld = I_1 rounded up
 *                   to 16 (padding bytes are ignored), ld x prod_{k>1} I_k bytes, then, from the next
 *                   16-byte boundary, the FP32 scales: element (i, p) of X_(1) has the value
 *                   fl32(e4m3[i + ld p] * scales[(i + ld p) / 128]) (FP32 product, ties to even).
 *                   The kernels of the first mode dequantize each tile in shared memory and round it
 *                   to one BF16 piece (ties to even; E4M3 holds 4 significant bits, so a second piece
 *                   would add nothing but work), so the results are bit-identical to RH_BF16 on
 *                   bf16 of the dequantized values; the first mode must run on the tensor cores.
 * The BF16 forms use the tensor cores (tcgen05) for the first mode's sketch and mode product, with
 * Omega rounded to BF16 (ties to even) and FP32 accumulation; the intermediate cores are FP32.  In
 * R-STHOSVD (truncating) the core after a mode is written with the next mode fastest when that
 * mode is the smallest other one, and that mode then runs on the tensor cores too (its FP32 core
 * split on the fly, Omega in BF16) if I_n % 8 == 0, I_n <= 1024 and r + p <= 64; the other modes
 * run in FP32 on the CUDA cores.  A first mode with few rows (mode 0 processed first, I_0 <= 128,
 * r + p <= 32, any I_0; every BF16 form, without subspace iteration) runs on the small-row
 * tensor-core kernels instead (plain loads converted in shared memory into the same pieces, Omega in
 * BF16, FP32 sums in tensor memory over a CTA's columns and FP64 across CTAs), and every later mode
 * in FP32 on the CUDA cores; such requests can run on the grouped engine of rsthosvd_batched.
 * info bit 4 marks the modes that ran on the tensor cores. */
enum { RH_F64 = 0, RH_F32 = 1, RH_BF16 = 2, RH_BF16X2 = 3, RH_F32_BF16X2 = 4, RH_FP8_E4M3 = 5, RH_F32_BF16X3 = 6 };

/* rh_fp8_layout -- storage of an RH_FP8_E4M3 tensor with sizes dims (see above): *ld = the stride
 * of the mode-1 fibres in bytes, *scale_offset = the byte offset of the scales, *nscales = their
 * count, *bytes = the whole buffer.  Any output pointer may be NULL.  RH_EINVAL on bad sizes. */
rh_status rh_fp8_layout(int32_t order, const int64_t* dims, int64_t* ld, size_t* scale_offset, size_t* nscales,
                        size_t* bytes);

/* Options of the fixed-rank algorithms (Alg. 2, Alg. 3). */
typedef struct rh_options {
  uint64_t seed;                 /* Philox key of every Omega_n                                   */
  int32_t tensor_id;             /* Philox stream word (0 .. 2^28-1); distinguishes tensors      */
  int32_t p;                     /* oversampling, ell_n = r_n + p (Alg. 1 REQUIRE)                */
  int32_t rho[RH_MAX_ORDER];     /* processing order, 0-based; rho[0] < 0: decreasing I_n,       */
                                 /* ties to the lower mode (Sec. 3.3, "Processing order")        */
  int32_t clamp;                 /* 0: RH_EINVAL when r_n + p > min(I_n, prod_{k!=n} I_k)        */
                                 /*    (Alg. 2/3 REQUIRE, checked on the current core);          */
                                 /* 1: ell_n = min(r_n + p, I_n, prod_{k!=n} I_k)                */
  int32_t truncate;              /* 1: rank r_n via the SVD of B (Alg. 1 steps 4-6, default)     */
                                 /* 0: keep all ell_n columns, A_n = Q_n, G <- Q_n^T G           */
  int32_t svd_route;             /* SVD of B for FP32 data: 0 = automatic (FP32 Gram, double-    */
                                 /* float Gram, tall-skinny QR, see rsthosvd); 1 = always the    */
                                 /* tall-skinny Householder QR of B^T (FP64 data always use it)  */
  int32_t power_iters;           /* q >= 0 steps of randomized subspace iteration in each range  */
                                 /* finder (Sec. 5 "Variants", used in Sec. 6): after Q = orth(Y)*/
                                 /* each step sets W = orth(G_(n)^T Q), Y = G_(n) W, Q = orth(Y) */
                                 /* (0 = Alg. 1 as printed; at most 8)                           */
  int32_t select;                /* row selection of the structure-preserving variants (Alg. 6   */
                                 /* step 6; Sec. 5): RH_SELECT_SRRQR (eta = 2, default), _CPQR,  */
                                 /* _DEIM, _UNIFORM, _LEVERAGE (see rh_subset_select); sampling  */
                                 /* draws with seed and stream (tensor_id << 4) | mode          */
  int32_t omega_prec;            /* Omega of the sparse sketches: RH_F32 (FP32 normals, default; */
                                 /* RH_F64 means the same) or RH_BF16 (each normal rounded to     */
                                 /* BF16, ties to even: the BF16-Omega form).  Dense paths ignore*/
                                 /* it (their Omega precision follows the input form)            */
} rh_options;

/* Fill ``opts`` with defaults: seed 0, tensor_id 0, p 5, rho decreasing, clamp 0, truncate 1,
 * svd_route 0, power_iters 0, select RH_SELECT_SRRQR, omega_prec RH_F32. */
void rh_options_default(rh_options* opts);

/* Version string and the message of the last failure on this thread ("" after success). */
const char* rh_version(void);
const char* rh_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all threads). */
uint64_t rh_kernel_launches(void);

/*
 * rh_test_wait_probe -- test support for the bounded waits of the tensor-core kernels (the paper
 * has no counterpart).  After rh_test_wait_probe(k) with k >= 0, the tensor-core launches of the
 * process are counted from 0 and launch number k runs as a probe: right after initialising its
 * mbarriers, before it allocates tensor memory or issues any copy or MMA, each CTA waits a short
 * bounded time on a barrier that nothing arrives at, records wait code 64 in the call's wait
 * status and returns without writing its outputs.  The call that made that launch then reports
 * the give-up as it reports any other: info bit 16 for that mode (rsthosvd, rsthosvd_host), the
 * first int32 of the workspace (rhosvd_sketch, rh_mode_product_bf16), RH_ETIMEOUT (adaptive_rank).
 * k < 0 (the default) turns the probe off.  Process-wide; not for concurrent use with other work.
 */
void rh_test_wait_probe(int64_t launch);

/*
 * Launch-shape knobs of the small-tensor kernels (the paper has no counterpart): how many CTAs the
 * small-row sketches and mode products, and the Gram matrix of B in the truncation, spread one
 * tensor's work over (a minimum of work per CTA and a maximum of CTAs per SM).  Their defaults are a
 * table written by the project's tuner (`python -m paper_1905_07311_gb300.tune`) from measurements
 * of the batched workload.  The setting changes how sums are split over CTAs, so results can differ
 * in the last bits between settings; calls with the same settings give the same results.
 *   rh_tuning_count / rh_tuning_name  the knobs (index 0 .. count - 1; NULL out of range).
 *   rh_tuning_get(name)  the current value, -1 for an unknown name.
 *   rh_tuning_set(name, value)  value in [1, 4096], or 0 for the table's value; RH_EINVAL otherwise.
 *   Process-wide; set them between calls, not while a call of another thread plans its launches.
 */
int32_t rh_tuning_count(void);
const char* rh_tuning_name(int32_t index);
int32_t rh_tuning_get(const char* name);
rh_status rh_tuning_set(const char* name, int32_t value);

/*
 * Per-launch timing of the main kernels (measurement support, off by default).
 *   rh_profile_enable(1) makes later calls bracket these launches with CUDA events on the
 *   caller's stream: kind 0 the sketch kernel, 1 the mode product B = Q^T G_(n),
 *   2 the QR of the sketch, 3 the truncation SVD, 4 the truncated-core mode product,
 *   5 the Jacobi SVD inside the truncation (tag 0);
 *   tag = step of the algorithm (0 = first processed mode).
 *   rh_profile_collect waits for the recorded events, writes up to ``cap`` records
 *   (kind, tag, milliseconds; any pointer may be NULL), clears the list and returns the
 *   number of records that were pending.
 */
void rh_profile_enable(int32_t on);
int32_t rh_profile_collect(int32_t* kinds, int32_t* tags, float* ms, int32_t cap);

/*
 * rh_omega -- materialise a block of Omega_mode (test and inspection use).
 *   Writes out[i + nrows * c] = Omega_mode(row0 + i, c) for 0 <= i < nrows, 0 <= c < ell,
 *   FP32.  Entries are bit-identical to the ones the sketch kernels generate.
 *   Defines the Gaussian test matrix of Alg. 1 (REQUIRE) / Alg. 2 step 2 / Alg. 3 step 3.
 *   RH_EINVAL: nrows < 0, ell < 1, mode not in [0,16), tensor_id not in [0, 2^28), out NULL.
 */
rh_status rh_omega(uint64_t seed, int32_t tensor_id, int32_t mode, int64_t row0, int64_t nrows,
                   int32_t ell, float* out, void* stream);

/*
 * rhosvd_sketch -- range-finder sketch Y = X_(mode) Omega_mode (Alg. 1 step 1 applied to an
 * unfolding, as in Alg. 2 step 3 and Alg. 3 step 4).
 *   X       order-``order`` tensor with sizes dims[0..order-1], column-major, dtype RH_F64/RH_F32, or
 *           RH_BF16/RH_BF16X2/RH_F32_BF16X2/RH_FP8_E4M3 for mode 0 (tensor cores; needs I_0 % 8 == 0,
 *           I_0 <= 1024, or I_0 <= 128 and ell <= 32 on the small-row kernel;
 *           Omega in BF16), or RH_F32_BF16X2 for a later mode whose earlier sizes
 *           multiply to a multiple of 64, I_mode <= 1024 (tensor cores, the FP32 values read through
 *           the 3-D view (l, i, r) of the mode and split on the fly).  norm2 is not computed for RH_BF16/RH_BF16X2 and must be
 *           NULL; for RH_F32_BF16X2 it is ||head + tail||^2 (FP32 sums over 32 values per thread
 *           and tile, FP64 above).  RH_F32_BF16X3: as RH_F32_BF16X2 with the exact three-piece split
 *           (no small-row route: I_0 % 8 == 0 for mode 0), norm2 = ||X||^2 of the FP32 values.
 *   mode    0-based mode n;  ell  number of columns, 1 <= ell <= RH_MAX_ELL.
 *   On the tensor-core forms the first int32 of the workspace receives the wait status once the
 *   stream has synchronised: 0, or the code of a bounded wait that gave up (Y is then invalid).
 *   Y       output, I_n x ell FP64, column-major (ld = I_n).
 *   norm2   optional (may be NULL): receives ||X||_F^2 (one FP64 value), accumulated
 *           in FP64 from the same pass over X.
 *   Omega is generated from (seed, tensor_id, mode); rows are Kolda column indices of X_(n).
 *   RH_EINVAL: order not in [1, RH_MAX_ORDER], a dim < 1, mode out of range, ell out of
 *   range, NULL X / Y.  RH_ENOMEM: workspace too small.
 */
size_t rhosvd_sketch_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode,
                                    int32_t ell);
rh_status rhosvd_sketch(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode,
                        int32_t ell, uint64_t seed, int32_t tensor_id, double* Y, double* norm2,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * rhosvd_sketch_offset -- rhosvd_sketch of a block of consecutive Kolda columns of a larger tensor's
 * unfolding: the rows of Omega_mode used are row0, row0 + 1, ... instead of 0, 1, ...  For a slab
 * X[..., k0:k1] of a tensor cut along its last mode, the slab's mode-n unfolding (n before the last
 * mode) holds the global columns p + L R' k0 (L, R' the products of the sizes before and between),
 * so the slabs' sketches with row0 = L R' k0 add up to the whole tensor's sketch (the partition of
 * Alg. 3 over slabs).  accumulate = 1 adds the slab's sketch (and ||slab||^2) to Y (and *norm2)
 * instead of overwriting them, so slabs streamed one after another sum on the device.  row0 >= 0;
 * the rest as rhosvd_sketch (which is row0 = 0, accumulate = 0).
 */
rh_status rhosvd_sketch_offset(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode,
                               int32_t ell, uint64_t seed, int32_t tensor_id, int64_t row0, int32_t accumulate,
                               double* Y, double* norm2, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_tall_skinny_r -- the triangle R of the tall-skinny Householder QR B_(mode)^T = Q_B R (the
 * factor the truncation of Alg. 1 step 4 starts from), for a tensor whose mode ``mode`` is short
 * (I_mode <= 64): a tree of per-block Householder QRs in B's precision, never the Gram matrix.
 *   R   device, I_mode x I_mode FP64 column-major, upper triangular (zeros below the diagonal); a
 *       block of fewer columns than I_mode gives a trapezoid padded with zero rows.
 *   Triangles of column blocks of one matrix combine by stacking and re-triangularising: the SVD of
 *   B = [B_1 ... B_S] has the left singular vectors of [R_1^T ... R_S^T] (rh_left_svd of that
 *   I_mode x S I_mode matrix), which is how the slab-sharded decomposition truncates.
 */
size_t rh_tall_skinny_r_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode);
rh_status rh_tall_skinny_r(int32_t order, const int64_t* dims, int32_t dtype, const void* B, int32_t mode, double* R,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_cast_f64 -- dst[i] = src[i] converted to RH_F32 (round to nearest even) or copied (RH_F64), for
 * i < n: the FP64 factors in the precision of an FP32 tensor's mode products.  Device pointers.
 *   The paper has no counterpart (a storage-precision helper of the slab partition).  n = 0 does
 *   nothing.  RH_EINVAL: n < 0, a NULL pointer with n > 0, dtype other than RH_F32 / RH_F64.
 */
rh_status rh_cast_f64(const double* src, int64_t n, int32_t dtype, void* dst, void* stream);

/*
 * rh_tucker_factor -- Alg. 1 step 5 with the library's column-sign convention: A = Q Ub(:, 1:r)
 * (I x r FP64), then each column of A flipped so that its largest-magnitude entry (first on ties) is
 * positive, and Ur = Ub(:, 1:r) (ell x r FP64) with the same flips, so that G <- Ur^T B keeps
 * A Ur^T B = Q Ub(:, 1:r) Ub(:, 1:r)^T B.  Q: I x ell, Ub: ell x ell, column-major device FP64.
 */
rh_status rh_tucker_factor(int64_t I, int32_t ell, int32_t r, const double* Q, const double* Ub, double* A, double* Ur,
                           void* stream);

/*
 * rhosvd_sketch_static -- rhosvd_sketch for callers that must not allocate device memory.
 *   The paper has no counterpart: this is a deployment variant of the sketch above, with the
 *   same arguments minus the workspace and the same output (up to the order of the FP32/FP64
 *   partial sums), for the plain forms only: dtype must be RH_F32 or RH_F64 (the BF16 and E4M3
 *   forms that rhosvd_sketch also accepts return RH_EINVAL here).  Its scratch lives in a 16 MiB static device array inside the library that
 *   every GPU loading the library keeps until the process exits; the caller allocates only
 *   X, Y and norm2.  Intended for code that may not call cudaMalloc: plugins whose host
 *   framework owns all device memory, loops that cannot take cudaMalloc's implicit device
 *   synchronisation, processes whose device memory budget is fully reserved.
 *   Limit: I_mode * ell * (4 or 8 bytes) plus a few KB of partial norms must fit in 16 MiB,
 *   otherwise RH_EINVAL with a message (the number of split-K partials shrinks to fit).
 *   Every call outside stream capture looks up the array's address (cudaGetSymbolAddress), so
 *   a device reset, which may move the array, is seen by the next call; a call on a capturing
 *   stream reuses the address of the last uncaptured call on that device, so the first call on
 *   a device must precede any stream capture (RH_EINVAL otherwise), and a graph captured before
 *   a device reset holds the old address like any other captured pointer.  All calls share the array and leave their contents in it;
 *   every element a call reads is written by that call first, but calls that overlap on the
 *   GPU race.  No cudaMalloc, cudaFree or allocating library routine is called.
 */
rh_status rhosvd_sketch_static(int32_t order, const int64_t* dims, int32_t dtype, const void* X,
                               int32_t mode, int32_t ell, uint64_t seed, int32_t tensor_id, double* Y,
                               double* norm2, void* stream);

/*
 * rh_split_bf16x2 -- write the RH_BF16X2 representation of an FP32 array: out[0..n) = bf16(x),
 * out[n..2n) = bf16(x - bf16(x)) (ties to even).  n % 8 == 0 keeps the tail 16-byte aligned.
 *   The paper has no counterpart (the storage form that the tensor-core kernels read; the FP32
 *   split form computes the same pieces inside the kernels).  X: n FP32 values, out: 2 n BF16
 *   values, device pointers owned by the caller.  n = 0 does nothing.  RH_EINVAL: n < 0, a NULL
 *   pointer with n > 0.
 */
rh_status rh_split_bf16x2(const float* X, int64_t n, uint16_t* out, void* stream);

/*
 * rh_orthonormalize -- thin QR of a tall matrix, Y = Q R, returning Q (Alg. 1 step 2).
 *   Y  m x n FP64 column-major (read only), 1 <= n <= RH_MAX_ELL, n <= m.
 *   Q  m x n FP64 column-major output with orthonormal columns spanning range(Y).
 *   Method: CholeskyQR2 in FP64; if a Cholesky pivot falls below 1e-14 of its diagonal
 *   (kappa(Y) beyond ~1e7) the result comes from a Householder QR instead.  The switch
 *   happens on the device (no host synchronisation).  ``info`` (optional device int32)
 *   receives 1 when the Householder branch produced Q, else 0.
 */
size_t rh_orthonormalize_workspace_size(int64_t m, int32_t n);
rh_status rh_orthonormalize(int64_t m, int32_t n, const double* Y, double* Q, int32_t* info,
                            void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_mode_product -- mode-n product (Sec. 2.1: Y = X x_n M means Y_(n) = M X_(n)), the step that
 * forms B = Q^T X in Alg. 1 step 3, the core G = X x_1 A_1^T ... of Alg. 2 step 6 and the
 * reconstruction G x_1 A_1 ... of a Tucker tensor.
 *   X          tensor (order, dims, dtype), column-major.
 *   transpose  1: A is I_mode x k (column-major), Y = X x_mode A^T;
 *              0: A is k x I_mode (column-major), Y = X x_mode A.   A has X's dtype; k >= 1.
 *   Y          output tensor with dims[mode] replaced by k, column-major, out_dtype = dtype or
 *              RH_F64 (FP32 input with FP64 output).  The unfolding is never materialised.
 */
rh_status rh_mode_product(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode,
                          int32_t k, const void* A, int32_t transpose, int32_t out_dtype, void* Y, void* stream);

/*
 * rh_mode_product_bf16 -- the first-mode product Y = X x_0 A^T on the tensor cores for a tensor in
 * a BF16 form (RH_BF16 / RH_BF16X2 / RH_F32_BF16X2): A is I_0 x k FP64 (1 <= k <= 64), split exactly into two BF16
 * pieces; Y is k x (N / I_0) FP32 (layout c + k p), all four piece products with FP32
 * accumulation.  Needs I_0 % 8 == 0, or I_0 <= 128 and k <= 32 (the small-row kernel).
 * RH_F32_BF16X3: the FP32 X split exactly into three pieces (I_0 % 8 == 0 only).
 * Workspace: rh_mode_product_workspace_size; its first int32
 * receives the wait status as in rhosvd_sketch (0, or the code of a bounded wait that gave up).
 * RH_FP8_E4M3 (the block-scaled layout of rh_fp8_layout) is read the same way, dequantized and
 * rounded to one BF16 piece.  This is Alg. 1 step 3 (B = Q^T X_(1)) with Q = A, for the input forms
 * whose first mode runs on the tensor cores.  RH_EINVAL: another dtype, bad order or dims, NULL
 * pointers; RH_EUNSUPPORTED: k or a shape that neither kernel takes; RH_ENOMEM: workspace_bytes
 * below the query.
 */
size_t rh_mode_product_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode, int32_t k);
rh_status rh_mode_product_bf16(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t k,
                               const double* A, float* Y, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_mode_product_split -- Y = X x_mode A^T on the tensor cores for an FP32 tensor read as
 * RH_F32_BF16X2 (each value split on the fly into BF16 head and tail, A (I_mode x k FP64, k <= 64)
 * into two pieces, all four piece products with FP32 accumulation): the mode product of Alg. 1
 * step 3 for mode 0 (I_0 % 8 == 0) or for a later mode whose earlier sizes multiply to a multiple of
 * 128 (its unfolding read through the 3-D view (l, i, r)).  Y (FP32) is in the layout of
 * rh_mode_product: dims with dims[mode] replaced by k, column-major.  Workspace:
 * rh_mode_product_split_workspace_size; its first int32 receives the wait status as in
 * rhosvd_sketch.  RH_EUNSUPPORTED for other shapes.
 */
size_t rh_mode_product_split_workspace_size(int32_t order, const int64_t* dims, int32_t mode, int32_t k);
rh_status rh_mode_product_split(int32_t order, const int64_t* dims, const float* X, int32_t mode, int32_t k,
                                const double* A, float* Y, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_left_svd -- left singular vectors and singular values of the mode-n unfolding B_(n) of a tensor
 * whose mode n is short (I_mode <= RH_MAX_ELL): the thin SVD of Alg. 1 step 4 applied to
 * B = Q^T X.  B_(n)^T is triangularised by a tree of Householder QRs (no Gram matrix); the
 * I_mode x I_mode triangle R gets a column-pivoted QR, R P = Q_2 R_2 (Drmac-Veselic
 * preconditioning), and R_2^T is diagonalised by one-sided Jacobi, all in B's precision.
 *   U   I_mode x I_mode FP64, column-major, columns ordered by decreasing singular value
 *       (column signs arbitrary);  sv  I_mode FP64 singular values, decreasing.
 */
size_t rh_left_svd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode);
rh_status rh_left_svd(int32_t order, const int64_t* dims, int32_t dtype, const void* B, int32_t mode,
                      double* U, double* sv, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rsthosvd -- R-STHOSVD (Alg. 3) with RandSVD (Alg. 1) on each current core unfolding.
 *   X        input tensor (order, dims, dtype), column-major device buffer.
 *   ranks    target ranks r_n (host array of ``order`` values, 1 <= r_n).
 *   opts     options (NULL = rh_options_default).
 *   factors  host array of ``order`` device pointers; factors[n] receives A_n, I_n x k_n FP64
 *            column-major with orthonormal columns, where k_n = r_n (truncate = 1) or
 *            ell_n (truncate = 0).
 *   core     device buffer receiving G, k_1 x ... x k_d FP64 column-major.
 *   norms    optional device buffer of 2 FP64 values: ||X||_F^2 and ||G||_F^2.  For the
 *            orthonormal factors of Alg. 3, ||X - X_hat||^2 = ||X||^2 - ||G||^2 exactly
 *            (Thm. lem:st_mode_err); the difference is meaningful only above ~1e-6 relative.
 *   info     optional device int32 array of ``order`` values, bit flags per mode n:
 *            1 = the QR of the sketch took the Householder branch; 2 = the truncation
 *            SVD went through the Gram matrix (FP32 data only, see below); 4 = the sketch and
 *            mode product of mode n ran on the tensor cores (BF16 forms); 8 = the truncation
 *            SVD went through the double-float Gram matrix; 16 = a tensor-core kernel of mode n
 *            gave up a bounded wait (a TMA or MMA completion that never arrived): the outputs
 *            of that mode and of every later step are invalid.  The call stays asynchronous;
 *            read info after the stream has synchronised.
 *   Size rule: ell_n <= min(I_n, prod of the other current sizes), else RH_EINVAL (or
 *   clamped, opts->clamp).  Steps per mode n (in order rho):
 *     sketch Y = G_(n) Omega_n; Q = orth(Y); B = Q^T G_(n) (mode-n product);
 *     R with B B^T = R^T R: FP32 data first form W = B B^T (FP64 sums of FP32 partial
 *     sums) and its pivoted Cholesky factor, kept when that succeeds and sigma_r^2 -
 *     sigma_{r+1}^2 >= 1e-5 sigma_1^2; otherwise W again with every product exact and the
 *     sums in double-float (~2^-44 relative), kept when its Cholesky succeeds; otherwise (and
 *     for FP64 data) B^T = Q_B R by a tall-skinny Householder QR, R P = Q_2 R_2 by a
 *     column-pivoted QR and one-sided Jacobi on R_2^T.  In every branch the one-sided
 *     Jacobi SVD of the final factor gives U_B;
 *     A_n = Q U_B(:, 1:r_n); G <- U_B(:, 1:r_n)^T B.
 */
size_t rsthosvd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                               const rh_options* opts);
rh_status rsthosvd(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const int32_t* ranks,
                   const rh_options* opts, double* const* factors, double* core, double* norms,
                   int32_t* info, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rsthosvd_batched -- R-STHOSVD (Alg. 3) applied independently to each of ``count`` tensors of
 * different orders and sizes in one call (each tensor is decomposed exactly as by rsthosvd).
 *   orders   host array of ``count`` tensor orders (1 .. 8).
 *   dims     host array of sum(orders) sizes, tensor i's sizes after those of tensors 0 .. i-1.
 *   ranks    host array laid out like dims.
 *   X        host array of ``count`` device pointers (all tensors of one dtype, column-major).
 *   factors  host array of sum(orders) device pointers, laid out like dims (FP64 as in rsthosvd).
 *   cores    host array of ``count`` device pointers (FP64 cores as in rsthosvd).
 *   norms    optional device buffer of 2 * count FP64 values (tensor i at 2 i); info optional
 *            device int32 array laid out like dims.
 *   opts     shared by every tensor; tensor i draws Omega with tensor_id = opts->tensor_id + i.
 *            opts->rho is the default order (rho[0] < 0) or one whose first order_i entries are a
 *            permutation of 0 .. order_i - 1 for every tensor i (tensor i takes those entries).
 *   streams  0 = the grouped engine when every request is FP32 or FP64 data with truncation
 *            (opts->truncate), or a BF16 form whose first mode
 *            runs on the small-row tensor-core kernels (see the element types above): each
 *            tensor's launch sequence is recorded on the host and the same
 *            stage of all tensors runs as one launch (about 30 launches per mode for the whole
 *            batch; the per-tensor argument tables are copied into the workspace by stream-ordered
 *            kernels that carry them in their parameters).  Otherwise, and for streams >= 1, that
 *            many internal streams (0 = min(8, count), at most 32): the caller's stream is forked
 *            into them with an event, tensors are placed largest first (by element count) on the
 *            least-loaded stream, and every stream is joined back into ``stream`` before the call
 *            returns.  Either way no host synchronisation, so the call is CUDA-graph capturable.
 *   workspace  grouped engine: one slice per tensor (its rsthosvd_workspace_size rounded to 256 B)
 *            and the launch tables; streams: one slice per internal stream, each the largest
 *            rsthosvd_workspace_size of the batch.  rsthosvd_batched_workspace_size returns the
 *            total for the engine that ``streams`` selects (0 on an invalid request).  Neither
 *            engine's result depends on timing: each tensor's result equals, bit for bit, that of a
 *            single rsthosvd call.
 *   Errors: RH_EINVAL names the first invalid tensor; on the stream engine a failing tensor stops
 *   the enqueueing of later tensors (earlier ones still run); the grouped engine validates every
 *   tensor before it launches anything.
 */
size_t rsthosvd_batched_workspace_size(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                                       const int32_t* ranks, const rh_options* opts, int32_t streams);
rh_status rsthosvd_batched(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                           const void* const* X, const int32_t* ranks, const rh_options* opts,
                           double* const* factors, double* const* cores, double* norms, int32_t* info,
                           int32_t streams, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Batched plan -- the grouped engine of rsthosvd_batched for a fixed set of requests, buffers and
 * workspace, recorded once and run many times.  create takes the arguments of rsthosvd_batched
 * (workspace of rsthosvd_batched_workspace_size(..., streams = 0) bytes, of which the plan uses the
 * per-tensor slices), records every tensor's program, and copies the launch tables into device
 * memory the plan owns (one synchronous copy).  run enqueues the grouped launches on ``stream``
 * (no host synchronisation; capturable); every run recomputes all outputs from the current
 * contents of X.  The buffers named at create must stay valid while the plan is used.  destroy
 * frees the tables (it synchronises the device through cudaFree).  RH_EUNSUPPORTED when a request
 * cannot run on the grouped engine.  The engine takes truncated requests (truncate = 1) of FP32 or
 * FP64 data, and of the BF16 forms whose first mode is processed first and takes the small-row
 * tensor-core kernels (I_0 <= 128, ell <= 32).
 */
typedef struct rh_batched_plan_s* rh_batched_plan;
rh_status rsthosvd_batched_plan_create(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                                      const void* const* X, const int32_t* ranks, const rh_options* opts,
                                      double* const* factors, double* const* cores, double* norms, int32_t* info,
                                      void* workspace, size_t workspace_bytes, rh_batched_plan* plan);
rh_status rsthosvd_batched_plan_run(rh_batched_plan plan, void* stream);
/* number of grouped launches one run enqueues (-1 for a NULL plan) */
int64_t rsthosvd_batched_plan_launches(rh_batched_plan plan);
void rsthosvd_batched_plan_destroy(rh_batched_plan plan);

/*
 * rhosvd -- R-HOSVD (Alg. 2): RandSVD (Alg. 1) of every unfolding X_(n) of the input with its own
 * Omega_n, then the core G = X x_1 A_1^T ... x_d A_d^T (Alg. 2 step 6).  Arguments, outputs,
 * options (rho is ignored: the modes are independent), size rule (on the input sizes, Alg. 2
 * REQUIRE) and errors as rsthosvd; norms[1] = ||G||^2 (for R-HOSVD ||X - X_hat||^2 <= ||X||^2 -
 * ||G||^2 only holds as an inequality; use rh_tucker_residual for the error).
 */
size_t rhosvd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                             const rh_options* opts);
rh_status rhosvd(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const int32_t* ranks,
                 const rh_options* opts, double* const* factors, double* core, double* norms, int32_t* info,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * core_ttm -- G = X x_1 A_1^T x_2 A_2^T ... x_d A_d^T (Alg. 2 step 6; Sec. 2.2, HOSVD core).
 *   factors  host array of ``order`` device pointers, A_n of size I_n x ks[n], FP64 column-major
 *            (cast to X's precision for the products).
 *   G        device output, ks[0] x ... x ks[order-1], FP64 column-major.
 *   The modes are applied in the order that shrinks the intermediate tensor most first.
 */
size_t core_ttm_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ks);
rh_status core_ttm(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const double* const* factors,
                   const int32_t* ks, double* G, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_orthonormalize_tucker -- the orthonormalising post-processing of Sec. 5 for the interpolatory
 * (non-orthonormal) factors of Alg. 6 and SP-HOSVD: for each mode n, the thin QR A_n = Q_n R_n
 * (Alg. 1 step 2's QR: CholeskyQR2 with the Householder fallback, each column's largest-magnitude
 * entry positive) and the aggregation G <- G x_n R_n.  G x_1 A_1 ... x_d A_d is unchanged (up to
 * rounding) and every factor becomes orthonormal, so ||G||_F = ||G x_1 A_1 ... x_d A_d||_F.
 *   dims, ks   A_n is I_n x k_n (1 <= k_n <= min(I_n, 64)); the core is k_1 x ... x k_d.
 *   factors    host array of device pointers to the FP64 column-major A_n: overwritten by Q_n.
 *   core       device FP64 column-major core: overwritten by the new core.
 *   Asynchronous; workspace: rh_orthonormalize_tucker_workspace_size.
 */
size_t rh_orthonormalize_tucker_workspace_size(int32_t order, const int64_t* dims, const int32_t* ks);
rh_status rh_orthonormalize_tucker(int32_t order, const int64_t* dims, const int32_t* ks, double* const* factors,
                                   double* core, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_tucker_residual -- direct error of a Tucker approximation (validation of Thm. lem:st_mode_err
 * and of the bounds of Sec. 3.2 without the cancellation of ||X||^2 - ||G||^2).
 *   out[0] = ||X - G x_1 A_1 ... x_d A_d||_F^2,  out[1] = ||X||_F^2  (device, FP64).
 *   factors: A_n, I_n x ks[n] FP64; core: ks[0] x ... FP64.  The reconstruction is computed in X's
 *   precision, expanding all modes but one and fusing the last expansion with the comparison, so
 *   X_hat is never stored; the squared differences are summed in FP64.
 */
size_t rh_tucker_residual_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ks);
rh_status rh_tucker_residual(int32_t order, const int64_t* dims, int32_t dtype, const void* X,
                             const double* const* factors, const int32_t* ks, const double* core, double* out,
                             void* workspace, size_t workspace_bytes, void* stream);

/*
 * adaptive_rank -- adaptive-rank randomized HOSVD (variant 0, Alg. 4) or STHOSVD (variant 1,
 * Alg. 5) to a target relative error: every mode's factor comes from the adaptive range finder
 * of Sec. 4 with the absolute tolerance tau = eps ||X||_F / sqrt(d).  Reading of the range finder
 * (the paper names it without listing it): blocks of ``block`` columns of the mode's Gaussian
 * stream are added until ||G_(n) - Q Q^T G_(n)||_F <= tau or max_ranks[n] columns are reached, then
 * opts->p more columns of the same stream; the SVD of B = Q^T G_(n) is trimmed to the smallest r
 * with sum_{i>r} sigma_i^2 + ||G_(n) - Q B||^2 <= tau^2.  One sketch of width max_ranks[n] + p
 * serves every block size (the leading columns of its thin QR span the leading blocks).
 *   X          tensor (order, dims, dtype), column-major, device.  RH_F64 and RH_F32 with either
 *              variant; the BF16 and E4M3 forms (RH_BF16, RH_BF16X2, RH_F32_BF16X2, RH_FP8_E4M3)
 *              with variant 1 only (RH_EUNSUPPORTED otherwise).  Their first mode runs on the tensor
 *              cores, which needs mode 0 processed first, I_0 % 8 == 0, I_0 <= 1024 and
 *              max_ranks[0] + p <= 64; otherwise RH_F32_BF16X2 runs as RH_F32 and the other forms
 *              return RH_EUNSUPPORTED.  RH_F32_BF16X3 is not taken (RH_EINVAL).
 *   max_ranks  host array: cap on the range-finder size per mode (max_ranks[n] + p <= 64 after
 *              clamping to min(I_n, prod of the other sizes)).
 *   opts       p (trim oversampling), seed, tensor_id, rho (variant 1; rho[0] < 0: decreasing
 *              I_n).  truncate and clamp are ignored.
 *   factors    host array of device pointers, factors[n] holds I_n x ell_n FP64 with
 *              ell_n = min(max_ranks[n] + p, I_n, prod of the other input sizes) (the trim runs over
 *              up to ell_n rows, so ranks[n] can exceed max_ranks[n]); the first ranks[n] columns
 *              receive A_n (orthonormal, column signs as in rsthosvd).
 *   core       device buffer of prod(ell_n) FP64; receives the ranks[0] x ... core, column-major.
 *   ranks      HOST array of ``order`` values receiving the chosen ranks.
 *   norms      optional device buffer of 2 FP64: ||X||^2 and ||G||^2.
 *   Synchronous: the chosen sizes drive the later launches, so the call synchronises ``stream``
 *   once per mode and returns when the result is complete.  Workspace:
 *   adaptive_rank_workspace_size.
 */
size_t adaptive_rank_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t variant,
                                    const int32_t* max_ranks, const rh_options* opts);
rh_status adaptive_rank(int32_t order, const int64_t* dims, int32_t dtype, const void* X, double eps,
                        int32_t variant, int32_t block, const int32_t* max_ranks, const rh_options* opts,
                        double* const* factors, double* core, int32_t* ranks, double* norms, void* workspace,
                        size_t workspace_bytes, void* stream);

/*
 * rhosvd_sketch_coo -- the range-finder sketch Y = X_(mode) Omega_mode of a sparse tensor given as
 * COO entries, without densifying (Alg. 6 step 4; Sec. 5).  Entry k is (idx[0][k], ..., idx[d-1][k])
 * with value vals[k]; it adds vals[k] Omega_mode(p, :) to row idx[mode][k] of Y, p the Kolda
 * column index of the entry in the mode-``mode`` unfolding (the Omega stream of rhosvd_sketch).
 *   idx   host array of ``order`` DEVICE pointers to int32 arrays of nnz 0-based indices
 *         (deduplicated; duplicates are summed).  vals: device FP32 array of nnz values.
 *   omega_prec  RH_F32 (RH_F64: the same FP32 normals) or RH_BF16: every normal rounded to BF16
 *         (ties to even) before the products (the BF16-Omega form); FP32 products and sums either way.
 *   Y     device, I_mode x ell FP64, column-major.
 *   The entries are stably sorted by their mode index and each row's sum is formed in a fixed
 *   order (FP32 sums over at most 512 entries, FP64 above): the result is deterministic.  The call
 *   synchronises ``stream`` once (the work split is built on the host from the row counts).
 *   Omega rows are shared between the entries with the same other-mode coordinates: when the
 *   unfolding has fewer than 2^31 columns each distinct row is generated once into a table in the
 *   workspace (up to nnz rows of ell rounded up to 4 entries, 4 bytes each) and read from there;
 *   the normals, and so the sums, are the same as generating them per entry.
 *   Needs nnz < 2^31 and every I_n < 2^31; ell <= 64.  Workspace: rhosvd_sketch_coo_workspace_size.
 *   Indices of mode ``mode`` outside [0, I_mode) are counted on the device and the call returns
 *   RH_EINVAL after its synchronisation (Y undefined); they are never used as addresses.  Indices of
 *   the other modes only select rows of Omega and are not checked.
 */
size_t rhosvd_sketch_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, int32_t mode, int32_t ell);
rh_status rhosvd_sketch_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                            const float* vals, int32_t mode, int32_t ell, uint64_t seed, int32_t tensor_id,
                            int32_t omega_prec, double* Y, void* workspace, size_t workspace_bytes, void* stream);

/*
 * sp_sthosvd_coo -- structure-preserving STHOSVD of a COO tensor (Alg. 6).  Per mode n in the order
 * rho: Y = G_(n) Omega_n from the nonzeros (opts->omega_prec: FP32 or BF16 Omega); Y = QR; P_n = ell_n
 * rows of Q chosen by opts->select: by default strong RRQR with eta = 2 (column-pivoted QR of Q^T,
 * then swaps while some |A_ij| > 2 on an unselected row, largest first, lowest (i, j) on ties), or
 * another selection of Sec. 5 (rh_subset_select); A_n = Q (P_n^T Q)^{-1}; G_(n) <- P_n^T G_(n), i.e. the
 * nonzeros whose mode-n index is selected, renumbered to their position in the sorted selection.
 * The core is the dense ell_1 x ... x ell_d array of the surviving entries (entries of X).
 *   ell_n = ranks[n] + opts->p must be < min(I_n, prod of the other current sizes) (Alg. 6's strict
 *   rule; opts->clamp lowers ell_n to that bound minus one instead of failing) and <= 64.
 *   idx, vals   as rhosvd_sketch_coo (not modified; the call works on a copy).
 *   factors     host array of device pointers, factors[n] receives A_n, I_n x ell_n FP64.
 *   selected    optional host array of device pointers, selected[n] receives P_n (ell_n int32,
 *               increasing); NULL or NULL entries skip it.
 *   core        device, prod(ell_n) FP64, column-major.  norms: optional device 2 FP64:
 *               ||X||^2 and ||G||^2.
 *   The selection runs on the host in FP64; the call synchronises ``stream`` several times per
 *   mode and returns when the result is complete.  Workspace: sp_sthosvd_coo_workspace_size.
 *   An index outside [0, I_n) is detected when mode n's nonzeros are counted (before any kernel
 *   addresses memory with it) and the call returns RH_EINVAL; the outputs are then undefined.
 */
size_t sp_sthosvd_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* ranks,
                                     const rh_options* opts);
rh_status sp_sthosvd_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx,
                         const float* vals, const int32_t* ranks, const rh_options* opts, double* const* factors,
                         int32_t* const* selected, double* core, double* norms, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * sp_hosvd_coo -- structure-preserving HOSVD of a COO tensor (Sec. 5, the first remark after Alg. 6:
 * the modes of Alg. 6 handled independently).  For every mode n of the INPUT: Y = X_(n) Omega_n from
 * the nonzeros (Omega_n the stream of R-HOSVD's mode n; opts->omega_prec), Y = QR, P_n by
 * opts->select, A_n = Q (P_n^T Q)^{-1}; the core is X at the selected coordinates, X(P_1, ..., P_d):
 * the nonzeros whose every index is selected, each index renumbered to its position in the sorted
 * selection, scattered into the dense ell_1 x ... x ell_d array.  Arguments, outputs and errors as
 * sp_sthosvd_coo, with Alg. 6's strict size rule ell_n < min(I_n, prod of the other INPUT sizes) and
 * the modes taken in increasing order (opts->rho is ignored).  Synchronous (host selection per mode).
 */
size_t sp_hosvd_coo_workspace_size(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* ranks,
                                   const rh_options* opts);
rh_status sp_hosvd_coo(int32_t order, const int64_t* dims, int64_t nnz, const int32_t* const* idx, const float* vals,
                       const int32_t* ranks, const rh_options* opts, double* const* factors, int32_t* const* selected,
                       double* core, double* norms, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rh_subset_select -- the row selection and interpolatory factor of Alg. 6 steps 6-7 on one basis:
 * the host step that sp_sthosvd_coo runs for each mode (with RH_SELECT_SRRQR, eta = 2), and the
 * other selections of Sec. 5's remark on subset selection (column-pivoted QR, DEIM, uniform and
 * leverage-score sampling).  Host memory only; no device call.
 *   Q         host, I x ell FP64 column-major (full column rank; sp_sthosvd_coo passes the thin-QR
 *             factor of the sketch).  Not modified.
 *   method    RH_SELECT_SRRQR: column-pivoted Householder QR of Q^T (largest remaining column norm,
 *               lowest index on ties), then, while some unselected |A_ij| > eta, row i replaces
 *               selected row j for the largest |A_ij| (lowest (i, j) on ties; at most 100000
 *               swaps), so |A_ij| <= eta on every unselected row;
 *             RH_SELECT_CPQR: the pivots of that column-pivoted QR alone (no bound on A);
 *             RH_SELECT_DEIM: the DEIM greedy (Chaturantabut-Sorensen; Sorensen-Embree): the largest
 *               |Q(i, 0)|, then for j = 1 .. ell-1 the largest |r_i| of r = Q(:, j) - Q(:, 0:j) c with
 *               Q(P, 0:j) c = Q(P, j) (lowest index on ties);
 *             RH_SELECT_UNIFORM / RH_SELECT_LEVERAGE: ell rows sampled without replacement with
 *               weights 1 or ||Q(i, :)||^2 (the leverage scores of range(Q)): draw k takes the first
 *               untaken row (increasing i) whose running weight sum exceeds u_k times the untaken
 *               total (FP64 sums), u_k = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 from the Philox4x32-10
 *               words of counter (k, stream, 0, 0x53454C45) under key (seed lo, seed hi).
 *   eta       strong-RRQR bound, >= 1 (RH_SELECT_SRRQR only).
 *   seed, stream  key and counter word of the sampling methods (ignored by the others).
 *   selected  host, ell int32 receiving P, the chosen rows of Q, increasing.
 *   A         host, I x ell FP64 column-major receiving A = Q (P^T Q)^{-1}, with the rows P stored as
 *             the exact identity.
 *   RH_EINVAL: ell < 1, ell > I, unknown method, eta < 1 with RH_SELECT_SRRQR, NULL pointers.
 *   RH_ENUMERIC: P^T Q singular, a vanishing DEIM residual, no sampling weight left, or non-finite
 *   values in Q.
 */
enum { RH_SELECT_SRRQR = 0, RH_SELECT_CPQR = 1, RH_SELECT_DEIM = 2, RH_SELECT_UNIFORM = 3, RH_SELECT_LEVERAGE = 4 };
rh_status rh_subset_select(int64_t I, int32_t ell, const double* Q, int32_t method, double eta, uint64_t seed,
                           uint32_t stream, int32_t* selected, double* A);

/*
 * rsthosvd_host -- the same R-STHOSVD with HOST buffers: enqueues the copy of X to the
 * device, the decomposition and the copies of the factors, the core and the norms back
 * to the host, all on ``stream``; the results are valid once the stream is synchronised.
 *   X_host       host tensor (pinned memory gives asynchronous copies), column-major.
 *   factors_host host array of ``order`` host pointers, I_n x k_n FP64 each.
 *   core_host    host buffer, k_1 x ... x k_d FP64;  norms_host optional, 2 FP64.
 *   info_host    optional host array of ``order`` int32 receiving the per-mode flags of rsthosvd
 *                (``info``), copied back with the results; bit 16 marks a mode whose tensor-core
 *                kernel gave up a bounded wait, so that mode's outputs and every later step's
 *                are invalid.  Read it after the stream has synchronised.
 *   workspace    DEVICE buffer of rsthosvd_host_workspace_size bytes; it holds the device
 *                copy of X, the device outputs and the rsthosvd workspace.
 *   The decomposition is Alg. 3 exactly as rsthosvd computes it (bit-identical results); the
 *   host copies are the end-to-end leg of the measurement, not part of the paper's method.
 *   Errors as rsthosvd (RH_EINVAL before anything is enqueued, RH_ENOMEM for a short workspace).
 */
size_t rsthosvd_host_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                                    const rh_options* opts);
rh_status rsthosvd_host(int32_t order, const int64_t* dims, int32_t dtype, const void* X_host,
                        const int32_t* ranks, const rh_options* opts, double* const* factors_host,
                        double* core_host, double* norms_host, int32_t* info_host, void* workspace,
                        size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RHOSVD_H */
