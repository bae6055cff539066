// Host drivers of the C ABI: rhosvd_sketch, rh_orthonormalize and rsthosvd (Alg. 3 with
// RandSVD, Alg. 1, on each current core unfolding).  Host code only sequences kernels
// on the caller's stream; every arithmetic step runs on the device.
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rh {
namespace {

bool dtype_ok(int32_t dtype) { return dtype == RH_F64 || dtype == RH_F32; }
// The Gram matrix of B rides with the tensor-core mode product from this many rows of the unfolding
// on (8 K stages of 64 rows per tile): with fewer, the epilogue's Gram work is no longer hidden
// behind the tile's MMAs (192^4: the first mode product +0.95 ms against 0.69 ms for a separate
// Gram pass).
constexpr int64_t kGramFuseMinRows = 512;
// forms whose first mode runs on the tensor cores over BF16 pieces
// input forms whose first mode runs on the tensor cores over BF16 pieces
bool bf16_form(int32_t dtype) {
  return dtype == RH_BF16 || dtype == RH_BF16X2 || dtype == RH_F32_BF16X2 || dtype == RH_FP8_E4M3;
}
// FP32 or E4M3 input converted to BF16 pieces inside the tensor-core kernels
bool converted_form(int32_t dtype) { return dtype == RH_F32_BF16X2 || dtype == RH_FP8_E4M3; }

// bytes of an input tensor buffer in the given form
size_t input_bytes(int32_t order, const int64_t* dims, int32_t dtype) {
  if (dtype == RH_FP8_E4M3) return fp8_layout(order, dims).bytes;
  size_t n = 1;
  for (int k = 0; k < order; ++k) n *= (size_t)dims[k];
  return n * (dtype == RH_F64 ? 8 : (dtype == RH_BF16 ? 2 : 4));
}

rh_status check_tensor(int32_t order, const int64_t* dims, int32_t dtype) {
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER, "order must be in [1, 8]");
  RH_CHECK_ARG(dims != nullptr, "dims is NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(dims[k] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(dtype_ok(dtype), "dtype must be RH_F64 or RH_F32");
  return RH_OK;
}

// ---- sketch -----------------------------------------------------------------------
struct SketchBufs {
  void* part;
  double* part_norm;
};

SketchBufs carve_sketch(Arena& ar, const SketchPlan& pl, int32_t dtype) {
  SketchBufs b;
  b.part = (dtype == RH_F64) ? (void*)ar.take<double>(pl.part_elems()) : (void*)ar.take<float>(pl.part_elems());
  b.part_norm = ar.take<double>(pl.norm_elems());
  return b;
}

template <typename T>
rh_status run_sketch(const SketchPlan& pl, const T* G, uint64_t seed, uint32_t sid, const SketchBufs& b, double* Y,
                     double* norm2, cudaStream_t st, int accumulate = 0) {
  rh_status s = launch_sketch<T>(pl, G, seed, sid, static_cast<T*>(b.part), b.part_norm, st);
  if (s != RH_OK) return s;
  return launch_sketch_reduce<T>(pl, static_cast<const T*>(b.part), b.part_norm, Y, norm2, st, SITE_SKETCH_REDUCE,
                                 accumulate);
}

// ---- R-STHOSVD plan ------------------------------------------------------------------
struct Step {
  int mode;
  ModeView v;   // view of the current core for this mode
  int ell;      // sketch width r + p (possibly clamped)
  int ko;       // output width of the mode: r (truncate) or ell
  SketchPlan sk;
  SketchPlan skd;       // sketch against a dense operand (subspace-iteration steps)
  TruncPlan tr;
  bool tc = false;      // sketch and mode product on the tensor cores (FP32 core split on the fly)
  bool cp = false;      // truncated core by the core product (B has the new mode fastest) in the order cout
  CoreOut cout;
  bool cp_tc = false;   // that core product on the tensor cores (B and U_r split into BF16 pieces)
  bool stc = false;     // first mode with few rows: sketch and mode product on the small-row
                        // tensor-core kernels (grouped operations), later modes FP32 on the CUDA cores
};

struct Plan {
  int d;
  int32_t dtype;
  std::vector<Step> steps;
  size_t max_I_ell = 0, max_tensor = 0, max_orth = 0, max_trunc = 0, max_part = 0, max_pnorm = 0;
  size_t fac_elems = 0;   // R-HOSVD: factor copies in the tensor's precision for the core chain
  int32_t in_form = -1;   // a bf16_form input (first mode on the tensor cores when possible), else -1
  size_t tc_part = 0, qa_elems = 0;
  std::vector<int64_t> dims0;   // the input sizes
  int power = 0;                // subspace-iteration steps per range finder
  int pieces = 2;               // BF16 pieces of the on-the-fly split (3: RH_F32_BF16X3, exact)
};

// Subspace iteration (opts.power_iters): the dense-operand sketch plan of every step and the
// workspace of its basis step.
rh_status plan_power(const rh_options& o, Plan& pl) {
  RH_CHECK_ARG(o.power_iters >= 0 && o.power_iters <= 8, "power_iters must be in [0, 8]");
  pl.power = o.power_iters;
  if (!pl.power) return RH_OK;
  if ((pl.in_form >= 0 && pl.in_form != RH_F32_BF16X2) || pl.pieces != 2) {
    set_error("unsupported: subspace iteration needs FP64, FP32 or RH_F32_BF16X2 input (its sketch reads G_(n) "
              "on the CUDA cores)");
    return RH_EUNSUPPORTED;
  }
  for (Step& st : pl.steps) {
    st.skd = plan_sketch_dense(st.v, st.ell);
    pl.max_part = std::max(pl.max_part, st.skd.part_elems());
    pl.max_trunc = std::max(pl.max_trunc, pl.dtype == RH_F64 ? power_workspace_elems<double>(st.tr)
                                                               : power_workspace_elems<float>(st.tr));
  }
  return RH_OK;
}

rh_status make_plan(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks, const rh_options& o,
                    Plan& pl) {
  // RH_F32_BF16X3 is the split form with three exact pieces in every tensor-core kernel
  pl.pieces = dtype == RH_F32_BF16X3 ? 3 : 2;
  if (dtype == RH_F32_BF16X3) dtype = RH_F32_BF16X2;
  rh_status s = check_tensor(order, dims, bf16_form(dtype) ? RH_F32 : dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(ranks != nullptr, "ranks is NULL");
  RH_CHECK_ARG(o.p >= 0, "oversampling p must be >= 0");
  RH_CHECK_ARG(o.tensor_id >= 0 && o.tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(o.svd_route == 0 || o.svd_route == 1, "svd_route must be 0 or 1");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(ranks[k] >= 1, "every rank must be >= 1");
  std::vector<int> rho(order);
  if (o.rho[0] < 0) {
    std::iota(rho.begin(), rho.end(), 0);
    std::stable_sort(rho.begin(), rho.end(), [&](int a, int b) { return dims[a] > dims[b]; });
  } else {
    std::vector<int> seen(order, 0);
    for (int k = 0; k < order; ++k) {
      RH_CHECK_ARG(o.rho[k] >= 0 && o.rho[k] < order && !seen[o.rho[k]], "rho must be a permutation of 0..order-1");
      seen[o.rho[k]] = 1;
      rho[k] = o.rho[k];
    }
  }
  pl.d = order;
  pl.dtype = dtype;
  pl.dims0.assign(dims, dims + order);
  std::vector<int64_t> cur(dims, dims + order);
  const size_t tsz = (dtype == RH_F64) ? sizeof(double) : sizeof(float);
  for (int j = 0; j < order; ++j) {
    Step st;
    st.mode = rho[j];
    st.v = mode_view(order, cur.data(), st.mode);
    const int64_t lim = std::min<int64_t>(st.v.I, st.v.M());
    int64_t ell = (int64_t)ranks[st.mode] + o.p;
    if (ell > lim) {
      if (!o.clamp) {
        set_error("invalid argument: r_n + p = " + std::to_string(ell) + " exceeds min(I_n, prod of the other sizes) = " +
                  std::to_string(lim) + " for mode " + std::to_string(st.mode));
        return RH_EINVAL;
      }
      ell = lim;
    }
    if (ell > RH_MAX_ELL) {
      set_error("unsupported: r_n + p = " + std::to_string(ell) + " exceeds RH_MAX_ELL (64)");
      return RH_EUNSUPPORTED;
    }
    st.ell = (int)ell;
    st.ko = o.truncate ? std::min<int>(ranks[st.mode], st.ell) : st.ell;
    st.sk = plan_sketch(st.v, st.ell);
    st.tr = plan_trunc(ModeView{st.v.L, st.ell, st.v.R}, st.ell);
    pl.max_I_ell = std::max(pl.max_I_ell, (size_t)(st.v.I * st.ell));
    pl.max_tensor = std::max(pl.max_tensor, (size_t)(st.v.M() * st.ell));   // B
    pl.max_part = std::max(pl.max_part, st.sk.part_elems());
    pl.max_pnorm = std::max(pl.max_pnorm, st.sk.norm_elems());
    pl.max_orth = std::max(pl.max_orth, orth_workspace_elems(st.v.I, st.ell));
    pl.max_trunc = std::max(pl.max_trunc, dtype == RH_F64 ? trunc_workspace_elems<double>(st.tr)
                                                           : trunc_workspace_elems<float>(st.tr));
    cur[st.mode] = st.ko;
    pl.steps.push_back(st);
  }
  (void)tsz;
  if (bf16_form(dtype)) {
    // The first processed mode runs on the tensor cores over the BF16 pieces.  FP32 input split
    // on the fly can also take the FP32 CUDA-core path for a first mode the tensor-core kernels
    // do not cover (later modes still go to the tensor cores where their shape allows).
    const Step& s0 = pl.steps[0];
    if (o.power_iters == 0 && pl.pieces == 2 && small_tc_supported(s0.v, s0.ell)) {
      // A first mode with few rows (mode 0, I_0 <= 128, ell <= 32): the small-row tensor-core
      // sketch and mode product, written as grouped operations; the later modes run in FP32 on
      // the CUDA cores on the FP32 core the first mode leaves.
      Step& f = pl.steps[0];
      f.stc = true;
      f.sk = plan_sketch_small_tc(f.v, f.ell);
      pl.max_part = std::max(pl.max_part, f.sk.part_elems());
      pl.max_pnorm = std::max(pl.max_pnorm, f.sk.norm_elems());
      pl.dtype = RH_F32;
      pl.in_form = dtype;
      return plan_power(o, pl);
    }
    const bool s0_tc = s0.mode == 0 && sketch_tc_supported(s0.v, s0.ell) && ttm_tc_supported(s0.v, s0.ell);
    if (!s0_tc && dtype != RH_F32_BF16X2) {
      set_error("unsupported: the BF16 and E4M3 forms need mode 0 processed first, I_0 % 8 == 0, I_0 <= 1024, "
                "r + p <= 64");
      return RH_EUNSUPPORTED;
    }
    pl.steps[0].tc = s0_tc;
    pl.max_pnorm = std::max<size_t>(pl.max_pnorm, 1024);   // partials of the norm over the BF16 pieces
    pl.dtype = RH_F32;        // intermediates
    pl.in_form = dtype;
    if (o.truncate) {
      // Later modes: the core product of a step whose B has its new mode fastest (unit-stride
      // view) writes the next core with the next mode m first and the other modes in increasing
      // order (CoreOut), so the next unfolding keeps its Kolda column order (Omega's rows line up)
      // and is read with unit stride; it runs on the tensor cores when its shape allows.  The
      // final core is written in the usual column-major order.
      std::vector<int64_t> sz(dims, dims + order);   // sizes of the current core
      for (int j = 0; j < order; ++j) {
        Step& sp = pl.steps[j];
        const int n = sp.mode;
        std::vector<int64_t> after = sz;
        after[n] = sp.ko;
        if (sp.v.L == 1) {
          sp.cp = true;
          if (j == order - 1) {
            int64_t ln = 1;
            for (int k = 0; k < n; ++k) ln *= after[k];
            sp.cout = CoreOut::make(1, 1, ln, sp.v.M());
          } else {
            Step& nx = pl.steps[j + 1];
            const int m = nx.mode;
            int64_t S = 1, Ln = 1, Mn = 1;
            for (int k = 0; k < order; ++k) {
              if (k != n && k < m) S *= sz[k];          // stride of mode m in the columns of G_(n)
              if (k < n && k != m) Ln *= after[k];      // modes before n in the new order
              if (k != m) Mn *= after[k];
            }
            sp.cout = CoreOut::make(S, sz[m], Ln, sp.v.M());
            nx.v = ModeView{1, sz[m], Mn};
            nx.sk = plan_sketch(nx.v, nx.ell);
            nx.tr = plan_trunc(ModeView{1, nx.ell, Mn}, nx.ell);
            nx.tc = sketch_tc_supported(nx.v, nx.ell) && ttm_tc_supported(nx.v, nx.ell);
            pl.max_part = std::max(pl.max_part, nx.sk.part_elems());
            pl.max_pnorm = std::max(pl.max_pnorm, nx.sk.norm_elems());
            pl.max_trunc = std::max(pl.max_trunc, trunc_workspace_elems<float>(nx.tr));
          }
        }
        sz = after;
      }
    }
    for (size_t j = 0; j < pl.steps.size(); ++j) {
      Step& sp = pl.steps[j];
      // the truncated core of a non-final mode on the tensor cores (the final core is FP64)
      if (sp.cp && j + 1 < pl.steps.size() && core_product_tc_supported(sp.ell, sp.ko, sp.v.M())) {
        sp.cp_tc = true;
        pl.qa_elems = std::max(pl.qa_elems, (size_t)128 * ((sp.ell + 7) / 8 * 8));
      }
      if (!sp.tc) continue;
      pl.tc_part = std::max(pl.tc_part, (size_t)sketch_tc_ctas(sp.v) * sp.ell * sp.v.I);
      pl.qa_elems = std::max(pl.qa_elems, (size_t)128 * sp.v.I);
    }
  }
  return plan_power(o, pl);
}

// Alg. 2: every mode is sketched on the input tensor itself (no current core).  RH_F32_BF16X2: every
// mode whose shape the tensor-core kernels cover (mode 0 with I_0 % 8 == 0, I_0 <= 1024; a mode with
// L % 128 == 0 and I_n <= 1024) runs its sketch and mode product there, the FP32 input split on the
// fly; the others, and the core chain's products that the tensor-core mode product does not cover,
// in FP32 on the CUDA cores.
rh_status make_plan_hosvd(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                          const rh_options& o, Plan& pl) {
  pl.pieces = dtype == RH_F32_BF16X3 ? 3 : 2;
  if (dtype == RH_F32_BF16X3) dtype = RH_F32_BF16X2;
  const bool split = dtype == RH_F32_BF16X2;
  rh_status s = check_tensor(order, dims, split ? RH_F32 : dtype);
  if (s != RH_OK) return s;
  if (split) {
    dtype = RH_F32;
    pl.in_form = RH_F32_BF16X2;
  }
  RH_CHECK_ARG(ranks != nullptr, "ranks is NULL");
  RH_CHECK_ARG(o.p >= 0, "oversampling p must be >= 0");
  RH_CHECK_ARG(o.tensor_id >= 0 && o.tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(o.svd_route == 0 || o.svd_route == 1, "svd_route must be 0 or 1");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(ranks[k] >= 1, "every rank must be >= 1");
  pl.d = order;
  pl.dtype = dtype;
  for (int n = 0; n < order; ++n) {
    Step st;
    st.mode = n;
    st.v = mode_view(order, dims, n);
    const int64_t lim = std::min<int64_t>(st.v.I, st.v.M());
    int64_t ell = (int64_t)ranks[n] + o.p;
    if (ell > lim) {
      if (!o.clamp) {
        set_error("invalid argument: r_n + p = " + std::to_string(ell) + " exceeds min(I_n, prod of the other sizes) = " +
                  std::to_string(lim) + " for mode " + std::to_string(n));
        return RH_EINVAL;
      }
      ell = lim;
    }
    if (ell > RH_MAX_ELL) {
      set_error("unsupported: r_n + p = " + std::to_string(ell) + " exceeds RH_MAX_ELL (64)");
      return RH_EUNSUPPORTED;
    }
    st.ell = (int)ell;
    st.ko = o.truncate ? std::min<int>(ranks[n], st.ell) : st.ell;
    st.sk = plan_sketch(st.v, st.ell);
    st.tr = plan_trunc(ModeView{st.v.L, st.ell, st.v.R}, st.ell);
    pl.max_I_ell = std::max(pl.max_I_ell, (size_t)(st.v.I * st.ell));
    pl.max_tensor = std::max(pl.max_tensor, (size_t)(st.v.M() * st.ell));
    pl.max_part = std::max(pl.max_part, st.sk.part_elems());
    pl.max_pnorm = std::max(pl.max_pnorm, st.sk.norm_elems());
    pl.max_orth = std::max(pl.max_orth, orth_workspace_elems(st.v.I, st.ell));
    pl.max_trunc = std::max(pl.max_trunc, dtype == RH_F64 ? trunc_workspace_elems<double>(st.tr)
                                                           : trunc_workspace_elems<float>(st.tr));
    pl.steps.push_back(st);
  }
  std::vector<int32_t> ks(order);
  for (const Step& st : pl.steps) ks[st.mode] = st.ko;
  size_t fe = 0;
  pl.max_tensor = std::max(pl.max_tensor, core_chain_elems(order, dims, ks.data(), &fe));
  pl.fac_elems = fe;
  if (split) {
    pl.max_pnorm = std::max<size_t>(pl.max_pnorm, 1024);
    for (Step& st : pl.steps) {
      const bool k0 = st.v.L == 1 && sketch_tc_supported(st.v, st.ell) && ttm_tc_supported(st.v, st.ell);
      const bool ks_ = st.v.L > 1 && sketch_tc_strided_supported(st.v, st.ell) &&
                       ttm_tc_strided_supported(st.v, st.ell);
      st.tc = k0 || ks_;
      if (st.tc) pl.tc_part = std::max(pl.tc_part, (size_t)sketch_tc_ctas(st.v) * st.ell * st.v.I);
    }
    int64_t imax = 1;
    for (int n = 0; n < order; ++n) imax = std::max<int64_t>(imax, dims[n]);
    pl.qa_elems = (size_t)128 * ((imax + 7) / 8 * 8);   // the split Q of any mode or factor of the core chain
  }
  return plan_power(o, pl);
}

struct Bufs {
  void* part;
  double* part_norm;
  double* normx;
  double* Y;
  double* orth;
  double* Q;
  void* Qc;
  void* W[2];
  void* trunc;
  double* Ub;
  double* sv;
  void* Uc;
  void* fac;
  float* tc_part;
  uint16_t* qa;
  int32_t* err;
};

Bufs carve(Arena& ar, const Plan& pl) {
  Bufs b;
  const bool f64 = pl.dtype == RH_F64;
  auto takeT = [&](size_t n) -> void* { return f64 ? (void*)ar.take<double>(n) : (void*)ar.take<float>(n); };
  b.part = takeT(pl.max_part);
  b.part_norm = ar.take<double>(std::max<size_t>(pl.max_pnorm, 256));   // also the final norm's partials
  b.normx = ar.take<double>(1);
  b.Y = ar.take<double>(pl.max_I_ell);
  b.orth = ar.take<double>(pl.max_orth);
  b.Q = ar.take<double>(pl.max_I_ell);
  b.Qc = takeT(pl.max_I_ell);
  b.W[0] = takeT(pl.max_tensor);
  b.W[1] = takeT(pl.max_tensor);
  b.trunc = takeT(pl.max_trunc);
  b.Ub = ar.take<double>(RH_MAX_ELL * RH_MAX_ELL);
  b.sv = ar.take<double>(RH_MAX_ELL);
  b.Uc = takeT(RH_MAX_ELL * RH_MAX_ELL);
  b.fac = pl.fac_elems ? takeT(pl.fac_elems) : nullptr;
  b.tc_part = pl.tc_part ? ar.take<float>(pl.tc_part) : nullptr;
  b.qa = pl.qa_elems ? ar.take<uint16_t>(pl.qa_elems) : nullptr;
  b.err = ar.take<int32_t>(4);
  return b;
}

// info |= bits, plus 16 when a tensor-core kernel recorded a bounded wait that gave up (*err != 0);
// the wait flag is cleared so that the next mode reports its own.
struct InfoOrOp {
  struct Args {
    int32_t* info;
    int32_t bits;
    int32_t* err;
  };
  static constexpr int kThreads = 32, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& a) {
    if (threadIdx.x == 0 && g.bx == 0 && g.by == 0) {
      int32_t bits = a.bits;
      if (a.err != nullptr && *a.err != 0) {
        bits |= 16;
        *a.err = 0;
      }
      if (bits) *a.info |= bits;
    }
  }
};
rh_status set_info_bits(int32_t* info, int32_t bits, cudaStream_t st, int32_t* err = nullptr) {
  return emit<InfoOrOp>(SITE_INFO, 0, dim3(1), 0, st, InfoOrOp::Args{info, bits, err});
}

// Randomized subspace iteration (Sec. 5 "Variants"; used with one step in Sec. 6): q steps of
// W = orth(G_(n)^T Q), Y = G_(n) W, Q = orth(Y) after the first QR of the range finder.  B = Q^T G_(n)
// is the mode product (on the tensor cores when the mode's sketch runs there, with Q split into
// BF16 pieces as for the mode product of Alg. 1 step 3), W replaces B in B's buffer
// (launch_power_basis), Y = G_(n) W is a sketch against the dense W (on a tensor-core mode every
// element of G enters as its BF16 head + tail, the value the tensor-core kernels read), then the
// QR of Alg. 1 step 2.  Step keys j kStepStride + 1 + it keep a recorded program's keys increasing.
template <typename T>
rh_status run_power(const Plan& pl, const Step& sp, int j, const T* cur, const float* tc_src, bool tc, const Bufs& b,
                    T* Bw, int32_t* info, cudaStream_t st) {
  rh_status s;
  for (int it = 0; it < pl.power; ++it) {
    record_step(kStepStride * j + 1 + it);
    ProfileScope ps(PROF_POWER, j, st);
    if (tc) {
      s = sp.v.L == 1 ? launch_ttm_tc_f32(sp.v, sp.ell, tc_src, b.Q, b.qa, reinterpret_cast<float*>(Bw), b.err, st)
                      : launch_ttm_tc_f32s(sp.v, sp.ell, tc_src, b.Q, b.qa, reinterpret_cast<float*>(Bw), b.err, st);
      if (s != RH_OK) return s;
    } else {
      if ((s = launch_cast<T>(b.Q, static_cast<T*>(b.Qc), sp.v.I * sp.ell, st, SITE_POWER_CAST)) != RH_OK) return s;
      if ((s = launch_ttm<T, T>(sp.v, cur, static_cast<const T*>(b.Qc), sp.ell, Bw, st, SITE_POWER_TTM)) != RH_OK)
        return s;
    }
    if ((s = launch_power_basis<T>(sp.tr, Bw, static_cast<T*>(b.trunc), st)) != RH_OK) return s;
    const T* G = tc ? reinterpret_cast<const T*>(tc_src) : cur;
    if ((s = launch_sketch_dense<T>(sp.skd, G, Bw, tc, static_cast<T*>(b.part), st, SITE_POWER_SKETCH)) != RH_OK)
      return s;
    if ((s = launch_sketch_reduce<T>(sp.skd, static_cast<const T*>(b.part), nullptr, b.Y, nullptr, st,
                                     SITE_POWER_SKETCH_REDUCE)) != RH_OK)
      return s;
    if ((s = launch_orthonormalize(sp.v.I, sp.ell, b.Y, b.Q, info ? info + sp.mode : nullptr, b.orth, st,
                                   sizeof(T) == 4)) != RH_OK)
      return s;
  }
  return RH_OK;
}

template <typename T>
rh_status run_rsthosvd(const Plan& pl, const void* Xraw, const rh_options& o, double* const* factors, double* core,
                       double* norms, int32_t* info, const Bufs& b, cudaStream_t st) {
  const T* X = static_cast<const T*>(Xraw);
  const T* cur = X;
  int cur_buf = -1;  // -1: the input tensor
  rh_status s;
  const int nsteps = (int)pl.steps.size();
  const bool tc0 = pl.in_form >= 0;
  const bool f32in = pl.in_form == RH_F32_BF16X2;   // FP32 input split on the fly
  const bool fp8in = pl.in_form == RH_FP8_E4M3;     // E4M3 input dequantized and split on the fly
  const Fp8Layout f8 = fp8in ? fp8_layout(pl.d, pl.dims0.data()) : Fp8Layout{};
  const uint8_t* x8 = static_cast<const uint8_t*>(Xraw);
  const float* scales8 = fp8in ? reinterpret_cast<const float*>(x8 + f8.scale_off) : nullptr;
  const uint16_t* piece0 = (f32in || fp8in) ? nullptr : static_cast<const uint16_t*>(Xraw);
  const uint16_t* piece1 = (pl.in_form == RH_BF16X2) ? piece0 + pl.steps[0].v.I * pl.steps[0].v.M() : nullptr;
  const bool stc0 = pl.steps[0].stc;
  const SmallInput small_in{Xraw, pl.in_form, fp8in ? f8.ld : 0, scales8};
  if (stc0) {
    if ((s = emit_memset(SITE_ENTRY, 1, b.err, sizeof(int32_t), st)) != RH_OK) return s;
  } else if (tc0) {
    RH_CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(int32_t), st));
  }
  for (int j = 0; j < nsteps; ++j) {
    record_step(kStepStride * j);
    const Step& sp = pl.steps[j];
    const bool last = (j == nsteps - 1);
    const bool tc = tc0 && sp.tc;
    const bool first = (j == 0);
    const uint32_t sid = ((uint32_t)o.tensor_id << 4) | (uint32_t)sp.mode;
    // Alg. 1 step 1: Y = G_(n) Omega_n   (+ ||X||^2 on the first pass)
    SketchBufs sb{b.part, b.part_norm};
    double* n2 = (j == 0) ? (norms ? norms : b.normx) : nullptr;
    // the input itself is split on the fly (FP32 input) or given as pieces; later cores are FP32
    const bool in_pieces = tc && first && !f32in && !fp8in;
    const bool in_fp8 = tc && first && fp8in;
    const float* tc_src = first ? static_cast<const float*>(Xraw) : reinterpret_cast<const float*>(cur);
    if (sp.stc) {
      {
        ProfileScope ps(PROF_SKETCH, j, st);
        if ((s = launch_sketch_small_tc(sp.sk, small_in, o.seed, sid, static_cast<float*>(sb.part), sb.part_norm, b.err,
                                        st)) != RH_OK)
          return s;
      }
      if ((s = launch_sketch_reduce<float>(sp.sk, static_cast<const float*>(sb.part), sb.part_norm, b.Y, n2, st)) !=
          RH_OK)
        return s;
    } else if (tc) {
      {
        ProfileScope ps(PROF_SKETCH, j, st);
        if (in_pieces)
          s = launch_sketch_tc(sp.v, sp.ell, piece0, piece1, o.seed, sid, b.tc_part, b.err, st);
        else if (in_fp8)
          s = launch_sketch_tc_fp8(sp.v, sp.ell, x8, scales8, f8.ld, o.seed, sid, b.tc_part,
                                   norms ? b.part_norm : nullptr, b.err, st);
        else
          s = launch_sketch_tc_f32(sp.v, sp.ell, tc_src, o.seed, sid, b.tc_part,
                                   (first && norms) ? b.part_norm : nullptr, b.err, st, 0, pl.pieces);
        if (s != RH_OK) return s;
      }
      SketchPlan rp = sp.sk;
      rp.S = sketch_tc_ctas(sp.v);
      if ((s = launch_sketch_reduce<float>(rp, b.tc_part, nullptr, b.Y, nullptr, st)) != RH_OK) return s;
      if (first && norms) {
        s = (f32in || fp8in) ? launch_sum_n(b.part_norm, rp.S, norms, st)
                             : launch_pieces_sumsq(piece0, piece1, sp.v.I * sp.v.M(), b.part_norm, norms, st);
        if (s != RH_OK) return s;
      }
    } else {
      {
        ProfileScope ps(PROF_SKETCH, j, st);
        if ((s = launch_sketch<T>(sp.sk, cur, o.seed, sid, static_cast<T*>(sb.part), sb.part_norm, st)) != RH_OK)
          return s;
      }
      if ((s = launch_sketch_reduce<T>(sp.sk, static_cast<const T*>(sb.part), sb.part_norm, b.Y, n2, st)) != RH_OK)
        return s;
    }
    // Alg. 1 step 2: Q = orth(Y)
    {
      ProfileScope ps(PROF_ORTH, j, st);
      if ((s = launch_orthonormalize(sp.v.I, sp.ell, b.Y, b.Q, info ? info + sp.mode : nullptr, b.orth, st,
                                    sizeof(T) == 4)) !=
          RH_OK)
        return s;
    }
    const int wb = (cur_buf == 0) ? 1 : 0;
    T* B = static_cast<T*>(b.W[wb]);
    if (pl.power && (s = run_power<T>(pl, sp, j, cur, tc_src, tc, b, B, info, st)) != RH_OK) return s;
    if ((s = launch_cast<T>(b.Q, static_cast<T*>(b.Qc), sp.v.I * sp.ell, st)) != RH_OK) return s;
    // Alg. 1 step 3: B = Q^T G_(n)   (the mode-n product G x_n Q^T)
    const bool direct_core = last && !o.truncate;
    // the FP32 Gram route of the truncation gets W's partials from the tensor-core mode product
    // (every tensor-core form, so that the forms stay bit-identical to one another), when a tile
    // has enough K stages (I >= 512) to hide the epilogue's extra work behind its MMAs
    const bool gram_fused = tc && !sp.stc && o.truncate && !o.svd_route && sp.ko >= 1 && sizeof(T) == 4 &&
                            ttm_tc_gram_supported(sp.ell) && sp.v.I >= kGramFuseMinRows;
    double* gram_part = gram_fused ? trunc_gram_part(sp.tr, reinterpret_cast<float*>(b.trunc)) : nullptr;
    const int gram_nparts = gram_fused ? ttm_tc_ctas(sp.v) : 0;
    if (sp.stc) {
      ProfileScope ps(PROF_TTM, j, st);
      if (direct_core) {
        set_error("unsupported: single-mode untruncated BF16 request");
        return RH_EUNSUPPORTED;
      }
      if ((s = launch_ttm_small_tc(sp.v, small_in, b.Q, sp.ell, reinterpret_cast<float*>(B), b.err, st)) != RH_OK)
        return s;
    } else if (tc) {
      ProfileScope ps(PROF_TTM, j, st);
      if (direct_core) {
        set_error("unsupported: single-mode untruncated BF16 request");
        return RH_EUNSUPPORTED;
      }
      if (in_pieces)
        s = launch_ttm_tc(sp.v, sp.ell, piece0, piece1, b.Q, b.qa, reinterpret_cast<float*>(B), b.err, st, gram_part);
      else if (in_fp8)
        s = launch_ttm_tc_fp8(sp.v, sp.ell, x8, scales8, f8.ld, b.Q, b.qa, reinterpret_cast<float*>(B), b.err, st,
                              gram_part);
      else
        s = launch_ttm_tc_f32(sp.v, sp.ell, tc_src, b.Q, b.qa, reinterpret_cast<float*>(B), b.err, st, pl.pieces,
                              gram_part);
      if (s != RH_OK) return s;
    } else {
      ProfileScope ps(PROF_TTM, j, st);
      if (direct_core) {
        if ((s = launch_ttm<T, double>(sp.v, cur, static_cast<const T*>(b.Qc), sp.ell, core, st, SITE_MODE_PRODUCT)) !=
            RH_OK)
          return s;
      } else {
        if ((s = launch_ttm<T, T>(sp.v, cur, static_cast<const T*>(b.Qc), sp.ell, B, st, SITE_MODE_PRODUCT)) != RH_OK)
          return s;
      }
    }
    if (o.truncate) {
      // Alg. 1 steps 4-6: SVD of B, A_n = Q U_B(:, 1:r), G_(n) <- S V^T = U_B(:, 1:r)^T B
      {
        ProfileScope ps(PROF_TRUNC, j, st);
        // r = 0 keeps the truncation SVD on the tall-skinny QR (svd_route 1)
        if ((s = launch_trunc_svd<T>(sp.tr, B, static_cast<T*>(b.trunc), b.Ub, b.sv, st, o.svd_route ? 0 : sp.ko,
                                      info ? info + sp.mode : nullptr, gram_nparts)) != RH_OK) return s;
      }
      if ((s = launch_factor_and_cast<T>(sp.v.I, sp.ell, sp.ko, b.Q, b.Ub, factors[sp.mode], static_cast<T*>(b.Uc),
                                         st)) != RH_OK)
        return s;
      const ModeView vb{sp.v.L, sp.ell, sp.v.R};
      ProfileScope ps(PROF_TTM_CORE, j, st);
      if (sp.cp) {
        // B has the new mode fastest: G <- U_r^T B written in the order the next step reads
        const float* Bf = reinterpret_cast<const float*>(B);
        const float* Uf = reinterpret_cast<const float*>(b.Uc);
        if (last) {
          if ((s = launch_core_product<double>(Bf, sp.ell, sp.ko, sp.v.M(), sp.cout, Uf, core, st)) != RH_OK)
            return s;
        } else {
          const int wg = 1 - wb;
          if (sp.cp_tc)
            s = launch_core_product_tc(Bf, sp.ell, sp.ko, sp.v.M(), sp.cout, Uf, b.qa, static_cast<float*>(b.W[wg]),
                                       b.err, st, pl.pieces);
          else
            s = launch_core_product<float>(Bf, sp.ell, sp.ko, sp.v.M(), sp.cout, Uf, static_cast<float*>(b.W[wg]),
                                           st);
          if (s != RH_OK) return s;
          cur = static_cast<const T*>(b.W[wg]);
          cur_buf = wg;
        }
      } else if (last) {
        if ((s = launch_ttm<T, double>(vb, B, static_cast<const T*>(b.Uc), sp.ko, core, st, SITE_CORE)) != RH_OK)
          return s;
      } else {
        const int wg = 1 - wb;
        if ((s = launch_ttm<T, T>(vb, B, static_cast<const T*>(b.Uc), sp.ko, static_cast<T*>(b.W[wg]), st, SITE_CORE)) !=
            RH_OK)
          return s;
        cur = static_cast<const T*>(b.W[wg]);
        cur_buf = wg;
      }
    } else {
      RH_CUDA_TRY(cudaMemcpyAsync(factors[sp.mode], b.Q, sizeof(double) * sp.v.I * sp.ell, cudaMemcpyDeviceToDevice, st));
      if (!last) {
        cur = B;
        cur_buf = wb;
      }
    }
    // info bit 4: this mode's sketch and mode product ran on the tensor cores; bit 16: a tensor-core
    // kernel of this mode gave up a bounded wait (the mode's outputs are invalid)
    if (info && (tc || sp.stc || (o.truncate && sp.cp && sp.cp_tc && !last)) &&
        (s = set_info_bits(info + sp.mode, (tc || sp.stc) ? 4 : 0, st, b.err)) != RH_OK)
      return s;
  }
  if (norms) {
    record_step(kStepStride * nsteps);
    int64_t ncore = 1;
    // final core sizes
    std::vector<int64_t> dims_out(pl.d, 0);
    for (const Step& sp : pl.steps) dims_out[sp.mode] = sp.ko;
    for (int k = 0; k < pl.d; ++k) ncore *= dims_out[k];
    if ((s = launch_sumsq(core, ncore, norms + 1, st, b.part_norm, std::max<size_t>(pl.max_pnorm, 256))) != RH_OK) return s;
  }
  return RH_OK;
}

template <typename T>
rh_status run_rhosvd(const Plan& pl, const int64_t* dims, const T* X, const rh_options& o, double* const* factors,
                     double* core, double* norms, int32_t* info, const Bufs& b, cudaStream_t st) {
  rh_status s;
  std::vector<int32_t> ks(pl.d);
  const bool split = pl.in_form == RH_F32_BF16X2;
  const float* Xf = reinterpret_cast<const float*>(X);
  if (split) RH_CUDA_TRY(cudaMemsetAsync(b.err, 0, sizeof(int32_t), st));
  for (size_t j = 0; j < pl.steps.size(); ++j) {
    const Step& sp = pl.steps[j];
    ks[sp.mode] = sp.ko;
    const uint32_t sid = ((uint32_t)o.tensor_id << 4) | (uint32_t)sp.mode;
    double* n2 = (j == 0) ? (norms ? norms : b.normx) : nullptr;
    const bool tc = split && sp.tc;
    if (tc) {
      // the sketch of Alg. 2 step 3 on the tensor cores (mode 0 MN-major, other modes K-major pieces)
      {
        ProfileScope ps(PROF_SKETCH, (int)j, st);
        double* np = n2 ? b.part_norm : nullptr;
        s = sp.v.L == 1 ? launch_sketch_tc_f32(sp.v, sp.ell, Xf, o.seed, sid, b.tc_part, np, b.err, st, 0, pl.pieces)
                        : launch_sketch_tc_f32s(sp.v, sp.ell, Xf, o.seed, sid, b.tc_part, np, b.err, st, 0, pl.pieces);
        if (s != RH_OK) return s;
      }
      SketchPlan rp = sp.sk;
      rp.S = sketch_tc_ctas(sp.v);
      if ((s = launch_sketch_reduce<float>(rp, b.tc_part, nullptr, b.Y, nullptr, st)) != RH_OK) return s;
      if (n2 && (s = launch_sum_n(b.part_norm, rp.S, n2, st)) != RH_OK) return s;
    } else {
      {
        ProfileScope ps(PROF_SKETCH, (int)j, st);
        if ((s = launch_sketch<T>(sp.sk, X, o.seed, sid, static_cast<T*>(b.part), b.part_norm, st)) != RH_OK)
          return s;
      }
      if ((s = launch_sketch_reduce<T>(sp.sk, static_cast<const T*>(b.part), b.part_norm, b.Y, n2, st)) != RH_OK)
        return s;
    }
    {
      ProfileScope ps(PROF_ORTH, (int)j, st);
      if ((s = launch_orthonormalize(sp.v.I, sp.ell, b.Y, b.Q, info ? info + sp.mode : nullptr, b.orth, st,
                                    sizeof(T) == 4)) !=
          RH_OK)
        return s;
    }
    T* B = static_cast<T*>(b.W[0]);
    if (pl.power && (s = run_power<T>(pl, sp, (int)j, X, Xf, tc, b, B, info, st)) != RH_OK) return s;
    if (!o.truncate) {
      RH_CUDA_TRY(cudaMemcpyAsync(factors[sp.mode], b.Q, sizeof(double) * sp.v.I * sp.ell, cudaMemcpyDeviceToDevice, st));
      if (info && tc && (s = set_info_bits(info + sp.mode, 4, st, b.err)) != RH_OK) return s;
      continue;
    }
    if ((s = launch_cast<T>(b.Q, static_cast<T*>(b.Qc), sp.v.I * sp.ell, st)) != RH_OK) return s;
    const bool gram_fused = tc && !o.svd_route && sp.ko >= 1 && sizeof(T) == 4 && ttm_tc_gram_supported(sp.ell) &&
                            sp.v.I >= kGramFuseMinRows;
    double* gram_part = gram_fused ? trunc_gram_part(sp.tr, reinterpret_cast<float*>(b.trunc)) : nullptr;
    const int gram_nparts = gram_fused ? ttm_tc_ctas(sp.v) : 0;
    {
      ProfileScope ps(PROF_TTM, (int)j, st);
      if (tc) {
        float* Bf = reinterpret_cast<float*>(B);
        s = sp.v.L == 1 ? launch_ttm_tc_f32(sp.v, sp.ell, Xf, b.Q, b.qa, Bf, b.err, st, pl.pieces, gram_part)
                        : launch_ttm_tc_f32s(sp.v, sp.ell, Xf, b.Q, b.qa, Bf, b.err, st, pl.pieces, gram_part);
        if (s != RH_OK) return s;
      } else if ((s = launch_ttm<T, T>(sp.v, X, static_cast<const T*>(b.Qc), sp.ell, B, st)) != RH_OK) {
        return s;
      }
    }
    {
      ProfileScope ps(PROF_TRUNC, (int)j, st);
      if ((s = launch_trunc_svd<T>(sp.tr, B, static_cast<T*>(b.trunc), b.Ub, b.sv, st, o.svd_route ? 0 : sp.ko,
                                      info ? info + sp.mode : nullptr, gram_nparts)) != RH_OK) return s;
    }
    if ((s = launch_factor_and_cast<T>(sp.v.I, sp.ell, sp.ko, b.Q, b.Ub, factors[sp.mode], static_cast<T*>(b.Uc),
                                       st)) != RH_OK)
      return s;
    // info bit 4: this mode's sketch and mode product ran on the tensor cores; 16: a wait gave up
    if (info && tc && (s = set_info_bits(info + sp.mode, 4, st, b.err)) != RH_OK) return s;
  }
  {
    ProfileScope ps(PROF_TTM_CORE, 0, st);
    if ((s = launch_core_ttm<T>(pl.d, dims, X, factors, ks.data(), core, static_cast<T*>(b.fac),
                                static_cast<T*>(b.W[0]), static_cast<T*>(b.W[1]), st, split, b.qa, b.err,
                                pl.pieces)) != RH_OK)
      return s;
  }
  if (split && info && (s = set_info_bits(info + pl.steps.back().mode, 0, st, b.err)) != RH_OK) return s;
  if (norms) {
    int64_t ncore = 1;
    for (int k = 0; k < pl.d; ++k) ncore *= ks[k];
    if ((s = launch_sumsq(core, ncore, norms + 1, st, b.part_norm, std::max<size_t>(pl.max_pnorm, 256))) != RH_OK) return s;
  }
  return RH_OK;
}

rh_options opts_or_default(const rh_options* o) {
  rh_options d;
  rh_options_default(&d);
  return o ? *o : d;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" {

static bool is_bf16_form(int32_t dtype) { return bf16_form(dtype); }

// The sketch of mode 0 in a BF16 form whose I_0 the persistent tensor-core kernel does not take
// (I_0 % 8 != 0) runs on the small-row kernel when I_0 <= 128 and ell <= 32.
static bool sketch_small_route(int32_t dtype, const ModeView& v, int32_t ell, int32_t mode) {
  (void)dtype;
  return mode == 0 && !sketch_tc_supported(v, ell) && small_tc_supported(v, ell);
}

static size_t sketch_tc_ws(int32_t order, const int64_t* dims, int32_t ell, int32_t mode = 0, int32_t dtype = RH_BF16,
                           bool allow_small = true) {
  const ModeView v = mode_view(order, dims, mode);
  const int64_t S =
      allow_small && sketch_small_route(dtype, v, ell, mode) ? plan_sketch_small_tc(v, ell).S : sketch_tc_ctas(v);
  Arena ar(nullptr);
  ar.take<int32_t>(4);   // wait status, first (documented)
  ar.take<float>((size_t)S * ell * v.I);
  ar.take<double>((size_t)S);
  return ar.used;
}

rh_status rh_fp8_layout(int32_t order, const int64_t* dims, int64_t* ld, size_t* scale_offset, size_t* nscales,
                        size_t* bytes) {
  clear_error();
  rh_status s = check_tensor(order, dims, RH_F32);
  if (s != RH_OK) return s;
  const Fp8Layout f = fp8_layout(order, dims);
  if (ld) *ld = f.ld;
  if (scale_offset) *scale_offset = f.scale_off;
  if (nscales) *nscales = f.nscales;
  if (bytes) *bytes = f.bytes;
  return RH_OK;
}

size_t rhosvd_sketch_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode, int32_t ell) {
  // RH_F32_BF16X3: the split form's tensor-core kernels with three exact pieces (no small-row route)
  const bool x3 = dtype == RH_F32_BF16X3;
  if (x3) dtype = RH_F32_BF16X2;
  if (is_bf16_form(dtype)) {
    if (order < 1 || order > RH_MAX_ORDER || dims == nullptr || mode < 0 || mode >= order || ell < 1 ||
        ell > RH_MAX_ELL)
      return 0;
    if (mode != 0 && dtype != RH_F32_BF16X2) return 0;
    for (int k = 0; k < order; ++k)
      if (dims[k] < 1) return 0;
    return sketch_tc_ws(order, dims, ell, mode, dtype, !x3);
  }
  if (check_tensor(order, dims, dtype) != RH_OK || mode < 0 || mode >= order || ell < 1 || ell > RH_MAX_ELL) return 0;
  const SketchPlan pl = plan_sketch(mode_view(order, dims, mode), ell);
  Arena ar(nullptr);
  carve_sketch(ar, pl, dtype);
  return ar.used;
}

rh_status rhosvd_sketch(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode, int32_t ell,
                        uint64_t seed, int32_t tensor_id, double* Y, double* norm2, void* workspace,
                        size_t workspace_bytes, void* stream) {
  return rhosvd_sketch_offset(order, dims, dtype, X, mode, ell, seed, tensor_id, 0, 0, Y, norm2, workspace,
                              workspace_bytes, stream);
}

rh_status rhosvd_sketch_offset(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode,
                               int32_t ell, uint64_t seed, int32_t tensor_id, int64_t row0, int32_t accumulate,
                               double* Y, double* norm2, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  RH_CHECK_ARG(row0 >= 0, "row0 must be >= 0");
  RH_CHECK_ARG(accumulate == 0 || accumulate == 1, "accumulate must be 0 or 1");
  const bool x3 = dtype == RH_F32_BF16X3;
  if (x3) dtype = RH_F32_BF16X2;
  if (is_bf16_form(dtype)) {
    RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
    for (int k = 0; k < order; ++k) RH_CHECK_ARG(dims[k] >= 1, "every dimension must be >= 1");
    RH_CHECK_ARG(mode >= 0 && mode < order, "mode out of range");
    RH_CHECK_ARG(mode == 0 || dtype == RH_F32_BF16X2, "the BF16 and E4M3 forms sketch mode 0 only");
    RH_CHECK_ARG(ell >= 1 && ell <= RH_MAX_ELL, "ell must be in [1, 64]");
    RH_CHECK_ARG(tensor_id >= 0 && tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
    RH_CHECK_ARG(X != nullptr && Y != nullptr, "X and Y must be non-NULL");
    RH_CHECK_ARG(norm2 == nullptr || converted_form(dtype), "norm2 is not available for RH_BF16 / RH_BF16X2");
    const ModeView v = mode_view(order, dims, mode);
    const bool small = !x3 && sketch_small_route(dtype, v, ell, mode);
    if (!small && (mode == 0 ? !sketch_tc_supported(v, ell) : !sketch_tc_strided_supported(v, ell))) {
      set_error(mode == 0 ? "unsupported: the BF16 sketch needs I_0 % 8 == 0 and I_0 <= 1024, or I_0 <= 128 and "
                            "ell <= 32"
                          : "unsupported: a split sketch of a later mode needs the product of the earlier sizes to "
                            "be a multiple of 64 and I_n <= 1024");
      return RH_EUNSUPPORTED;
    }
    const size_t need = sketch_tc_ws(order, dims, ell, mode, dtype, !x3);
    if (workspace == nullptr || workspace_bytes < need) {
      set_error("workspace too small: need " + std::to_string(need) + " bytes");
      return RH_ENOMEM;
    }
    Arena ar(workspace);
    SketchPlan sp_small;
    if (small) {
      sp_small = plan_sketch_small_tc(v, ell);
      sp_small.row0 = row0;
    }
    const int S = small ? sp_small.S : sketch_tc_ctas(v);
    int32_t* err = ar.take<int32_t>(4);   // wait status: the first int32 of the workspace
    float* part = ar.take<float>((size_t)S * ell * v.I);
    double* norm_part = ar.take<double>((size_t)S);
    cudaStream_t st = (cudaStream_t)stream;
    RH_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    const uint32_t sid = ((uint32_t)tensor_id << 4) | (uint32_t)mode;
    rh_status s;
    if (small) {
      SmallInput in{X, dtype};
      if (dtype == RH_FP8_E4M3) {
        const Fp8Layout f8 = fp8_layout(order, dims);
        in.ld = f8.ld;
        in.scales = reinterpret_cast<const float*>(static_cast<const uint8_t*>(X) + f8.scale_off);
      }
      s = launch_sketch_small_tc(sp_small, in, seed, sid, part, norm2 ? norm_part : nullptr, err, st, SITE_OTHER);
      if (s == RH_OK && norm2) s = launch_sum_n(norm_part, S, norm2, st, accumulate);
    } else if (dtype == RH_F32_BF16X2) {
      s = mode == 0 ? launch_sketch_tc_f32(v, ell, static_cast<const float*>(X), seed, sid, part,
                                           norm2 ? norm_part : nullptr, err, st, row0, x3 ? 3 : 2)
                    : launch_sketch_tc_f32s(v, ell, static_cast<const float*>(X), seed, sid, part,
                                            norm2 ? norm_part : nullptr, err, st, row0, x3 ? 3 : 2);
      if (s == RH_OK && norm2) s = launch_sum_n(norm_part, S, norm2, st, accumulate);
    } else if (dtype == RH_FP8_E4M3) {
      const Fp8Layout f8 = fp8_layout(order, dims);
      const uint8_t* x8 = static_cast<const uint8_t*>(X);
      s = launch_sketch_tc_fp8(v, ell, x8, reinterpret_cast<const float*>(x8 + f8.scale_off), f8.ld, seed, sid, part,
                               norm2 ? norm_part : nullptr, err, st, row0);
      if (s == RH_OK && norm2) s = launch_sum_n(norm_part, S, norm2, st, accumulate);
    } else {
      const uint16_t* p0 = static_cast<const uint16_t*>(X);
      const uint16_t* p1 = dtype == RH_BF16X2 ? p0 + v.I * v.M() : nullptr;
      s = launch_sketch_tc(v, ell, p0, p1, seed, sid, part, err, st, row0);
    }
    if (s != RH_OK) return s;
    SketchPlan rp;
    rp.v = v;
    rp.ell = ell;
    rp.ellp = ell_pad_of(ell);
    rp.gx = 0;
    rp.S = S;
    rp.chunk = 0;
    return launch_sketch_reduce<float>(rp, part, nullptr, Y, nullptr, st, SITE_SKETCH_REDUCE, accumulate);
  }
  rh_status s = check_tensor(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(mode >= 0 && mode < order && mode < 16, "mode out of range");
  RH_CHECK_ARG(ell >= 1 && ell <= RH_MAX_ELL, "ell must be in [1, 64]");
  RH_CHECK_ARG(tensor_id >= 0 && tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(X != nullptr && Y != nullptr, "X and Y must be non-NULL");
  SketchPlan pl = plan_sketch(mode_view(order, dims, mode), ell);
  pl.row0 = row0;
  Arena ar(workspace);
  Arena meas(nullptr);
  carve_sketch(meas, pl, dtype);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  const SketchBufs b = carve_sketch(ar, pl, dtype);
  const uint32_t sid = ((uint32_t)tensor_id << 4) | (uint32_t)mode;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == RH_F64)
    return run_sketch<double>(pl, static_cast<const double*>(X), seed, sid, b, Y, norm2, st, accumulate);
  return run_sketch<float>(pl, static_cast<const float*>(X), seed, sid, b, Y, norm2, st, accumulate);
}

size_t rh_mode_product_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode, int32_t k) {
  if (!(bf16_form(dtype) || dtype == RH_F32_BF16X3) || order < 1 || order > RH_MAX_ORDER || dims == nullptr ||
      mode != 0)
    return 0;
  Arena ar(nullptr);
  ar.take<int32_t>(4);   // wait status, first (documented)
  ar.take<uint16_t>((size_t)128 * dims[0]);
  (void)k;
  return ar.used;
}

rh_status rh_mode_product(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t mode,
                          int32_t k, const void* A, int32_t transpose, int32_t out_dtype, void* Y, void* stream) {
  clear_error();
  if (bf16_form(dtype)) {
    RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
    for (int q = 0; q < order; ++q) RH_CHECK_ARG(dims[q] >= 1, "every dimension must be >= 1");
    RH_CHECK_ARG(mode == 0 && transpose == 1 && out_dtype == RH_F32, "BF16 forms: mode 0, transpose 1, FP32 output");
    RH_CHECK_ARG(X != nullptr && A != nullptr && Y != nullptr, "X, A and Y must be non-NULL");
    const ModeView v = mode_view(order, dims, 0);
    if (!ttm_tc_supported(v, k)) {
      set_error("unsupported: the BF16 mode product needs I_0 % 8 == 0 and k <= 64");
      return RH_EUNSUPPORTED;
    }
    RH_CHECK_ARG(false, "BF16 forms need scratch: use rh_mode_product_bf16");
  }
  rh_status s = check_tensor(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(mode >= 0 && mode < order, "mode out of range");
  RH_CHECK_ARG(k >= 1, "k must be >= 1");
  RH_CHECK_ARG(transpose == 0 || transpose == 1, "transpose must be 0 or 1");
  RH_CHECK_ARG(out_dtype == RH_F64 || out_dtype == dtype, "out_dtype must equal dtype or be RH_F64");
  RH_CHECK_ARG(X != nullptr && A != nullptr && Y != nullptr, "X, A and Y must be non-NULL");
  const ModeView v = mode_view(order, dims, mode);
  cudaStream_t st = (cudaStream_t)stream;
  // transpose = 1: A is I_n x k, Y = X x_n A^T;  transpose = 0: A is k x I_n, Y = X x_n A
  const int64_t qsi = transpose ? 1 : k, qsc = transpose ? v.I : 1;
  if (dtype == RH_F64)
    return launch_ttm_strided<double, double>(v, static_cast<const double*>(X), static_cast<const double*>(A), qsi, qsc,
                                              k, static_cast<double*>(Y), st);
  if (out_dtype == RH_F64)
    return launch_ttm_strided<float, double>(v, static_cast<const float*>(X), static_cast<const float*>(A), qsi, qsc,
                                             k, static_cast<double*>(Y), st);
  return launch_ttm_strided<float, float>(v, static_cast<const float*>(X), static_cast<const float*>(A), qsi, qsc, k,
                                          static_cast<float*>(Y), st);
}

rh_status rh_mode_product_bf16(int32_t order, const int64_t* dims, int32_t dtype, const void* X, int32_t k,
                               const double* A, float* Y, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const bool x3 = dtype == RH_F32_BF16X3;   // the split form with three exact pieces
  if (x3) dtype = RH_F32_BF16X2;
  RH_CHECK_ARG(bf16_form(dtype), "dtype must be RH_BF16, RH_BF16X2, RH_F32_BF16X2, RH_F32_BF16X3 or RH_FP8_E4M3");
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
  for (int q = 0; q < order; ++q) RH_CHECK_ARG(dims[q] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(X != nullptr && A != nullptr && Y != nullptr, "X, A and Y must be non-NULL");
  const ModeView v = mode_view(order, dims, 0);
  // I_0 % 8 != 0: the small-row kernel (I_0 <= 128, k <= 32); not for the three-piece form
  const bool small = !x3 && !ttm_tc_supported(v, k) && small_tc_supported(v, k);
  if (!ttm_tc_supported(v, k) && !small) {
    set_error("unsupported: the BF16 mode product needs I_0 % 8 == 0 and 1 <= k <= 64, or I_0 <= 128 and k <= 32");
    return RH_EUNSUPPORTED;
  }
  const size_t need = rh_mode_product_workspace_size(order, dims, dtype, 0, k);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  int32_t* err = ar.take<int32_t>(4);   // wait status: the first int32 of the workspace
  uint16_t* qa = ar.take<uint16_t>((size_t)128 * dims[0]);
  cudaStream_t st = (cudaStream_t)stream;
  RH_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  if (small) {
    SmallInput in{X, dtype};
    if (dtype == RH_FP8_E4M3) {
      const Fp8Layout f8 = fp8_layout(order, dims);
      in.ld = f8.ld;
      in.scales = reinterpret_cast<const float*>(static_cast<const uint8_t*>(X) + f8.scale_off);
    }
    return launch_ttm_small_tc(v, in, A, k, Y, err, st, SITE_OTHER);
  }
  if (dtype == RH_F32_BF16X2)
    return launch_ttm_tc_f32(v, k, static_cast<const float*>(X), A, qa, Y, err, st, x3 ? 3 : 2);
  if (dtype == RH_FP8_E4M3) {
    const Fp8Layout f8 = fp8_layout(order, dims);
    const uint8_t* x8 = static_cast<const uint8_t*>(X);
    return launch_ttm_tc_fp8(v, k, x8, reinterpret_cast<const float*>(x8 + f8.scale_off), f8.ld, A, qa, Y, err, st);
  }
  const uint16_t* p0 = static_cast<const uint16_t*>(X);
  const uint16_t* p1 = dtype == RH_BF16X2 ? p0 + v.I * v.M() : nullptr;
  return launch_ttm_tc(v, k, p0, p1, A, qa, Y, err, st);
}

size_t rh_mode_product_split_workspace_size(int32_t order, const int64_t* dims, int32_t mode, int32_t k) {
  if (order < 1 || order > RH_MAX_ORDER || dims == nullptr || mode < 0 || mode >= order || k < 1 || k > 64) return 0;
  for (int q = 0; q < order; ++q)
    if (dims[q] < 1) return 0;
  Arena ar(nullptr);
  ar.take<int32_t>(4);   // wait status, first (documented)
  ar.take<uint16_t>((size_t)128 * ((dims[mode] + 7) / 8 * 8));
  return ar.used;
}

rh_status rh_mode_product_split(int32_t order, const int64_t* dims, const float* X, int32_t mode, int32_t k,
                                const double* A, float* Y, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER && dims != nullptr, "bad order or dims");
  for (int q = 0; q < order; ++q) RH_CHECK_ARG(dims[q] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(mode >= 0 && mode < order, "mode out of range");
  RH_CHECK_ARG(k >= 1 && k <= 64, "k must be in [1, 64]");
  RH_CHECK_ARG(X != nullptr && A != nullptr && Y != nullptr, "X, A and Y must be non-NULL");
  const ModeView v = mode_view(order, dims, mode);
  const bool ok = mode == 0 ? ttm_tc_supported(v, k) : ttm_tc_strided_supported(v, k);
  if (!ok) {
    set_error("unsupported: the split mode product needs I_0 % 8 == 0 (mode 0) or the product of the earlier "
              "sizes to be a multiple of 128 (later modes)");
    return RH_EUNSUPPORTED;
  }
  const size_t need = rh_mode_product_split_workspace_size(order, dims, mode, k);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  int32_t* err = ar.take<int32_t>(4);
  uint16_t* qa = ar.take<uint16_t>((size_t)128 * ((dims[mode] + 7) / 8 * 8));
  cudaStream_t st = (cudaStream_t)stream;
  RH_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  return mode == 0 ? launch_ttm_tc_f32(v, k, X, A, qa, Y, err, st) : launch_ttm_tc_f32s(v, k, X, A, qa, Y, err, st);
}

size_t rh_left_svd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode) {
  if (check_tensor(order, dims, dtype) != RH_OK || mode < 0 || mode >= order || dims[mode] > RH_MAX_ELL) return 0;
  const ModeView v = mode_view(order, dims, mode);
  const TruncPlan tp = plan_trunc(v, (int)v.I);
  const size_t e = dtype == RH_F64 ? trunc_workspace_elems<double>(tp) * sizeof(double)
                                   : trunc_workspace_elems<float>(tp) * sizeof(float);
  return e + 256;
}

rh_status rh_left_svd(int32_t order, const int64_t* dims, int32_t dtype, const void* B, int32_t mode, double* U,
                      double* sv, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_status s = check_tensor(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(mode >= 0 && mode < order, "mode out of range");
  RH_CHECK_ARG(dims[mode] <= RH_MAX_ELL, "I_mode must be <= 64");
  RH_CHECK_ARG(B != nullptr && U != nullptr && sv != nullptr, "B, U and sv must be non-NULL");
  const size_t need = rh_left_svd_workspace_size(order, dims, dtype, mode);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  const ModeView v = mode_view(order, dims, mode);
  const TruncPlan tp = plan_trunc(v, (int)v.I);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == RH_F64)
    return launch_trunc_svd<double>(tp, static_cast<const double*>(B), static_cast<double*>(workspace), U, sv, st, 0, nullptr);
  return launch_trunc_svd<float>(tp, static_cast<const float*>(B), static_cast<float*>(workspace), U, sv, st, 0, nullptr);
}

rh_status rh_split_bf16x2(const float* X, int64_t n, uint16_t* out, void* stream) {
  clear_error();
  RH_CHECK_ARG(n >= 0, "n must be >= 0");
  RH_CHECK_ARG((X != nullptr && out != nullptr) || n == 0, "X and out must be non-NULL");
  if (n == 0) return RH_OK;
  return launch_split_bf16x2(X, n, out, out + n, (cudaStream_t)stream);
}

size_t rh_tall_skinny_r_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, int32_t mode) {
  if (check_tensor(order, dims, dtype) != RH_OK || mode < 0 || mode >= order || dims[mode] > RH_MAX_ELL) return 0;
  const TruncPlan tp = plan_trunc(mode_view(order, dims, mode), (int)dims[mode]);
  return (dtype == RH_F64 ? trunc_workspace_elems<double>(tp) * sizeof(double)
                          : trunc_workspace_elems<float>(tp) * sizeof(float)) + 256;
}

rh_status rh_tall_skinny_r(int32_t order, const int64_t* dims, int32_t dtype, const void* B, int32_t mode, double* R,
                           void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  rh_status s = check_tensor(order, dims, dtype);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(mode >= 0 && mode < order, "mode out of range");
  RH_CHECK_ARG(dims[mode] <= RH_MAX_ELL, "I_mode must be <= 64");
  RH_CHECK_ARG(B != nullptr && R != nullptr, "B and R must be non-NULL");
  const size_t need = rh_tall_skinny_r_workspace_size(order, dims, dtype, mode);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  const TruncPlan tp = plan_trunc(mode_view(order, dims, mode), (int)dims[mode]);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == RH_F64)
    return launch_tall_skinny_r<double>(tp, static_cast<const double*>(B), static_cast<double*>(workspace), R, st);
  return launch_tall_skinny_r<float>(tp, static_cast<const float*>(B), static_cast<float*>(workspace), R, st);
}

rh_status rh_cast_f64(const double* src, int64_t n, int32_t dtype, void* dst, void* stream) {
  clear_error();
  RH_CHECK_ARG(n >= 0 && (n == 0 || (src != nullptr && dst != nullptr)), "src and dst must be non-NULL");
  RH_CHECK_ARG(dtype == RH_F32 || dtype == RH_F64, "dtype must be RH_F32 or RH_F64");
  if (n == 0) return RH_OK;
  if (dtype == RH_F32) return launch_cast<float>(src, static_cast<float*>(dst), n, (cudaStream_t)stream, SITE_OTHER);
  return launch_cast<double>(src, static_cast<double*>(dst), n, (cudaStream_t)stream, SITE_OTHER);
}

rh_status rh_tucker_factor(int64_t I, int32_t ell, int32_t r, const double* Q, const double* Ub, double* A, double* Ur,
                           void* stream) {
  clear_error();
  RH_CHECK_ARG(I >= 1 && ell >= 1 && ell <= RH_MAX_ELL && r >= 1 && r <= ell, "need I >= 1, 1 <= r <= ell <= 64");
  RH_CHECK_ARG(Q != nullptr && Ub != nullptr && A != nullptr && Ur != nullptr, "Q, Ub, A and Ur must be non-NULL");
  return launch_factor_and_cast<double>(I, ell, r, Q, Ub, A, Ur, (cudaStream_t)stream);
}

size_t rh_orthonormalize_workspace_size(int64_t m, int32_t n) {
  if (m < 1 || n < 1 || n > RH_MAX_ELL || n > m) return 0;
  return sizeof(double) * orth_workspace_elems(m, n) + 256;
}

rh_status rh_orthonormalize(int64_t m, int32_t n, const double* Y, double* Q, int32_t* info, void* workspace,
                            size_t workspace_bytes, void* stream) {
  clear_error();
  RH_CHECK_ARG(m >= 1 && n >= 1 && n <= RH_MAX_ELL && n <= m, "need 1 <= n <= min(m, 64)");
  RH_CHECK_ARG(Y != nullptr && Q != nullptr, "Y and Q must be non-NULL");
  if (workspace == nullptr || workspace_bytes < rh_orthonormalize_workspace_size(m, n)) {
    set_error("workspace too small");
    return RH_ENOMEM;
  }
  return launch_orthonormalize(m, n, Y, Q, info, static_cast<double*>(workspace), (cudaStream_t)stream);
}

size_t rsthosvd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                               const rh_options* opts) {
  const rh_options o = opts_or_default(opts);
  Plan pl;
  if (make_plan(order, dims, dtype, ranks, o, pl) != RH_OK) return 0;
  Arena ar(nullptr);
  carve(ar, pl);
  return ar.used;
}

}  // extern "C"

namespace rh {
// A request whose whole R-STHOSVD program goes through emit (FP32 or FP64 data on the CUDA cores,
// truncated), so that it can be recorded for a grouped launch.
bool rsthosvd_groupable(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                        const rh_options* opts) {
  const rh_options o = opts_or_default(opts);
  Plan pl;
  if (make_plan(order, dims, dtype, ranks, o, pl) != RH_OK) return false;
  return (((dtype == RH_F32 || dtype == RH_F64) && pl.in_form < 0) || pl.steps[0].stc) && o.truncate;
}
}  // namespace rh

extern "C" {

rh_status rsthosvd(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const int32_t* ranks,
                   const rh_options* opts, double* const* factors, double* core, double* norms, int32_t* info,
                   void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const rh_options o = opts_or_default(opts);
  Plan pl;
  rh_status s = make_plan(order, dims, dtype, ranks, o, pl);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(X != nullptr && factors != nullptr && core != nullptr, "X, factors and core must be non-NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(factors[k] != nullptr, "every factors[n] must be non-NULL");
  Arena meas(nullptr);
  carve(meas, pl);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  const Bufs b = carve(ar, pl);
  cudaStream_t st = (cudaStream_t)stream;
  record_step(-1);
  if (info && (s = emit_memset(SITE_ENTRY, 0, info, sizeof(int32_t) * order, st)) != RH_OK) return s;
  if (pl.dtype == RH_F64) return run_rsthosvd<double>(pl, X, o, factors, core, norms, info, b, st);
  return run_rsthosvd<float>(pl, X, o, factors, core, norms, info, b, st);
}

size_t rhosvd_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                             const rh_options* opts) {
  const rh_options o = opts_or_default(opts);
  Plan pl;
  if (make_plan_hosvd(order, dims, dtype, ranks, o, pl) != RH_OK) return 0;
  Arena ar(nullptr);
  carve(ar, pl);
  return ar.used;
}

rh_status rhosvd(int32_t order, const int64_t* dims, int32_t dtype, const void* X, const int32_t* ranks,
                 const rh_options* opts, double* const* factors, double* core, double* norms, int32_t* info,
                 void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const rh_options o = opts_or_default(opts);
  Plan pl;
  rh_status s = make_plan_hosvd(order, dims, dtype, ranks, o, pl);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(X != nullptr && factors != nullptr && core != nullptr, "X, factors and core must be non-NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(factors[k] != nullptr, "every factors[n] must be non-NULL");
  Arena meas(nullptr);
  carve(meas, pl);
  if (workspace == nullptr || workspace_bytes < meas.used) {
    set_error("workspace too small: need " + std::to_string(meas.used) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  const Bufs b = carve(ar, pl);
  cudaStream_t st = (cudaStream_t)stream;
  if (info) RH_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int32_t) * order, st));
  if (pl.dtype == RH_F64)
    return run_rhosvd<double>(pl, dims, static_cast<const double*>(X), o, factors, core, norms, info, b, st);
  return run_rhosvd<float>(pl, dims, static_cast<const float*>(X), o, factors, core, norms, info, b, st);
}

size_t rsthosvd_host_workspace_size(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                                    const rh_options* opts) {
  const rh_options o = opts_or_default(opts);
  Plan pl;
  if (make_plan(order, dims, dtype, ranks, o, pl) != RH_OK) return 0;
  Arena ar(nullptr);
  int64_t n = 1, ncore = 1;
  for (int k = 0; k < order; ++k) n *= dims[k];
  ar.take<char>(input_bytes(order, dims, dtype));
  std::vector<int64_t> kout(order, 0);
  for (const Step& sp : pl.steps) kout[sp.mode] = sp.ko;
  for (int k = 0; k < order; ++k) {
    ar.take<double>((size_t)dims[k] * kout[k]);
    ncore *= kout[k];
  }
  ar.take<double>((size_t)ncore);
  ar.take<double>(2);
  ar.take<int32_t>((size_t)order);
  carve(ar, pl);
  return ar.used;
}

rh_status rsthosvd_host(int32_t order, const int64_t* dims, int32_t dtype, const void* X_host, const int32_t* ranks,
                        const rh_options* opts, double* const* factors_host, double* core_host, double* norms_host,
                        int32_t* info_host, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const rh_options o = opts_or_default(opts);
  Plan pl;
  rh_status s = make_plan(order, dims, dtype, ranks, o, pl);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(X_host != nullptr && factors_host != nullptr && core_host != nullptr,
               "X_host, factors_host and core_host must be non-NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(factors_host[k] != nullptr, "every factors_host[n] must be non-NULL");
  const size_t need = rsthosvd_host_workspace_size(order, dims, dtype, ranks, opts);
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  Arena ar(workspace);
  int64_t n = 1, ncore = 1;
  for (int k = 0; k < order; ++k) n *= dims[k];
  const size_t xbytes = input_bytes(order, dims, dtype);
  void* Xd = ar.take<char>(xbytes);
  std::vector<int64_t> kout(order, 0);
  for (const Step& sp : pl.steps) kout[sp.mode] = sp.ko;
  std::vector<double*> fd(order);
  for (int k = 0; k < order; ++k) {
    fd[k] = ar.take<double>((size_t)dims[k] * kout[k]);
    ncore *= kout[k];
  }
  double* cored = ar.take<double>((size_t)ncore);
  double* normsd = ar.take<double>(2);
  int32_t* infod = ar.take<int32_t>((size_t)order);
  const Bufs b = carve(ar, pl);
  cudaStream_t st = (cudaStream_t)stream;
  RH_CUDA_TRY(cudaMemcpyAsync(Xd, X_host, xbytes, cudaMemcpyHostToDevice, st));
  if ((s = emit_memset(SITE_ENTRY, 0, infod, sizeof(int32_t) * order, st)) != RH_OK) return s;
  if (pl.dtype == RH_F64)
    s = run_rsthosvd<double>(pl, Xd, o, fd.data(), cored, normsd, infod, b, st);
  else
    s = run_rsthosvd<float>(pl, Xd, o, fd.data(), cored, normsd, infod, b, st);
  if (s != RH_OK) return s;
  if (info_host) RH_CUDA_TRY(cudaMemcpyAsync(info_host, infod, sizeof(int32_t) * order, cudaMemcpyDeviceToHost, st));
  for (int k = 0; k < order; ++k)
    RH_CUDA_TRY(cudaMemcpyAsync(factors_host[k], fd[k], sizeof(double) * dims[k] * kout[k], cudaMemcpyDeviceToHost, st));
  RH_CUDA_TRY(cudaMemcpyAsync(core_host, cored, sizeof(double) * ncore, cudaMemcpyDeviceToHost, st));
  if (norms_host) RH_CUDA_TRY(cudaMemcpyAsync(norms_host, normsd, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  return RH_OK;
}

}  // extern "C"
