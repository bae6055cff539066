// Shared host/device helpers of the library: status plumbing, workspace carving,
// launch checks.  No arithmetic of the method lives here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>

#include "../../include/rhosvd.h"

namespace rh {

// Thread-local message of the last failure (rh_last_error).
void set_error(const std::string& msg);
void clear_error();

struct Status {
  rh_status code = RH_OK;
  bool ok() const { return code == RH_OK; }
};

#define RH_CHECK_ARG(cond, msg)                      \
  do {                                               \
    if (!(cond)) {                                   \
      ::rh::set_error(std::string("invalid argument: ") + (msg)); \
      return RH_EINVAL;                              \
    }                                                \
  } while (0)

#define RH_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::rh::set_error(std::string("CUDA error ") + cudaGetErrorString(_e) + " at " +  \
                      __FILE__ + ":" + std::to_string(__LINE__));                      \
      return RH_ECUDA;                                                                 \
    }                                                                                  \
  } while (0)

// Every kernel launch of the library goes through RH_LAUNCH_CHECK, which also counts it
// (rh_kernel_launches() in the C ABI).
void count_launch();
#define RH_LAUNCH_CHECK()   \
  do {                      \
    ::rh::count_launch();   \
    RH_CUDA_TRY(cudaGetLastError()); \
  } while (0)

// Bump allocator over the caller's workspace.  With base == nullptr it only
// measures, so the *_workspace_size queries run the same carving code as the calls.
struct Arena {
  char* base = nullptr;
  size_t used = 0;
  explicit Arena(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + ((count * sizeof(T) + 255) & ~size_t(255));
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

// Wait-timeout probe (profile.cu): 1 for the tensor-core launch that rh_test_wait_probe armed,
// else 0; every tensor-core launch calls it once.
int tc_probe_next();

// Per-launch timing (profile.cu): a scope records an event before and after the kernels
// it encloses when profiling is on.  kind: 0 sketch, 1 mode product, 2 QR of the sketch,
// 3 truncation SVD; tag: the step of the algorithm (0 = first processed mode).
enum { PROF_SKETCH = 0, PROF_TTM = 1, PROF_ORTH = 2, PROF_TRUNC = 3, PROF_TTM_CORE = 4, PROF_JACOBI = 5, PROF_POWER = 6,
       PROF_SP_TABLE = 7, PROF_SP_SORT = 8, PROF_SP_ITEMS = 9, PROF_SP_REDUCE = 10 };
class ProfileScope {
 public:
  ProfileScope(int kind, int tag, cudaStream_t st);
  ~ProfileScope();
  ProfileScope(const ProfileScope&) = delete;
  ProfileScope& operator=(const ProfileScope&) = delete;

 private:
  cudaStream_t st_;
  int idx_ = -1;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// SM count of the device current at the first call (initialised once, thread-safe); 152 (GB300)
// when no device answers, as in workspace queries on a machine without a GPU.
// Launch-shape knobs of the small-tensor kernels (tuning.cu; defaults in tuning_table.inc).
enum TuneKey : int {
#define RH_TUNE(key, name, value) key,
#include "tuning_table.inc"
#undef RH_TUNE
  TUNE_COUNT
};
int32_t tune(TuneKey k);

inline int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        v <= 0)
      v = 152;
    return v;
  }();
  return n;
}

// 3-D view (L, I, R) of mode n of a column-major tensor: L = prod_{k<n} dims,
// I = dims[n], R = prod_{k>n} dims.  Element (l, i, r) sits at l + L*(i + I*r); the
// Kolda column index of X_(n) for (l, r) is p = l + L*r.
struct ModeView {
  int64_t L, I, R;
  int64_t M() const { return L * R; }
};

inline ModeView mode_view(int order, const int64_t* dims, int n) {
  ModeView v{1, dims[n], 1};
  for (int k = 0; k < n; ++k) v.L *= dims[k];
  for (int k = n + 1; k < order; ++k) v.R *= dims[k];
  return v;
}

inline int ell_pad_of(int ell) { return ell <= 32 ? 32 : 64; }

// Division of 32-bit unsigned integers by an invariant divisor d >= 1 with one multiply-high and
// shifts (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> 1)) >> (l - 1) for l >= 1, and n / 1 = n.
struct FastDiv {
  uint32_t d = 1, m = 0;
  int l = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t dv) : d(dv) {
    while ((uint64_t(1) << l) < d) ++l;
    m = l ? (uint32_t)((((uint64_t)1 << 32) * ((uint64_t(1) << l) - d)) / d + 1) : 0u;
  }
  __host__ __device__ uint32_t div(uint32_t n) const {
    if (l == 0) return n;
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
    return (t + ((n - t) >> 1)) >> (l - 1);
  }
};

// Where a truncated core G <- U_r^T B (B: ell x M, column p = Kolda column of the unfolding of
// mode n) stores element (c, p): the next mode m first, then the other modes in increasing order,
// with the new index c of mode n (ko values) in its place.  With p's digits in increasing mode
// order, i_m = (p / S) % I is mode m's digit and r = (p % S) + S (p / (S I)) the rest;
//   out(c, p) = i_m + I ((r % Ln) + Ln (c + ko (r / Ln))) = base(p) + c I Ln.
// S = I = 1 is the usual column-major order with c inserted after the modes before n (Ln of them).
// For M < 2^31 the divisions use FastDiv (make() prepares them).
struct CoreOut {
  int64_t S = 1, I = 1, Ln = 1;
  bool fast = false;
  FastDiv fS, fI, fLn;
  static CoreOut make(int64_t S, int64_t I, int64_t Ln, int64_t M) {
    CoreOut c;
    c.S = S;
    c.I = I;
    c.Ln = Ln;
    c.fast = M < (int64_t(1) << 31) && S < (int64_t(1) << 31) && I < (int64_t(1) << 31) && Ln < (int64_t(1) << 31);
    if (c.fast) {
      c.fS = FastDiv((uint32_t)S);
      c.fI = FastDiv((uint32_t)I);
      c.fLn = FastDiv((uint32_t)Ln);
    }
    return c;
  }
  __host__ __device__ int64_t base(int64_t p, int ko) const {
    if (fast) {
      const uint32_t pp = (uint32_t)p;
      const uint32_t q = fS.div(pp), q2 = fI.div(q);
      const uint32_t im = q - q2 * (uint32_t)I;
      const uint32_t r = (pp - q * (uint32_t)S) + (uint32_t)S * q2;
      const uint32_t rq = fLn.div(r);
      return (int64_t)im + I * ((int64_t)(r - rq * (uint32_t)Ln) + Ln * (int64_t)ko * rq);
    }
    const int64_t q = p / S, im = q % I;
    const int64_t r = (p - q * S) + S * (q / I);
    const int64_t rq = r / Ln;
    return im + I * ((r - rq * Ln) + Ln * (int64_t)ko * rq);
  }
  __host__ __device__ int64_t cstride() const { return I * Ln; }
  __host__ __device__ bool plain() const { return S == 1 && I == 1 && Ln == 1; }
};

// Storage of an RH_FP8_E4M3 tensor: E4M3 bytes column-major with the mode-1 fibres at a stride
// of ld = I_1 rounded up to 16 (zero padding), i.e. ld x M bytes (M = prod of the other sizes),
// then, from the next 16-byte boundary, one FP32 scale per 128 consecutive bytes of that array:
// element (i, p) is e4m3[i + ld p] * scales[(i + ld p) / 128].
struct Fp8Layout {
  int64_t ld = 0;
  size_t scale_off = 0, nscales = 0, bytes = 0;
};
inline Fp8Layout fp8_layout(int order, const int64_t* dims) {
  Fp8Layout f;
  int64_t m = 1;
  for (int k = 1; k < order; ++k) m *= dims[k];
  f.ld = (dims[0] + 15) / 16 * 16;
  const size_t data = (size_t)f.ld * (size_t)m;
  f.scale_off = (data + 15) / 16 * 16;
  f.nscales = (data + 127) / 128;
  f.bytes = f.scale_off + 4 * f.nscales;
  return f;
}


// ---- launches: direct, or recorded for a grouped launch ---------------------------------------
// A kernel that can run grouped is an Op: a plain argument struct Args, a device body(Grid, Args)
// written against the block coordinates in Grid (not blockIdx / gridDim), and its block size
// kThreads (and kMinBlocks for the launch bounds).  single_kernel<Op> is the ordinary launch (the
// hardware grid); group_kernel<Op> runs the same body for many independent problems in one launch:
// the blocks of problem t are [start[t], start[t+1]), read as t's own gx x gy grid (x fastest),
// and get t's Args, so each problem computes exactly what its own launch would.
struct Grid {
  uint32_t bx, by, gx, gy;
};

#ifdef __CUDACC__
__device__ __forceinline__ Grid hw_grid() { return Grid{blockIdx.x, blockIdx.y, gridDim.x, gridDim.y}; }

// The problem whose block range holds this block: the t with start[t] <= blockIdx.x < start[t+1]
// (start[0] = 0 and start[n] = the launch's block count, so empty ranges are never chosen).
__device__ __forceinline__ int group_find(const int32_t* __restrict__ start, int n) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Programmatic dependent launch.  Op kernels are launched with programmatic stream serialization,
// so a grid may start while the grid before it in the stream is still running; the first thing
// every Op kernel does is wait for that grid to complete and its memory to be visible
// (griddepcontrol.wait, a no-op when nothing is pending), and only then does it let the next grid
// launch.  The next grid's blocks thus get resident (and past their launch latency) while this one
// runs, and no Op touches memory before its predecessor has finished.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class Op>
__global__ void __launch_bounds__(Op::kThreads, Op::kMinBlocks) single_kernel(const typename Op::Args a) {
  pdl_enter();
  Op::body(hw_grid(), a);
}

template <class Op>
__global__ void __launch_bounds__(Op::kThreads, Op::kMinBlocks)
    group_kernel(const typename Op::Args* __restrict__ args, const int32_t* __restrict__ start,
                 const uint2* __restrict__ gdim, int n) {
  pdl_enter();
  const int t = group_find(start, n);
  const uint2 d = gdim[t];
  const uint32_t lb = blockIdx.x - (uint32_t)start[t];
  const typename Op::Args a = args[t];
  Op::body(Grid{lb % d.x, lb / d.x, d.x, d.y}, a);
}
#endif

struct KernelRef {
  const void* single;   // single_kernel<Op>
  const void* group;    // group_kernel<Op>
  uint32_t args_bytes;
  int threads;
  std::atomic<size_t> smem_single{0}, smem_group{0};   // dynamic shared memory opted in so far (host)
};

#ifdef __CUDACC__
template <class Op>
KernelRef* kref() {
  static KernelRef r{reinterpret_cast<const void*>(&single_kernel<Op>), reinterpret_cast<const void*>(&group_kernel<Op>),
                     (uint32_t)sizeof(typename Op::Args), Op::kThreads};
  return &r;
}
#endif

// Launch sites of the per-tensor R-STHOSVD program, numbered in the order one step runs them.  A
// recorded program must visit (step, site, sub) in increasing order; launches of different
// problems with the same key and kernel become one grouped launch (grouped.cu).
enum LaunchSite : int {
  SITE_ENTRY = 0,
  // a subspace-iteration step (its own step key, before the QR sites it reuses)
  SITE_POWER_CAST = 1,
  SITE_POWER_TTM,
  SITE_POWER_ZERO,
  SITE_POWER_TSQR,          // sub = level of the reduction tree
  SITE_POWER_TRSM,
  SITE_POWER_GRAM,          // + 1: its reduce
  SITE_POWER_GRAM_REDUCE,
  SITE_POWER_CHOL,
  SITE_POWER_TRSM2,
  SITE_POWER_SKETCH = 12,
  SITE_POWER_SKETCH_REDUCE,
  SITE_SKETCH = 10,
  SITE_SKETCH_REDUCE,
  SITE_ORTH_ZERO = 20,
  SITE_ORTH_GRAM,
  SITE_ORTH_GRAM_REDUCE,
  SITE_ORTH_CHOL,
  SITE_ORTH_TRSM,
  SITE_ORTH_CAST,
  SITE_ORTH_GRAM2,
  SITE_ORTH_GRAM2_REDUCE,
  SITE_ORTH_CHOL2,
  SITE_ORTH_TRSM2,
  SITE_ORTH_CAST2,
  SITE_ORTH_HOUSEHOLDER,
  SITE_ORTH_SIGN,
  SITE_CAST_Q = 40,
  SITE_MODE_PRODUCT = 45,
  SITE_TRUNC_ZERO = 50,
  SITE_TRUNC_GRAM,
  SITE_TRUNC_GRAM_REDUCE,
  SITE_TRUNC_PCHOL,
  SITE_TRUNC_JACOBI,
  SITE_TRUNC_DECIDE,
  SITE_TRUNC_GRAM_DF,
  SITE_TRUNC_GRAM_DF_REDUCE,
  SITE_TRUNC_PCHOL2,
  SITE_TRUNC_JACOBI2,
  SITE_TRUNC_TSQR,          // sub = level of the reduction tree
  SITE_TRUNC_PIVQR,
  SITE_TRUNC_JACOBI_SVD,
  SITE_FACTOR = 70,
  SITE_FACTOR_SIGN,
  SITE_CORE = 80,
  SITE_INFO = 85,           // info bits of the mode (and the wait status of its tensor-core kernels)
  SITE_FINAL = 90,
  SITE_OTHER = 1000         // launches of entry points that never run grouped
};

// Launch of an Op kernel (single_kernel or group_kernel) with programmatic stream serialization
// (pdl_enter); RHOSVD_PDL=0 in the environment launches them in plain stream order instead.
rh_status launch_op_kernel(const void* fn, dim3 grid, int threads, size_t smem, cudaStream_t st, void** params);

// Direct launch (the caller's stream), or, while this thread records a tape, an entry of it.
rh_status emit_raw(KernelRef* k, int site, int sub, dim3 grid, size_t smem, cudaStream_t st, const void* args);
#ifdef __CUDACC__
template <class Op>
rh_status emit(int site, int sub, dim3 grid, size_t smem, cudaStream_t st, const typename Op::Args& a) {
  return emit_raw(kref<Op>(), site, sub, grid, smem, st, &a);
}
#endif
// Zero fill of bytes at p (cudaMemsetAsync, or a recorded fill).
rh_status emit_memset(int site, int sub, void* p, size_t bytes, cudaStream_t st);
bool recording();
void record_step(int step);
// Step keys of a recorded program: mode step j of the algorithm starts key kStepStride j, its
// subspace-iteration steps take the keys that follow (at most kStepStride - 1 of them).
constexpr int kStepStride = 32;

}  // namespace rh
