// rhosvd_sketch_static: the range-finder sketch Y = X_(mode) Omega_mode without any
// device allocation by the caller or the library.
//
// Who needs it: callers that may not call cudaMalloc themselves -- for example a plugin
// running inside a host framework that owns every byte of device memory through its own
// allocator and forbids private allocations, a latency-critical loop that cannot afford
// the implicit device synchronisation cudaMalloc may perform, or a process whose device
// memory budget is already fully reserved.  Such a caller still owns X, Y and norm2; only
// the scratch (the split-K partial sketches and partial norms) moves into a fixed
// file-scope device array that every GPU loading this library holds until the process
// exits.
//
// Limits and behaviour:
//   * the scratch array is kStaticScratchBytes = 16 MiB; the split count is reduced to fit,
//     and a request whose single-split scratch (I_mode * ell * sizeof(element) plus the
//     partial norms) still exceeds it is rejected with RH_EINVAL and a message;
//   * every call made outside stream capture looks up the array's device address with
//     cudaGetSymbolAddress (with the device current), so a device reset, which reloads the
//     module and may move the array, is picked up by the next call; a call made while its
//     stream is capturing uses the address of the last uncaptured call on that device, so the
//     first call on a device must come before any stream capture;
//   * every call on a device shares the one array and leaves the last call's contents in
//     it; each call overwrites every scratch element it reads, so nothing needs clearing,
//     but calls that overlap on the GPU (different streams, no ordering) race on the array.
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.cuh"

namespace rh {
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_sketch_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sketch_scratch on the current device: looked up on every call outside
// stream capture (the module, and with it the array, is reloaded after a device reset); inside a
// capture the address of the last uncaptured call on this device is used.
rh_status scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  RH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("rhosvd_sketch_static: device ordinal beyond the supported 64 devices");
    return RH_EUNSUPPORTED;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RH_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    RH_CUDA_TRY(cudaGetSymbolAddress(&p, g_sketch_scratch));
    g_scratch_addr[dev] = p;
  } else if (g_scratch_addr[dev] == nullptr) {
    set_error("rhosvd_sketch_static: the first call on a device must come before any stream capture");
    return RH_EINVAL;
  }
  *out = g_scratch_addr[dev];
  return RH_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// The plan of plan_sketch with the number of splits capped so that the partial sketches
// (S x ell x I elements) and partial norms (S x gx doubles) fit the static array.
rh_status plan_static(const ModeView& v, int ell, size_t esz, SketchPlan& pl) {
  pl = plan_sketch(v, ell);
  const size_t per_split = (size_t)ell * (size_t)v.I * esz + (size_t)pl.gx * sizeof(double);
  const size_t usable = kStaticScratchBytes - 512;   // two 256-byte alignment gaps
  if (per_split > usable) {
    set_error("rhosvd_sketch_static: I_mode * ell * element size = " + std::to_string(per_split) +
              " bytes of scratch exceeds the 16 MiB static scratch array; use rhosvd_sketch with a workspace");
    return RH_EINVAL;
  }
  const int64_t smax = (int64_t)(usable / per_split);
  if (pl.S > smax) {
    const int64_t M = v.M();
    pl.chunk = ceil_div(ceil_div(M, smax), 32) * 32;
    pl.S = (int)ceil_div(M, pl.chunk);
  }
  if (align256(pl.part_elems() * esz) + align256(pl.norm_elems() * sizeof(double)) > kStaticScratchBytes) {
    set_error("rhosvd_sketch_static: internal scratch plan exceeds the static array");
    return RH_EINVAL;
  }
  return RH_OK;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" rh_status rhosvd_sketch_static(int32_t order, const int64_t* dims, int32_t dtype, const void* X,
                                          int32_t mode, int32_t ell, uint64_t seed, int32_t tensor_id, double* Y,
                                          double* norm2, void* stream) {
  clear_error();
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER, "order must be in [1, 8]");
  RH_CHECK_ARG(dims != nullptr, "dims is NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(dims[k] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(dtype == RH_F64 || dtype == RH_F32, "dtype must be RH_F64 or RH_F32");
  RH_CHECK_ARG(mode >= 0 && mode < order && mode < 16, "mode out of range");
  RH_CHECK_ARG(ell >= 1 && ell <= RH_MAX_ELL, "ell must be in [1, 64]");
  RH_CHECK_ARG(tensor_id >= 0 && tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(X != nullptr && Y != nullptr, "X and Y must be non-NULL");
  const size_t esz = dtype == RH_F64 ? sizeof(double) : sizeof(float);
  SketchPlan pl;
  rh_status s = plan_static(mode_view(order, dims, mode), ell, esz, pl);
  if (s != RH_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  if ((s = scratch_address(st, &base)) != RH_OK) return s;
  char* b = static_cast<char*>(base);
  void* part = b;
  double* part_norm = reinterpret_cast<double*>(b + align256(pl.part_elems() * esz));
  const uint32_t sid = ((uint32_t)tensor_id << 4) | (uint32_t)mode;
  if (dtype == RH_F64) {
    if ((s = launch_sketch<double>(pl, static_cast<const double*>(X), seed, sid, static_cast<double*>(part), part_norm,
                                   st)) != RH_OK)
      return s;
    return launch_sketch_reduce<double>(pl, static_cast<const double*>(part), part_norm, Y, norm2, st);
  }
  if ((s = launch_sketch<float>(pl, static_cast<const float*>(X), seed, sid, static_cast<float*>(part), part_norm,
                                st)) != RH_OK)
    return s;
  return launch_sketch_reduce<float>(pl, static_cast<const float*>(part), part_norm, Y, norm2, st);
}
