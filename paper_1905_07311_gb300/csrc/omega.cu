// rh_omega: materialise a block of Omega (test / inspection entry point), plus the
// thread-local error state and the version string of the C ABI.
#include <atomic>
#include <string>

#include "common.cuh"
#include "grouped.cuh"
#include "philox.cuh"

namespace rh {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

static std::atomic<uint64_t> g_launches{0};
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  note_direct_launch();
}

// out[i + nrows * c] = Omega(row0 + i, c); one thread per (row, group of 4 columns).
__global__ void omega_kernel(uint32_t k0, uint32_t k1, uint32_t sid, int64_t row0, int64_t nrows, int ell,
                             float* __restrict__ out) {
  const int nq = (ell + 3) / 4;
  const int64_t total = nrows * nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % nrows;
    const int q = (int)(t / nrows);
    const float4 v = rng::omega4(k0, k1, sid, row0 + i, (uint32_t)q);
    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * q + j;
      if (c < ell) out[i + nrows * c] = vv[j];
    }
  }
}

}  // namespace rh

extern "C" {

const char* rh_version(void) { return "rhosvd-gb300 0.1 (sm_103a)"; }

const char* rh_last_error(void) { return rh::g_last_error.c_str(); }

uint64_t rh_kernel_launches(void) { return rh::g_launches.load(std::memory_order_relaxed); }

void rh_options_default(rh_options* o) {
  if (!o) return;
  o->seed = 0;
  o->tensor_id = 0;
  o->p = 5;
  for (int i = 0; i < RH_MAX_ORDER; ++i) o->rho[i] = -1;
  o->clamp = 0;
  o->truncate = 1;
  o->svd_route = 0;
  o->power_iters = 0;
  o->select = RH_SELECT_SRRQR;
  o->omega_prec = RH_F32;
}

rh_status rh_omega(uint64_t seed, int32_t tensor_id, int32_t mode, int64_t row0, int64_t nrows, int32_t ell,
                   float* out, void* stream) {
  rh::clear_error();
  RH_CHECK_ARG(nrows >= 0 && row0 >= 0, "nrows and row0 must be non-negative");
  RH_CHECK_ARG(ell >= 1 && ell <= 4096, "ell must be in [1, 4096]");
  RH_CHECK_ARG(mode >= 0 && mode < 16, "mode must be in [0, 16)");
  RH_CHECK_ARG(tensor_id >= 0 && tensor_id < (1 << 28), "tensor_id must be in [0, 2^28)");
  RH_CHECK_ARG(out != nullptr || nrows == 0, "out is NULL");
  if (nrows == 0) return RH_OK;
  const int64_t total = nrows * ((ell + 3) / 4);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>(rh::ceil_div(total, threads), 65535LL * 8);
  rh::omega_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
      (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), ((uint32_t)tensor_id << 4) | (uint32_t)mode, row0,
      nrows, ell, out);
  RH_LAUNCH_CHECK();
  return RH_OK;
}

}  // extern "C"
