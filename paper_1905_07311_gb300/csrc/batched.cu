// Batched R-STHOSVD (Alg. 3 on many independent tensors of different orders and sizes in one call).
//
// Small tensors leave most of the GPU idle in a single decomposition (its sketches, QRs and small
// SVDs are short, few-CTA launches), so the batch runs concurrently: the caller's stream is forked
// (an event) into K internal streams, the tensors are assigned largest first to the least loaded
// stream (load = tensor elements), each stream runs its tensors one after another in its own
// workspace slice (sized for the largest tensor), and the streams are joined back into the caller's
// stream.  Nothing synchronises the host, so the whole call can be captured in a CUDA graph.
// Tensor i uses the Omega stream of tensor_id = opts->tensor_id + i.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

namespace rh {
namespace {

constexpr int kMaxBatchStreams = 32;

std::mutex g_bs_mu;
cudaStream_t g_bs[64][kMaxBatchStreams] = {};

rh_status batch_streams(int k, cudaStream_t* out) {
  int dev = 0;
  RH_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device index out of range");
    return RH_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_bs_mu);
  for (int i = 0; i < k; ++i) {
    if (!g_bs[dev][i]) RH_CUDA_TRY(cudaStreamCreateWithFlags(&g_bs[dev][i], cudaStreamNonBlocking));
    out[i] = g_bs[dev][i];
  }
  return RH_OK;
}

struct BatchLayout {
  std::vector<int64_t> dim_off, ws;
  std::vector<int> stream_of;
  size_t slice = 0;
};

rh_status batch_layout(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                       const int32_t* ranks, const rh_options* opts, int k, BatchLayout& bl) {
  RH_CHECK_ARG(count >= 1, "count must be >= 1");
  RH_CHECK_ARG(orders != nullptr && dims != nullptr && ranks != nullptr, "orders, dims and ranks must be non-NULL");
  RH_CHECK_ARG(k >= 1 && k <= kMaxBatchStreams, "streams must be in [1, 32]");
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  RH_CHECK_ARG(o.rho[0] < 0, "batched calls use the default processing order (opts->rho[0] < 0)");
  RH_CHECK_ARG(o.tensor_id >= 0 && (int64_t)o.tensor_id + count <= (int64_t(1) << 28),
               "tensor_id + count must stay below 2^28");
  bl.dim_off.assign(count + 1, 0);
  bl.ws.assign(count, 0);
  for (int i = 0; i < count; ++i) {
    RH_CHECK_ARG(orders[i] >= 1 && orders[i] <= RH_MAX_ORDER, "every order must be in [1, 8]");
    bl.dim_off[i + 1] = bl.dim_off[i] + orders[i];
  }
  std::vector<int64_t> load(count, 1);
  for (int i = 0; i < count; ++i) {
    rh_options oi = o;
    oi.tensor_id = o.tensor_id + i;
    const size_t w = rsthosvd_workspace_size(orders[i], dims + bl.dim_off[i], dtype, ranks + bl.dim_off[i], &oi);
    if (w == 0) {
      const std::string why = rh_last_error();
      set_error("tensor " + std::to_string(i) + ": " + (why.empty() ? "invalid request" : why));
      return RH_EINVAL;
    }
    bl.ws[i] = (int64_t)w;
    bl.slice = std::max(bl.slice, (w + 255) & ~size_t(255));
    for (int n = 0; n < orders[i]; ++n) load[i] *= dims[bl.dim_off[i] + n];
  }
  // largest first onto the least loaded stream
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return load[a] > load[b]; });
  std::vector<int64_t> acc(k, 0);
  bl.stream_of.assign(count, 0);
  for (int i : idx) {
    const int s = (int)(std::min_element(acc.begin(), acc.end()) - acc.begin());
    bl.stream_of[i] = s;
    acc[s] += load[i];
  }
  return RH_OK;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" {

size_t rsthosvd_batched_workspace_size(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                                       const int32_t* ranks, const rh_options* opts, int32_t streams) {
  BatchLayout bl;
  const int k = streams > 0 ? std::min<int>(streams, count) : std::min<int>(8, count);
  if (batch_layout(count, orders, dims, dtype, ranks, opts, std::max(k, 1), bl) != RH_OK) return 0;
  return bl.slice * (size_t)std::max(k, 1);
}

rh_status rsthosvd_batched(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                           const void* const* X, const int32_t* ranks, const rh_options* opts,
                           double* const* factors, double* const* cores, double* norms, int32_t* info,
                           int32_t streams, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  const int k = std::max(1, streams > 0 ? std::min<int>(streams, count) : std::min<int>(8, count));
  BatchLayout bl;
  rh_status s = batch_layout(count, orders, dims, dtype, ranks, opts, k, bl);
  if (s != RH_OK) return s;
  RH_CHECK_ARG(X != nullptr && factors != nullptr && cores != nullptr, "X, factors and cores must be non-NULL");
  for (int i = 0; i < count; ++i) RH_CHECK_ARG(X[i] != nullptr && cores[i] != nullptr, "null tensor or core");
  const size_t need = bl.slice * (size_t)k;
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  cudaStream_t user = (cudaStream_t)stream;
  cudaStream_t st[kMaxBatchStreams];
  if ((s = batch_streams(k, st)) != RH_OK) return s;
  cudaEvent_t fork, join[kMaxBatchStreams];
  RH_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (int i = 0; i < k; ++i) RH_CUDA_TRY(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
  RH_CUDA_TRY(cudaEventRecord(fork, user));
  for (int i = 0; i < k; ++i) RH_CUDA_TRY(cudaStreamWaitEvent(st[i], fork, 0));
  rh_status first_err = RH_OK;
  std::string msg;
  for (int i = 0; i < count && first_err == RH_OK; ++i) {
    const int sidx = bl.stream_of[i];
    rh_options oi = o;
    oi.tensor_id = o.tensor_id + i;
    char* slice = static_cast<char*>(workspace) + bl.slice * (size_t)sidx;
    const rh_status r = rsthosvd(orders[i], dims + bl.dim_off[i], dtype, X[i], ranks + bl.dim_off[i], &oi,
                                 factors + bl.dim_off[i], cores[i], norms ? norms + 2 * i : nullptr,
                                 info ? info + bl.dim_off[i] : nullptr, slice, bl.slice, st[sidx]);
    if (r != RH_OK) {
      first_err = r;
      msg = "tensor " + std::to_string(i) + ": " + rh_last_error();
    }
  }
  // join every stream back into the caller's stream, also after an error
  for (int i = 0; i < k; ++i) {
    cudaEventRecord(join[i], st[i]);
    cudaStreamWaitEvent(user, join[i], 0);
  }
  cudaEventDestroy(fork);
  for (int i = 0; i < k; ++i) cudaEventDestroy(join[i]);
  if (first_err != RH_OK) {
    set_error(msg);
    return first_err;
  }
  RH_CUDA_TRY(cudaGetLastError());
  return RH_OK;
}

}  // extern "C"
