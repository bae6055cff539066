// Batched R-STHOSVD (Alg. 3 on many independent tensors of different orders and sizes in one call).
//
// Small tensors leave most of the GPU idle in a single decomposition (its sketches, QRs and small
// SVDs are short, few-CTA launches).  Two engines:
//  * grouped (streams = 0, FP32 / FP64 truncated requests): every tensor's program is recorded
//    (grouped.cu) and the same stage of all tensors runs as one launch, about 30 launches per mode
//    for the whole batch; each tensor works in its own workspace slice and computes exactly what
//    its own rsthosvd call would.
//  * streams (streams >= 1, or requests the grouped engine does not cover): the caller's stream is
//    forked (an event) into K internal streams, the tensors are assigned largest first to the least
//    loaded stream (load = tensor elements), each stream runs its tensors one after another in its
//    own workspace slice (sized for the largest tensor), and the streams are joined back.
// Nothing synchronises the host, so either call can be captured in a CUDA graph.
// Tensor i uses the Omega stream of tensor_id = opts->tensor_id + i.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "grouped.cuh"

namespace rh {

bool rsthosvd_groupable(int32_t order, const int64_t* dims, int32_t dtype, const int32_t* ranks,
                        const rh_options* opts);

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
  bool groupable = true;   // every request runs on the grouped engine
  size_t slices_total = 0; // grouped engine: sum of the per-tensor slices (256-byte aligned)
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

rh_status batch_layout(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                       const int32_t* ranks, const rh_options* opts, int k, BatchLayout& bl) {
  RH_CHECK_ARG(count >= 1, "count must be >= 1");
  RH_CHECK_ARG(orders != nullptr && dims != nullptr && ranks != nullptr, "orders, dims and ranks must be non-NULL");
  RH_CHECK_ARG(k >= 1 && k <= kMaxBatchStreams, "streams must be in [1, 32]");
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  // opts->rho: the default order, or an order whose first order_i entries every tensor i takes
  // (make_plan checks that they are a permutation of 0 .. order_i - 1)
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
    bl.slices_total += align256(w);
    if (!rsthosvd_groupable(orders[i], dims + bl.dim_off[i], dtype, ranks + bl.dim_off[i], &oi)) bl.groupable = false;
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

// Records tensor i's rsthosvd program (its workspace slice at ws + the slices before it) for every
// tensor and merges the programs into grouped launches.
rh_status record_batch(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype, const void* const* X,
                       const int32_t* ranks, const rh_options& o, double* const* factors, double* const* cores,
                       double* norms, int32_t* info, char* ws, const BatchLayout& bl, GroupedProgram& gp) {
  std::vector<Tape> tapes(count);
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    rh_options oi = o;
    oi.tensor_id = o.tensor_id + i;
    rh_status r;
    {
      TapeScope rec(&tapes[i]);
      r = rsthosvd(orders[i], dims + bl.dim_off[i], dtype, X[i], ranks + bl.dim_off[i], &oi, factors + bl.dim_off[i],
                   cores[i], norms ? norms + 2 * i : nullptr, info ? info + bl.dim_off[i] : nullptr, ws + off,
                   (size_t)bl.ws[i], nullptr);
    }
    if (r != RH_OK) {
      set_error("tensor " + std::to_string(i) + ": " + rh_last_error());
      return r;
    }
    off += align256((size_t)bl.ws[i]);
  }
  return build_grouped(tapes, gp);
}

// Launch tables of the grouped engine for these requests (the pointers do not change their size).
rh_status grouped_table_bytes(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                              const int32_t* ranks, const rh_options& o, const BatchLayout& bl, size_t* bytes) {
  int64_t nd = bl.dim_off[count];
  char* fake = reinterpret_cast<char*>(uintptr_t(1) << 20);   // never dereferenced: recording only
  std::vector<const void*> X(count, fake);
  std::vector<double*> f((size_t)nd, reinterpret_cast<double*>(fake));
  std::vector<double*> c(count, reinterpret_cast<double*>(fake));
  GroupedProgram gp;
  rh_status s = record_batch(count, orders, dims, dtype, X.data(), ranks, o, f.data(), c.data(),
                             reinterpret_cast<double*>(fake), reinterpret_cast<int32_t*>(fake), fake, bl, gp);
  if (s != RH_OK) return s;
  *bytes = align256(gp.blob.size());
  return RH_OK;
}

}  // namespace
}  // namespace rh

struct rh_batched_plan_s {
  rh::GroupedProgram gp;
  void* tables = nullptr;
};

using namespace rh;

extern "C" {

size_t rsthosvd_batched_workspace_size(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                                       const int32_t* ranks, const rh_options* opts, int32_t streams) {
  BatchLayout bl;
  const int k = streams > 0 ? std::min<int>(streams, count) : std::min<int>(8, count);
  if (batch_layout(count, orders, dims, dtype, ranks, opts, std::max(k, 1), bl) != RH_OK) return 0;
  if (streams == 0 && bl.groupable) {
    rh_options o;
    rh_options_default(&o);
    if (opts) o = *opts;
    size_t tb = 0;
    if (grouped_table_bytes(count, orders, dims, dtype, ranks, o, bl, &tb) != RH_OK) return 0;
    return bl.slices_total + tb;
  }
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
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  cudaStream_t user = (cudaStream_t)stream;
  if (streams == 0 && bl.groupable) {
    GroupedProgram gp;
    if (workspace == nullptr || workspace_bytes < bl.slices_total) {
      set_error("workspace too small: need " + std::to_string(bl.slices_total) + " bytes and the launch tables");
      return RH_ENOMEM;
    }
    if ((s = record_batch(count, orders, dims, dtype, X, ranks, o, factors, cores, norms, info,
                          static_cast<char*>(workspace), bl, gp)) != RH_OK)
      return s;
    const size_t need = bl.slices_total + align256(gp.blob.size());
    if (workspace_bytes < need) {
      set_error("workspace too small: need " + std::to_string(need) + " bytes");
      return RH_ENOMEM;
    }
    void* tables = static_cast<char*>(workspace) + bl.slices_total;
    if ((s = upload_tables_async(gp, tables, user)) != RH_OK) return s;
    return run_grouped(gp, tables, user);
  }
  const size_t need = bl.slice * (size_t)k;
  if (workspace == nullptr || workspace_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes");
    return RH_ENOMEM;
  }
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

rh_status rsthosvd_batched_plan_create(int32_t count, const int32_t* orders, const int64_t* dims, int32_t dtype,
                                      const void* const* X, const int32_t* ranks, const rh_options* opts,
                                      double* const* factors, double* const* cores, double* norms, int32_t* info,
                                      void* workspace, size_t workspace_bytes, rh_batched_plan* plan) {
  clear_error();
  RH_CHECK_ARG(plan != nullptr, "plan must be non-NULL");
  *plan = nullptr;
  BatchLayout bl;
  rh_status s = batch_layout(count, orders, dims, dtype, ranks, opts, 1, bl);
  if (s != RH_OK) return s;
  if (!bl.groupable) {
    set_error("unsupported: a batched plan needs every request on the grouped engine (truncated, FP32 or FP64 "
              "data, or a BF16 form whose first mode takes the small-row tensor-core kernels)");
    return RH_EUNSUPPORTED;
  }
  RH_CHECK_ARG(X != nullptr && factors != nullptr && cores != nullptr, "X, factors and cores must be non-NULL");
  for (int i = 0; i < count; ++i) RH_CHECK_ARG(X[i] != nullptr && cores[i] != nullptr, "null tensor or core");
  if (workspace == nullptr || workspace_bytes < bl.slices_total) {
    set_error("workspace too small: need " + std::to_string(bl.slices_total) + " bytes");
    return RH_ENOMEM;
  }
  rh_options o;
  rh_options_default(&o);
  if (opts) o = *opts;
  rh_batched_plan_s* p = new rh_batched_plan_s;
  s = record_batch(count, orders, dims, dtype, X, ranks, o, factors, cores, norms, info, static_cast<char*>(workspace), bl,
                   p->gp);
  if (s == RH_OK) {
    const cudaError_t e1 = cudaMalloc(&p->tables, std::max<size_t>(16, p->gp.blob.size()));
    const cudaError_t e2 =
        e1 == cudaSuccess ? cudaMemcpy(p->tables, p->gp.blob.data(), p->gp.blob.size(), cudaMemcpyHostToDevice) : e1;
    if (e2 != cudaSuccess) {
      set_error(std::string("CUDA error ") + cudaGetErrorString(e2) + " while storing the launch tables");
      s = e1 == cudaSuccess ? RH_ECUDA : RH_ENOMEM;
    }
  }
  if (s != RH_OK) {
    if (p->tables) cudaFree(p->tables);
    delete p;
    return s;
  }
  *plan = p;
  return RH_OK;
}

rh_status rsthosvd_batched_plan_run(rh_batched_plan plan, void* stream) {
  clear_error();
  RH_CHECK_ARG(plan != nullptr, "plan must be non-NULL");
  return run_grouped(plan->gp, plan->tables, (cudaStream_t)stream);
}

int64_t rsthosvd_batched_plan_launches(rh_batched_plan plan) {
  return plan ? (int64_t)plan->gp.launches.size() : -1;
}

void rsthosvd_batched_plan_destroy(rh_batched_plan plan) {
  if (!plan) return;
  if (plan->tables) cudaFree(plan->tables);
  delete plan;
}

}  // extern "C"
