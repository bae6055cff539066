// Optional per-launch timing of the library's main kernels with CUDA events recorded on
// the launching stream (rh_profile_enable / rh_profile_collect in the C ABI).  Off by
// default; when on, each timed launch is bracketed by two events from a pool.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rh {

namespace {
struct Rec {
  int kind, tag;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

bool profiling() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

ProfileScope::ProfileScope(int kind, int tag, cudaStream_t st) : st_(st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || recording()) return;   // a recorded program is timed as a whole
  Rec r{kind, tag, get_event(), get_event()};
  if (!r.a || !r.b) return;
  if (cudaEventRecord(r.a, st) != cudaSuccess) return;
  idx_ = (int)g_recs.size();
  g_recs.push_back(r);
}

ProfileScope::~ProfileScope() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (idx_ < (int)g_recs.size()) cudaEventRecord(g_recs[idx_].b, st_);
}

// Wait-timeout probe: the tensor-core launches of this process are numbered from the last
// rh_test_wait_probe call on; the one whose number equals the armed index gets probe = 1.
namespace {
std::atomic<int64_t> g_probe_at{-1};
std::atomic<int64_t> g_tc_count{0};
}  // namespace

int tc_probe_next() {
  const int64_t at = g_probe_at.load();
  const int64_t k = g_tc_count.fetch_add(1);
  return (at >= 0 && k == at) ? 1 : 0;
}

}  // namespace rh

extern "C" {

void rh_test_wait_probe(int64_t launch) {
  rh::g_tc_count.store(0);
  rh::g_probe_at.store(launch);
}

void rh_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(rh::g_mu);
  rh::g_on = on != 0;
}

int32_t rh_profile_collect(int32_t* kinds, int32_t* tags, float* ms, int32_t cap) {
  std::lock_guard<std::mutex> lk(rh::g_mu);
  int32_t n = 0;
  for (auto& r : rh::g_recs) {
    float t = -1.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess) cudaEventElapsedTime(&t, r.a, r.b);
    if (n < cap) {
      if (kinds) kinds[n] = r.kind;
      if (tags) tags[n] = r.tag;
      if (ms) ms[n] = t;
    }
    ++n;
    rh::g_pool.push_back(r.a);
    rh::g_pool.push_back(r.b);
  }
  rh::g_recs.clear();
  return n;
}

}  // extern "C"
