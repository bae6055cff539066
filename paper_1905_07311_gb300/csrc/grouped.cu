// Launch plumbing of the library: every kernel written as an Op (common.cuh) goes through
// emit_raw, which either launches it on the caller's stream or, while this thread records, appends
// it to a tape.  A tape is the launch sequence of one problem's program (one R-STHOSVD of one
// tensor); tapes of many independent problems merge into grouped launches, one per (step, site,
// sub, kernel) key, each running the blocks of every problem that has that launch.  Within a
// problem the keys increase strictly in program order (checked), so launching the groups in key
// order keeps every problem's own order; problems never wait on one another.
//
// A grouped launch reads its per-problem arguments, block offsets and grids from device tables
// (GroupedProgram::blob).  They reach the device either by one synchronous copy (plans) or by
// stream-ordered copy kernels whose payload travels in their parameters, which CUDA graph capture
// records by value, so a captured call needs no host memory to stay alive.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "grouped.cuh"

namespace rh {

namespace {

thread_local Tape* g_tape = nullptr;
std::mutex g_attr_mu;

struct MemsetOp {
  struct Args {
    uint8_t* p;
    uint64_t bytes;
  };
  static constexpr int kThreads = 256, kMinBlocks = 1;
  __device__ static void body(const Grid g, const Args& a) {
    for (uint64_t i = (uint64_t)g.bx * kThreads + threadIdx.x; i < a.bytes; i += (uint64_t)g.gx * kThreads) a.p[i] = 0;
  }
};

// One chunk of the launch tables, carried in the kernel's parameters (<= 32 KB of parameters).
constexpr int kChunkVec = 2000;   // uint4 words: 32000 bytes
struct TableChunk {
  uint4 w[kChunkVec];
};
__global__ void __launch_bounds__(256) table_copy_kernel(const TableChunk c, uint4* __restrict__ dst, int nvec) {
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = c.w[i];
}

// The default dynamic shared-memory limit of a kernel is 48 KB minus its static shared memory, so
// any dynamic size is opted in explicitly (once per kernel and size).
rh_status opt_in_smem(const void* fn, size_t smem, std::atomic<size_t>* done) {
  if (smem == 0 || smem <= done->load(std::memory_order_acquire)) return RH_OK;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  if (smem > done->load(std::memory_order_relaxed)) {
    RH_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done->store(smem, std::memory_order_release);
  }
  return RH_OK;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

bool recording() { return g_tape != nullptr; }
void record_step(int step) {
  if (g_tape) g_tape->step = step;
}
void note_direct_launch() {
  if (g_tape) ++g_tape->stray;
}

TapeScope::TapeScope(Tape* t) : prev_(g_tape) { g_tape = t; }
TapeScope::~TapeScope() { g_tape = prev_; }

rh_status launch_op_kernel(const void* fn, dim3 grid, int threads, size_t smem, cudaStream_t st, void** params) {
  static const bool pdl = [] {
    const char* v = std::getenv("RHOSVD_PDL");
    return !(v != nullptr && v[0] == '0');
  }();
  if (!pdl) {
    RH_CUDA_TRY(cudaLaunchKernel(fn, grid, dim3(threads), params, smem, st));
    return RH_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RH_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, params));
  return RH_OK;
}

rh_status emit_raw(KernelRef* k, int site, int sub, dim3 grid, size_t smem, cudaStream_t st, const void* args) {
  if (g_tape) {
    TapeEntry e{k, g_tape->step, site, sub, grid, smem, g_tape->bytes.size()};
    const uint8_t* p = static_cast<const uint8_t*>(args);
    g_tape->bytes.insert(g_tape->bytes.end(), p, p + k->args_bytes);
    g_tape->e.push_back(e);
    return RH_OK;
  }
  rh_status s = opt_in_smem(k->single, smem, &k->smem_single);
  if (s != RH_OK) return s;
  void* params[1] = {const_cast<void*>(args)};
  count_launch();
  return launch_op_kernel(k->single, grid, k->threads, smem, st, params);
}

rh_status emit_memset(int site, int sub, void* p, size_t bytes, cudaStream_t st) {
  if (g_tape) {
    const unsigned blocks = (unsigned)std::max<size_t>(1, std::min<size_t>((bytes + 4095) / 4096, 256));
    return emit<MemsetOp>(site, sub, dim3(blocks), 0, st, MemsetOp::Args{static_cast<uint8_t*>(p), bytes});
  }
  RH_CUDA_TRY(cudaMemsetAsync(p, 0, bytes, st));
  return RH_OK;
}

rh_status build_grouped(const std::vector<Tape>& tapes, GroupedProgram& gp) {
  gp.launches.clear();
  gp.blob.clear();
  // kernel ordinals in order of first appearance, so that the grouping is deterministic
  std::map<const KernelRef*, int> kord;
  using Key = std::tuple<int, int, int, int>;   // step, site, sub, kernel ordinal
  std::map<Key, std::vector<std::pair<int, int>>> groups;   // -> (problem, entry)
  for (int t = 0; t < (int)tapes.size(); ++t) {
    const Tape& tp = tapes[t];
    if (tp.stray) {
      set_error("internal: problem " + std::to_string(t) + " launched outside its recorded program");
      return RH_EUNSUPPORTED;
    }
    for (int i = 0; i < (int)tp.e.size(); ++i) {
      const TapeEntry& e = tp.e[i];
      if (i > 0) {
        const TapeEntry& q = tp.e[i - 1];
        if (std::make_tuple(q.step, q.site, q.sub) >= std::make_tuple(e.step, e.site, e.sub)) {
          set_error("internal: launch keys of problem " + std::to_string(t) + " do not increase (step " +
                    std::to_string(e.step) + ", site " + std::to_string(e.site) + ")");
          return RH_EUNSUPPORTED;
        }
      }
      if (e.site == SITE_OTHER || e.grid.z != 1 || (uint64_t)e.grid.x * e.grid.y == 0) {
        set_error("internal: a launch of problem " + std::to_string(t) + " cannot run grouped");
        return RH_EUNSUPPORTED;
      }
      auto it = kord.find(e.k);
      if (it == kord.end()) it = kord.emplace(e.k, (int)kord.size()).first;
      groups[Key(e.step, e.site, e.sub, it->second)].push_back({t, i});
    }
  }
  for (const auto& kv : groups) {
    const auto& mem = kv.second;
    const TapeEntry& e0 = tapes[mem[0].first].e[mem[0].second];
    KernelRef* k = e0.k;
    GroupedProgram::Launch L;
    L.k = k;
    L.n = (int)mem.size();
    L.smem = 0;
    L.args_off = align16(gp.blob.size());
    gp.blob.resize(L.args_off + (size_t)L.n * k->args_bytes);
    std::vector<int32_t> start(L.n + 1, 0);
    std::vector<uint32_t> gdim(2 * (size_t)L.n);
    int64_t total = 0;
    for (int j = 0; j < L.n; ++j) {
      const Tape& tp = tapes[mem[j].first];
      const TapeEntry& e = tp.e[mem[j].second];
      std::memcpy(gp.blob.data() + L.args_off + (size_t)j * k->args_bytes, tp.bytes.data() + e.off, k->args_bytes);
      start[j] = (int32_t)total;
      total += (int64_t)e.grid.x * e.grid.y;
      gdim[2 * j] = e.grid.x;
      gdim[2 * j + 1] = e.grid.y;
      L.smem = std::max(L.smem, e.smem);
      if (total >= (int64_t(1) << 31)) {
        set_error("grouped launch too large (more than 2^31 - 1 blocks)");
        return RH_EUNSUPPORTED;
      }
    }
    start[L.n] = (int32_t)total;
    L.blocks = total;
    L.start_off = align16(gp.blob.size());
    gp.blob.resize(L.start_off + sizeof(int32_t) * start.size());
    std::memcpy(gp.blob.data() + L.start_off, start.data(), sizeof(int32_t) * start.size());
    L.gdim_off = align16(gp.blob.size());
    gp.blob.resize(L.gdim_off + sizeof(uint32_t) * gdim.size());
    std::memcpy(gp.blob.data() + L.gdim_off, gdim.data(), sizeof(uint32_t) * gdim.size());
    gp.launches.push_back(L);
  }
  gp.blob.resize(align16(gp.blob.size()));
  return RH_OK;
}

rh_status upload_tables_async(const GroupedProgram& gp, void* dev, cudaStream_t st) {
  const size_t nvec = gp.blob.size() / 16;
  const uint4* src = reinterpret_cast<const uint4*>(gp.blob.data());
  uint4* dst = static_cast<uint4*>(dev);
  TableChunk c;
  for (size_t v0 = 0; v0 < nvec; v0 += kChunkVec) {
    const int n = (int)std::min<size_t>(kChunkVec, nvec - v0);
    std::memcpy(c.w, src + v0, sizeof(uint4) * n);
    table_copy_kernel<<<1, 256, 0, st>>>(c, dst + v0, n);
    RH_LAUNCH_CHECK();
  }
  return RH_OK;
}

rh_status run_grouped(const GroupedProgram& gp, const void* dev, cudaStream_t st) {
  const uint8_t* base = static_cast<const uint8_t*>(dev);
  for (const GroupedProgram::Launch& L : gp.launches) {
    rh_status s = opt_in_smem(L.k->group, L.smem, &L.k->smem_group);
    if (s != RH_OK) return s;
    const void* args = base + L.args_off;
    const int32_t* start = reinterpret_cast<const int32_t*>(base + L.start_off);
    const uint2* gdim = reinterpret_cast<const uint2*>(base + L.gdim_off);
    int n = L.n;
    void* params[4] = {&args, &start, &gdim, &n};
    count_launch();
    if ((s = launch_op_kernel(L.k->group, dim3((unsigned)L.blocks), L.k->threads, L.smem, st, params)) != RH_OK)
      return s;
  }
  return RH_OK;
}

}  // namespace rh
