// Recording of per-problem launch sequences and their replay as grouped launches (grouped.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace rh {

struct TapeEntry {
  KernelRef* k;
  int step, site, sub;
  dim3 grid;
  size_t smem;
  size_t off;   // argument bytes at Tape::bytes[off, off + k->args_bytes)
};

struct Tape {
  std::vector<TapeEntry> e;
  std::vector<uint8_t> bytes;
  int step = -1;
  int stray = 0;   // launches that bypassed emit while recording (the program cannot run grouped)
};

// Records the launches this thread emits into *t for the scope's lifetime.
class TapeScope {
 public:
  explicit TapeScope(Tape* t);
  ~TapeScope();
  TapeScope(const TapeScope&) = delete;
  TapeScope& operator=(const TapeScope&) = delete;

 private:
  Tape* prev_;
};

struct GroupedProgram {
  struct Launch {
    KernelRef* k;
    size_t smem;
    int n;            // problems in the group
    int64_t blocks;   // sum of their grids
    size_t args_off, start_off, gdim_off;   // tables in blob
  };
  std::vector<Launch> launches;
  std::vector<uint8_t> blob;   // launch tables, 16-byte aligned, as they go to the device
};

rh_status build_grouped(const std::vector<Tape>& tapes, GroupedProgram& gp);
// stream-ordered copy of gp.blob to dev (16-byte aligned, gp.blob.size() bytes); graph capturable
rh_status upload_tables_async(const GroupedProgram& gp, void* dev, cudaStream_t st);
rh_status run_grouped(const GroupedProgram& gp, const void* dev, cudaStream_t st);

void note_direct_launch();   // count_launch's hook: a launch that bypassed emit

}  // namespace rh
