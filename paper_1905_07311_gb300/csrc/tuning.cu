// Process-wide launch-shape knobs of the small-tensor kernels (grid sizes of the small-row sketch
// and mode products and of the Gram matrix of B).  Defaults come from tuning_table.inc, which the
// project's tuner writes from measurements; rh_tuning_set lets the tuner (or a caller) try other
// values.  A knob changes how work is split over CTAs, so results may differ in the last bits
// between settings (the order of FP32 sums); calls with equal settings stay bit-identical.
#include <atomic>
#include <cstring>

#include "common.cuh"

namespace rh {
namespace {

struct TuneEntry {
  const char* name;
  int32_t def;
};

constexpr TuneEntry kTune[TUNE_COUNT] = {
#define RH_TUNE(key, name, value) {name, value},
#include "tuning_table.inc"
#undef RH_TUNE
};

std::atomic<int32_t> g_tune[TUNE_COUNT] = {
#define RH_TUNE(key, name, value) value,
#include "tuning_table.inc"
#undef RH_TUNE
};

int find_key(const char* name) {
  if (name == nullptr) return -1;
  for (int k = 0; k < TUNE_COUNT; ++k)
    if (std::strcmp(name, kTune[k].name) == 0) return k;
  return -1;
}

}  // namespace

int32_t tune(TuneKey k) { return g_tune[k].load(std::memory_order_relaxed); }

}  // namespace rh

extern "C" {

rh_status rh_tuning_set(const char* name, int32_t value) {
  rh::clear_error();
  const int k = rh::find_key(name);
  if (k < 0) {
    rh::set_error(std::string("invalid argument: unknown tuning key ") + (name ? name : "(null)"));
    return RH_EINVAL;
  }
  if (value == 0) value = rh::kTune[k].def;
  if (value < 1 || value > 4096) {
    rh::set_error("invalid argument: a tuning value must be in [1, 4096] (0 restores the table's value)");
    return RH_EINVAL;
  }
  rh::g_tune[k].store(value, std::memory_order_relaxed);
  return RH_OK;
}

int32_t rh_tuning_get(const char* name) {
  const int k = rh::find_key(name);
  return k < 0 ? -1 : rh::tune((rh::TuneKey)k);
}

int32_t rh_tuning_count(void) { return rh::TUNE_COUNT; }

const char* rh_tuning_name(int32_t index) {
  return (index >= 0 && index < rh::TUNE_COUNT) ? rh::kTune[index].name : nullptr;
}

}  // extern "C"
