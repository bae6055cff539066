// Host-side helpers shared by the C-ABI drivers (argument checks, column-major views).
#pragma once

#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rh {

inline rh_status check_tensor_args(int32_t order, const int64_t* dims, int32_t dtype) {
  RH_CHECK_ARG(order >= 1 && order <= RH_MAX_ORDER, "order must be in [1, 8]");
  RH_CHECK_ARG(dims != nullptr, "dims is NULL");
  for (int k = 0; k < order; ++k) RH_CHECK_ARG(dims[k] >= 1, "every dimension must be >= 1");
  RH_CHECK_ARG(dtype == RH_F64 || dtype == RH_F32, "dtype must be RH_F64 or RH_F32");
  return RH_OK;
}

inline int64_t prod(const std::vector<int64_t>& d) {
  int64_t n = 1;
  for (int64_t v : d) n *= v;
  return n;
}

}  // namespace rh
