// The opaque handle behind stmg_handle: parameters, stream, levels and device allocations.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/stmg.h"
#include "level.hpp"

namespace stmg {

struct Handle {
  stmg_params prm{};
  cudaStream_t stream = nullptr;
  Problem pb{};
  std::vector<Level> levels;
  std::vector<void*> allocs;
  std::string err;
  ~Handle();
  void* dalloc(size_t bytes);          // cudaMalloc tracked for release; throws std::bad_alloc
  stmg_status fail(stmg_status s, const std::string& msg);
};

}  // namespace stmg
