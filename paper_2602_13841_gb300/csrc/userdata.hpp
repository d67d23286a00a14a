// Caller-supplied problem data (STMG_USER): refresh of the device tables of f and g for a slab.
#pragma once
#include <cuda_runtime.h>

namespace stmg {

struct Handle;
// Evaluate the caller's f and g callbacks at the Radau times of the slab starting at t0 and upload
// them (no work when the tables already hold that slab or the problem is not STMG_USER).
// cudaErrorInvalidValue if a callback returned a non-finite value.
cudaError_t refresh_user_data(Handle* h, double t0);

}  // namespace stmg
