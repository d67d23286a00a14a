// Batched preconditioning across the slab solves of handles attached to one group (group.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg.hpp"

namespace stmg {

struct Handle;
struct Group;

// z = B^{-1} v for the attached handle h (FP64 level-0 vectors on h's stream): joins the next
// batched V-cycle of the group.
cudaError_t group_vcycle(Handle* h, const double* v, double* z);
// Smoother build of h's slot at the Newton state U (FP64, finest level).
cudaError_t group_build(Handle* h, const double* U);
// Detach h from its group (its destruction).
void group_forget(Handle* h);
// A slab solve of h starts / ends (the group waits for the handles inside a solve).
void group_enter(Handle* h);
void group_leave(Handle* h);
// The group's hierarchy (the MG of h's group, of h's preconditioner precision).
template <typename T>
MG<T>* group_core_mg(Handle* h);

}  // namespace stmg
