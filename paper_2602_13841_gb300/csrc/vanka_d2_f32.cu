// Vanka build and sweep launches for d = 2, float (one translation unit per dimension and element
// type, compiled in parallel).
#include "vanka_launch.cuh"

namespace stmg {

template cudaError_t vanka_build_dim<float, 2>(const Level&, const Problem&, const float*, float*, float*, float*, float*, float*,
                                              void*, float*, int*, float*, cudaStream_t);
template cudaError_t vanka_apply_dim<float, 2>(const Level&, const Problem&, const float*, const void*, const float*,
                                              const float*, float*, double, double, int, int*, cudaStream_t, unsigned, int);

}  // namespace stmg
