// Vanka build and sweep launches for d = 3, double (one translation unit per dimension and element
// type, compiled in parallel).
#include "vanka_launch.cuh"

namespace stmg {

template cudaError_t vanka_build_dim<double, 3>(const Level&, const Problem&, const double*, double*, double*, double*, double*, double*,
                                              void*, float*, int*, double*, cudaStream_t);
template cudaError_t vanka_apply_dim<double, 3>(const Level&, const Problem&, const double*, const void*, const float*,
                                              const double*, double*, double, double, int, int*, cudaStream_t, unsigned, int);

}  // namespace stmg
