// Persistent FullADMM (lifted and as-written block 2) and NRTO-DR kernels of the quadcopter (n_x, n_u) = (12, 4), in both compute precisions.
#include "solver_impl.cuh"

namespace nrto {
template struct SolverKernel<12, 4, float>;
template struct SolverKernel<12, 4, double>;
}  // namespace nrto
