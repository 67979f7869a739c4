// Persistent FullADMM (lifted and as-written block 2) and NRTO-DR kernels of the unicycle (n_x, n_u) = (3, 2), in both compute precisions.
#include "solver_impl.cuh"

namespace nrto {
template struct SolverKernel<3, 2, float>;
template struct SolverKernel<3, 2, double>;
}  // namespace nrto
