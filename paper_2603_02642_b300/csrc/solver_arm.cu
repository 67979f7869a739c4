// Persistent FullADMM (lifted and as-written block 2) and NRTO-DR kernels of the arm (n_x, n_u) = (14, 7), in both compute precisions.
#include "solver_impl.cuh"

namespace nrto {
template struct SolverKernel<14, 7, float>;
template struct SolverKernel<14, 7, double>;
}  // namespace nrto
