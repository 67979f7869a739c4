// Host-side entry to the persistent inner-loop kernels (FullADMM, NRTO-DR).  The kernels are
// compiled in one translation unit per dynamics kind (solver_*.cu), so that the library's slowest
// compilations run in parallel; the host code in api.cu only sees these declarations.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "nrto_dev.cuh"

namespace nrto {

struct SolveParams;

enum : int { SOLVER_KERNEL_FULLADMM = 0, SOLVER_KERNEL_DR = 1, SOLVER_KERNEL_FULLADMM_AW = 2 };

template <int NX, int NU, typename Real>
struct SolverKernel {
  // Threads per CTA of both kernels.
  static int threads();
  // Raise the kernel's dynamic shared-memory limit to `smem` and return its resident CTAs per SM.
  static cudaError_t configure(int solver, size_t smem, int* per_sm);
  // Enqueue one persistent launch on `st`; returns the launch error, if any.
  static cudaError_t launch(int solver, int grid, size_t smem, cudaStream_t st, const Dev<Real>& D,
                            const SolveParams& sp);
};

extern template struct SolverKernel<3, 2, float>;
extern template struct SolverKernel<3, 2, double>;
extern template struct SolverKernel<12, 4, float>;
extern template struct SolverKernel<12, 4, double>;
extern template struct SolverKernel<14, 7, float>;
extern template struct SolverKernel<14, 7, double>;

}  // namespace nrto
