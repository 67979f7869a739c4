// Definitions behind solver_kernels.h; included by the per-kind translation units only.
#pragma once
#include "fulladmm_aw.cuh"
#include "solver_kernels.h"

namespace nrto {

template <int NX, int NU, typename Real>
int SolverKernel<NX, NU, Real>::threads() {
  return FACfg<NX, NU, Real>::NT;
}

template <int NX, int NU, typename Real>
cudaError_t SolverKernel<NX, NU, Real>::configure(int solver, size_t smem, int* per_sm) {
  const void* k = solver == SOLVER_KERNEL_FULLADMM ? (const void*)k_fulladmm<NX, NU, Real>
                  : solver == SOLVER_KERNEL_DR     ? (const void*)k_dr<NX, NU, Real>
                                                   : (const void*)k_fulladmm_aw<NX, NU, Real>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, FACfg<NX, NU, Real>::NT, smem);
}

template <int NX, int NU, typename Real>
cudaError_t SolverKernel<NX, NU, Real>::launch(int solver, int grid, size_t smem, cudaStream_t st, const Dev<Real>& D,
                                               const SolveParams& sp) {
  if (solver == SOLVER_KERNEL_FULLADMM)
    k_fulladmm<NX, NU, Real><<<grid, FACfg<NX, NU, Real>::NT, smem, st>>>(D, sp);
  else if (solver == SOLVER_KERNEL_DR)
    k_dr<NX, NU, Real><<<grid, FACfg<NX, NU, Real>::NT, smem, st>>>(D, sp);
  else
    k_fulladmm_aw<NX, NU, Real><<<grid, FACfg<NX, NU, Real>::NT, smem, st>>>(D, sp);
  return cudaGetLastError();
}

}  // namespace nrto
