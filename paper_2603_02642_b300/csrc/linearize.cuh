// Linearization prologue kernels (once per outer step) and per-solve factor kernels.
//
// Problem 2 data (Supplementary Sec. I) without dense matrices: for a state constraint j at
// time t with a_j = ∇g_j(x̂_t), the adjoint vectors v_t = a_j, v_i = A_iᵀ v_{i+1} give
//   b_{j,i} = (F_uᵀ a_j)_i = B_iᵀ v_{i+1}      and      b̂_{j,i} = √τ Ψ_i v_i      (i <= t),
// because F_u's block (t,i) is A_{t-1}⋯A_{i+1}B_i and F_ζ's block (t,m) is A_{t-1}⋯A_m.
// Control bounds have b_{j,k} = ±e_i and b̂_j = 0.
#pragma once
#include "dynamics.cuh"

namespace nrto {

// Slot selector of the linearization kernels: >= 0 a fixed slot, -1 the instance's current slot,
// -2 its candidate slot (the other one).
__device__ __forceinline__ int resolve_slot(const int* is, int i, int sel) {
  const int cur = is[i * NIS + IS_SLOT];
  return sel >= 0 ? sel : (sel == -1 ? cur : 1 - cur);
}

__device__ __forceinline__ long long kbuf_off(const Arena& L, int kbuf) {
  return kbuf == 0 ? L.K0 : (kbuf == 1 ? L.K1 : (kbuf == 2 ? L.Kt : L.Kacc));
}

// Ψ_m = L_mᵀ (L_m L_mᵀ = Σ_m), Σ_m = U_m diag(λ_m) U_mᵀ, Φ_m = Ψ_m U_m.  Block per instance.
template <typename Real>
__global__ void k_setup(Dev<Real> D) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  const int nx = I.nx;
  for (int m = threadIdx.x; m <= I.T; m += blockDim.x) {
    double S[196], V[196], lam[14], C[196];
    for (int k = 0; k < nx * nx; ++k) { S[k] = ar[L.Sigma + (long long)m * nx * nx + k]; C[k] = S[k]; }
    const bool pd = chol_inplace(C, nx);
    double* Psi = ar + L.Psi + (long long)m * nx * nx;
    if (pd)
      for (int r = 0; r < nx; ++r)
        for (int c = 0; c < nx; ++c) Psi[r * nx + c] = C[c * nx + r];   // Ψ = Lᵀ (upper triangular)
    jacobi_eig(S, nx, lam, V);
    if (!pd) {
      // Σ_i = Γ_i S_i⁻¹ Γ_iᵀ of a general block-diagonal Γ, positive semidefinite: Ψ = Λ^{1/2} Vᵀ
      for (int r = 0; r < nx; ++r)
        for (int c = 0; c < nx; ++c) Psi[r * nx + c] = sqrt(fmax(lam[r], 0.0)) * V[c * nx + r];
    }
    double* U = ar + L.SigU + (long long)m * nx * nx;
    for (int k = 0; k < nx * nx; ++k) U[k] = V[k];
    for (int k = 0; k < nx; ++k) ar[L.SigL + (long long)m * nx + k] = lam[k];
    double* Phi = ar + L.Phi + (long long)m * nx * nx;
    for (int r = 0; r < nx; ++r)
      for (int c = 0; c < nx; ++c) {
        double acc = 0.0;
        for (int k = 0; k < nx; ++k) acc += Psi[r * nx + k] * V[k * nx + c];
        Phi[r * nx + c] = acc;
      }
  }
}

// Nominal rollout x̂ (thread 0, sequential) then A_k, B_k in parallel.  Block per instance.
template <typename Real>
__global__ void k_rollout_jac(Dev<Real> D, int slot_sel) {
  const int i = blockIdx.x;
  const int slot = resolve_slot(D.is, i, slot_sel);
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const double* ar = D.arena + I.arena0;
  double* sa = D.slot[slot].arena + I.slot0;
  const int nx = I.nx, nu = I.nu;
  if (threadIdx.x == 0) {
    double* x = sa + SL.x_hat;
    for (int c = 0; c < nx; ++c) x[c] = ar[L.x0 + c];
    for (int k = 0; k < I.T; ++k)
      dyn_step(I.kind, ar + L.dyn, I.dt, x + (long long)k * nx, sa + SL.u_hat + (long long)k * nu,
               x + (long long)(k + 1) * nx, nullptr, nullptr, ar + L.xlo, ar + L.xhi);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < I.T; k += blockDim.x) {
    double xn[14];
    dyn_step(I.kind, ar + L.dyn, I.dt, sa + SL.x_hat + (long long)k * nx, sa + SL.u_hat + (long long)k * nu, xn,
             sa + SL.A + (long long)k * nx * nx, sa + SL.B + (long long)k * nx * nu, ar + L.xlo, ar + L.xhi);
  }
}

// g_j(x̂) and ∇g_j for every state row; g for control rows.  Block per instance.
template <typename Real>
__global__ void k_rows(Dev<Real> D, int slot_sel) {
  const int i = blockIdx.x;
  const int slot = resolve_slot(D.is, i, slot_sel);
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const double* ar = D.arena + I.arena0;
  const double* sa = D.slot[slot].arena + I.slot0;
  LinSlot<Real> S = D.slot[slot];
  const int nx = I.nx, nu = I.nu;
  for (int r = threadIdx.x; r < I.n_sr; r += blockDim.x) {
    const long long R = I.row0 + r;
    const int4 ri = D.rinfo[R];
    double grad[14];
    S.g0[R] = row_g_grad(I, ar, L, ri, sa + SL.x_hat + (long long)ri.x * nx, grad);
    for (int c = 0; c < nx; ++c) S.arow[I.arow0 + (long long)r * nx + c] = grad[c];
  }
  for (int r = threadIdx.x; r < I.n_cr; r += blockDim.x) {
    const long long R = I.row0 + I.n_sr + r;
    const int4 ri = D.rinfo[R];
    const double u = sa[SL.u_hat + (long long)ri.x * nu + ri.z];
    S.g0[R] = (ri.y == ROW_UHI) ? (u - ar[L.uhi + ri.z]) : (ar[L.ulo + ri.z] - u);
  }
}

// Adjoint rows of one instance (Supplementary Sec. I): for state row j at time t_j with gradient
// a_j, v_{j,t_j} = a_j, v_{j,i} = A_iᵀ v_{j,i+1}; b̂_{j,i} = √τ Ψ_i v_{j,i} (i = 0..t_j) and
// b_{j,i} = B_iᵀ v_{j,i+1} (i < t_j), b_{j,t_j} = 0.  One sweep over i = T..0 for all rows at once:
// each thread keeps RB rows' v in registers, the step's Ψ_i, A_{i-1}, B_{i-1} are staged in shared
// memory (double buffered, prefetched one step ahead) and shared by every row.  Arithmetic in the
// compute precision.
// Store N consecutive values of one row's block.  Blocks of n_x (or n_u) values start on a multiple
// of n_x (n_u) inside a row, rows start on 4-element boundaries inside a chunk, and chunks on 4-element
// boundaries of the array, so a block whose length is a multiple of 4 (2) is 16-byte (8-byte)
// aligned for FP32 and is stored with vector stores.
template <int N, typename Real>
__device__ __forceinline__ void st_block(Real* p, const Real (&v)[N]) {
  if constexpr (sizeof(Real) == 4 && N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 4) *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else if constexpr (sizeof(Real) == 4 && N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) *reinterpret_cast<float2*>(p + i) = make_float2(v[i], v[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

template <int NX, int NU, int RB, typename Real>
__device__ void adjoint_rows(const Dev<Real>& D, const Inst& I, const double* ar, const Arena& L, const double* sa,
                             const SlotL& SL, LinSlot<Real>& S, Real* smem) {
  constexpr int MW = NX * NX + NX * NX + NX * NU;   // Ψ_i, A_{i-1}, B_{i-1} of one step
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rpt = I.rows_per_t, nsr = I.n_sr;
  const Real sq = (Real)I.sqrt_tau;
  const double* Psi = ar + L.Psi;
  const double* A = sa + SL.A;
  const double* B = sa + SL.B;
  // step i's matrices: [Ψ_i | A_{i-1} | B_{i-1}] (A, B only for i >= 1)
  auto fetch = [&](int i, int q) -> Real {
    if (q < NX * NX) return (Real)Psi[(long long)i * NX * NX + q];
    if (i < 1) return (Real)0;
    if (q < 2 * NX * NX) return (Real)A[(long long)(i - 1) * NX * NX + (q - NX * NX)];
    return (Real)B[(long long)(i - 1) * NX * NU + (q - 2 * NX * NX)];
  };
  constexpr int PF = (MW + 127) / 128;   // values per thread for blockDim >= 128
  for (int r0 = 0; r0 < nsr; r0 += RB * nthr) {
    Real v[RB][NX];
    int tr[RB];
    long long e0[RB], b0[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int r = r0 + b * nthr + tid;
      tr[b] = -1;
      if (r < nsr) {
        const long long R = I.row0 + r;
        tr[b] = D.rinfo[R].x;
        e0[b] = D.rent[R];
        b0[b] = D.rbent[R];
      }
    }
    const int r_last = min(nsr - 1, r0 + RB * nthr - 1);
    const int kmax = r_last / rpt + 1;   // rows are ordered by t = 1..T
    // stage step kmax
    __syncthreads();
    for (int q = tid; q < MW; q += nthr) smem[(kmax & 1) * MW + q] = fetch(kmax, q);
    __syncthreads();
    for (int k = kmax; k >= 0; --k) {
      const Real* m = smem + (k & 1) * MW;
      const Real* sPsi = m;
      const Real* sA = m + NX * NX;
      const Real* sB = m + 2 * NX * NX;
      // prefetch step k-1 into registers
      Real nxt[PF];
#pragma unroll
      for (int w = 0; w < PF; ++w) {
        const int q = tid + w * nthr;
        nxt[w] = (k >= 1 && q < MW) ? fetch(k - 1, q) : (Real)0;
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        if (tr[b] < k) continue;
        const int r = r0 + b * nthr + tid;
        if (tr[b] == k) {
#pragma unroll
          for (int c = 0; c < NX; ++c) v[b][c] = (Real)S.arow[I.arow0 + (long long)r * NX + c];
          Real z[NU];
#pragma unroll
          for (int u = 0; u < NU; ++u) z[u] = (Real)0;
          st_block<NU>(S.bvec + b0[b] + (long long)k * NU, z);
        }
        {
          Real h[NX];
#pragma unroll
          for (int c = 0; c < NX; ++c) {
            Real acc = 0;
#pragma unroll
            for (int q = 0; q < NX; ++q) acc += sPsi[c * NX + q] * v[b][q];
            h[c] = sq * acc;
          }
          st_block<NX>(S.bhat + e0[b] + (long long)k * NX, h);
        }
        if (k >= 1) {
          Real bk[NU];
#pragma unroll
          for (int u = 0; u < NU; ++u) {
            Real acc = 0;
#pragma unroll
            for (int q = 0; q < NX; ++q) acc += sB[q * NU + u] * v[b][q];
            bk[u] = acc;
          }
          st_block<NU>(S.bvec + b0[b] + (long long)(k - 1) * NU, bk);
          Real vn[NX];
#pragma unroll
          for (int c = 0; c < NX; ++c) {
            Real acc = 0;
#pragma unroll
            for (int q = 0; q < NX; ++q) acc += sA[q * NX + c] * v[b][q];
            vn[c] = acc;
          }
#pragma unroll
          for (int c = 0; c < NX; ++c) v[b][c] = vn[c];
        }
      }
      if (k >= 1) {
        Real* mn = smem + ((k - 1) & 1) * MW;
#pragma unroll
        for (int w = 0; w < PF; ++w) {
          const int q = tid + w * nthr;
          if (q < MW) mn[q] = nxt[w];
        }
      }
      __syncthreads();
    }
  }
}

constexpr int ADJ_SMEM = 2 * (14 * 14 * 2 + 14 * 7);   // two steps of the largest kind

template <typename Real>
__global__ void __launch_bounds__(256) k_adjoint(Dev<Real> D, int slot_sel) {
  __shared__ Real smem[ADJ_SMEM];
  const int i = blockIdx.x;
  const int slot = resolve_slot(D.is, i, slot_sel);
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const double* ar = D.arena + I.arena0;
  const double* sa = D.slot[slot].arena + I.slot0;
  LinSlot<Real> S = D.slot[slot];
  if (I.n_sr == 0) return;
  if (I.kind == KIND_UNICYCLE) adjoint_rows<3, 2, 8, Real>(D, I, ar, L, sa, SL, S, smem);
  else if (I.kind == KIND_QUADCOPTER) adjoint_rows<12, 4, 4, Real>(D, I, ar, L, sa, SL, S, smem);
  else adjoint_rows<14, 7, 2, Real>(D, I, ar, L, sa, SL, S, smem);
}

// G_m = Σ_j b_{j,m} b_{j,m}ᵀ over state rows (from the stored, possibly rounded b) plus e_ie_iᵀ per
// control bound at step m.  Block per instance; a warp per block index m (gram_rows).
template <int NU, typename Real>
__device__ __forceinline__ void gram_rows(const Dev<Real>& D, const Inst& I, const Real* bv, double* sa, const SlotL& SL) {
  // A warp per block index m; its lanes take rows lane, lane+32, ... with independent loads and keep
  // the NU(NU+1)/2 distinct products in the compute precision, and the warp sums the lanes' partials
  // in FP64.
  constexpr int NP = NU * (NU + 1) / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = warp; m < I.T; m += nw) {
    Real acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = (Real)0;
    // state rows with t > m start at local row m·rows_per_t (rows are ordered by t = 1..T)
#pragma unroll 4
    for (int r = m * I.rows_per_t + lane; r < I.n_sr; r += 32) {
      const Real* b = bv + D.rbent[I.row0 + r] + (long long)m * NU;
      Real bb[NU];
#pragma unroll
      for (int u = 0; u < NU; ++u) bb[u] = b[u];
      int k = 0;
#pragma unroll
      for (int u1 = 0; u1 < NU; ++u1)
#pragma unroll
        for (int u2 = u1; u2 < NU; ++u2) acc[k++] += bb[u1] * bb[u2];
    }
    int k = 0;
#pragma unroll
    for (int u1 = 0; u1 < NU; ++u1)
#pragma unroll
      for (int u2 = u1; u2 < NU; ++u2, ++k) {
        double v = warp_sum((double)acc[k]);
        if (lane == 0) {
          if (u1 == u2 && I.n_groups > 0) {
            const int gpk = I.n_groups / I.T;   // control groups are ordered by step, gpk per step
            for (int g = m * gpk; g < (m + 1) * gpk; ++g) {
              const int2 gr = D.groups[I.grp0 + g];
              if (D.rinfo[gr.x].z == u1) v += (double)gr.y;
            }
          }
          sa[SL.Gm + (long long)m * NU * NU + u1 * NU + u2] = v;
          sa[SL.Gm + (long long)m * NU * NU + u2 * NU + u1] = v;
        }
      }
  }
}

template <typename Real>
__global__ void k_gram(Dev<Real> D, int slot_sel) {
  const int i = blockIdx.x;
  const int slot = resolve_slot(D.is, i, slot_sel);
  const Inst I = D.inst[i];
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  double* sa = D.slot[slot].arena + I.slot0;
  const Real* bv = D.slot[slot].bvec;
  if (I.kind == KIND_UNICYCLE) gram_rows<2, Real>(D, I, bv, sa, SL);
  else if (I.kind == KIND_QUADCOPTER) gram_rows<4, Real>(D, I, bv, sa, SL);
  else gram_rows<7, Real>(D, I, bv, sa, SL);
}

// Gain-solve factors for H_m = I⊗(2W + shift·I) + coef·τ Σ_m⊗G_m (W = R_KᵀR_K):
// with a = (2W+shift)^{-1/2}, a G_m a = V diag(γ) Vᵀ:  Pf_m = a V,  Dv_m[u][c] = 1/(1 + coef τ γ_u λ_c).
// Then H_m vec(K) = vec(R) is solved by K = Pf X U_mᵀ with X = (Pfᵀ R U_m) ⊙ Dv.  Thread per (inst, m).
template <typename Real>
__global__ void k_gain_factors(Dev<Real> D, double coef0, double shift, int warm) {
  const int i = blockIdx.x;
  const double coef = start_rho(D.is, D.sc, i, warm, coef0);
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[i * NIS + IS_SLOT];
  const double* sa = D.slot[sl].arena + I.slot0;
  const int nx = I.nx, nu = I.nu;
  for (int m = threadIdx.x; m < I.T; m += blockDim.x) {
    double a[7], G[49], V[49], gam[7];
    for (int u = 0; u < nu; ++u) a[u] = 1.0 / sqrt(2.0 * ar[L.RK + u] * ar[L.RK + u] + shift);
    for (int u = 0; u < nu; ++u)
      for (int v = 0; v < nu; ++v) G[u * nu + v] = a[u] * sa[SL.Gm + (long long)m * nu * nu + u * nu + v] * a[v];
    jacobi_eig(G, nu, gam, V);
    double* Pf = ar + L.Pf + (long long)m * nu * nu;
    for (int u = 0; u < nu; ++u)
      for (int v = 0; v < nu; ++v) Pf[u * nu + v] = a[u] * V[u * nu + v];
    for (int u = 0; u < nu; ++u) ar[L.Gam + (long long)m * nu + u] = gam[u];
    double* Dv = ar + L.Dv + (long long)m * nu * nx;
    for (int u = 0; u < nu; ++u)
      for (int c = 0; c < nx; ++c)
        Dv[u * nx + c] = 1.0 / (1.0 + coef * I.tau * gam[u] * ar[L.SigL + (long long)m * nx + c]);
  }
}

// warp-cooperative small matrix product C = op(A)·op(B) (row-major), lanes over outputs.
__device__ inline void wmm(double* C, const double* A, bool tA, int lda, const double* B, bool tB, int ldb,
                           int m, int n, int k, double alpha, bool accumulate) {
  for (int q = threadIdx.x & 31; q < m * n; q += 32) {
    int r = q / n, c = q % n;
    double acc = 0.0;
    for (int j = 0; j < k; ++j) {
      double av = tA ? A[j * lda + r] : A[r * lda + j];
      double bv = tB ? B[c * ldb + j] : B[j * ldb + c];
      acc += av * bv;
    }
    C[r * n + c] = accumulate ? C[r * n + c] + alpha * acc : alpha * acc;
  }
  __syncwarp();
}

// Riccati factorization of the FullADMM Block-2 LQ problem (lifted reading): stage Hessians
//   Q_t = 2Q_x + ρ I + (ρ/2) Σ_{state rows j at t} a_j a_jᵀ (t = 1..T),
//   R_k = 2R_u + (ρ/2) Σ_{control rows j at k} e_i e_iᵀ,
// dynamics δx_{k+1} = A_k δx_k + B_k δu_k, δx_0 = 0.  Stores per step
//   L_k = -Huu⁻¹Hux, Acl_k = A_k + B_k L_k, N_k = Huu⁻¹, M_k = Huu⁻¹ B_kᵀ.
// Run by one warp; `scr` is shared scratch of RIC_SCRATCH doubles.
constexpr int RIC_SCRATCH = 1176;
template <typename Real>
__device__ __noinline__ void riccati_factor_warp(const Dev<Real>& D, int i, double rho, double* scr) {
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[i * NIS + IS_SLOT];
  const double* sa = D.slot[sl].arena + I.slot0;
  const double* arow = D.slot[sl].arow;
  const int nx = I.nx, nu = I.nu;
  const int lane = threadIdx.x & 31;
  double* P = scr;
  double* PA = P + 196;
  double* PB = PA + 196;
  double* Huu = PB + 98;
  double* Hux = Huu + 49;
  double* Nm = Hux + 98;
  double* Lm = Nm + 49;
  double* Q = Lm + 98;
  double* tmp = Q + 196;
  auto build_Q = [&](int t) {
    for (int q = lane; q < nx * nx; q += 32) {
      int r = q / nx, c = q % nx;
      double v = (r == c) ? (2.0 * ar[L.Qx + r] + rho) : 0.0;
      for (int s = 0; s < I.rows_per_t; ++s) {
        long long rr = (long long)(t - 1) * I.rows_per_t + s;
        v += 0.5 * rho * arow[I.arow0 + rr * nx + r] * arow[I.arow0 + rr * nx + c];
      }
      Q[q] = v;
    }
    __syncwarp();
  };
  build_Q(I.T);
  for (int q = lane; q < nx * nx; q += 32) P[q] = Q[q];
  __syncwarp();
  for (int k = I.T - 1; k >= 0; --k) {
    const double* Ak = sa + SL.A + (long long)k * nx * nx;
    const double* Bk = sa + SL.B + (long long)k * nx * nu;
    wmm(PA, P, false, nx, Ak, false, nx, nx, nx, nx, 1.0, false);
    wmm(PB, P, false, nx, Bk, false, nu, nx, nu, nx, 1.0, false);
    wmm(Huu, Bk, true, nu, PB, false, nu, nu, nu, nx, 1.0, false);
    wmm(Hux, Bk, true, nu, PA, false, nx, nu, nx, nx, 1.0, false);
    if (lane == 0) {
      for (int u = 0; u < nu; ++u) Huu[u * nu + u] += 2.0 * ar[L.Ru + u];
      if (I.n_groups > 0) {
        const int gpk = I.n_groups / I.T;
        for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
          const int2 gr = D.groups[I.grp0 + g];
          const int iu = D.rinfo[gr.x].z;
          Huu[iu * nu + iu] += 0.5 * rho * gr.y;
        }
      }
      // N = Huu⁻¹ through Cholesky
      double C[49];
      for (int q = 0; q < nu * nu; ++q) C[q] = Huu[q];
      chol_inplace(C, nu);
      for (int col = 0; col < nu; ++col) {
        double y[7];
        for (int r = 0; r < nu; ++r) {
          double v = (r == col) ? 1.0 : 0.0;
          for (int s = 0; s < r; ++s) v -= C[r * nu + s] * y[s];
          y[r] = v / C[r * nu + r];
        }
        for (int r = nu - 1; r >= 0; --r) {
          double v = y[r];
          for (int s = r + 1; s < nu; ++s) v -= C[s * nu + r] * y[s];
          y[r] = v / C[r * nu + r];
        }
        for (int r = 0; r < nu; ++r) Nm[r * nu + col] = y[r];
      }
    }
    __syncwarp();
    wmm(Lm, Nm, false, nu, Hux, false, nx, nu, nx, nu, -1.0, false);
    double* gL = ar + L.RicL + (long long)k * nu * nx;
    double* gAcl = ar + L.RicAcl + (long long)k * nx * nx;
    double* gN = ar + L.RicN + (long long)k * nu * nu;
    double* gM = ar + L.RicM + (long long)k * nu * nx;
    for (int q = lane; q < nu * nx; q += 32) gL[q] = Lm[q];
    for (int q = lane; q < nu * nu; q += 32) gN[q] = Nm[q];
    wmm(gM, Nm, false, nu, Bk, true, nu, nu, nx, nu, 1.0, false);
    for (int q = lane; q < nx * nx; q += 32) gAcl[q] = Ak[q];
    __syncwarp();
    wmm(gAcl, Bk, false, nu, Lm, false, nx, nx, nx, nu, 1.0, true);
    {
      // packed record of step k in the compute precision: N, M, L, A_cl, B
      Real* pk = reinterpret_cast<Real*>(ar + L.RicPk) + (long long)k * pk_stride(nx, nu);
      const int oM = nu * nu, oL = oM + nu * nx, oA = oL + nu * nx, oB = oA + nx * nx;
      for (int q = lane; q < nu * nu; q += 32) pk[q] = (Real)Nm[q];
      for (int q = lane; q < nu * nx; q += 32) { pk[oM + q] = (Real)gM[q]; pk[oL + q] = (Real)Lm[q]; pk[oB + q] = (Real)Bk[q]; }
      for (int q = lane; q < nx * nx; q += 32) pk[oA + q] = (Real)gAcl[q];
      __syncwarp();
    }
    if (k >= 1) {
      build_Q(k);
      wmm(tmp, Ak, true, nx, PA, false, nx, nx, nx, nx, 1.0, false);        // AᵀPA
      wmm(tmp, Hux, true, nx, Lm, false, nx, nx, nx, nu, 1.0, true);        // + HuxᵀL
      for (int q = lane; q < nx * nx; q += 32) {
        int r = q / nx, c = q % nx;
        P[q] = Q[q] + 0.5 * (tmp[r * nx + c] + tmp[c * nx + r]);
      }
      __syncwarp();
    }
  }
}

// One warp per instance (block per instance, blockDim = 32).
// C (m×n) = α·op(A)·op(B) (+ C), compile-time shapes, each element summed over j in order (the
// same order as wmm).
template <int M, int N, int K, bool TA, bool TB, int LDA, int LDB>
__device__ __forceinline__ void wmm_c(double* C, const double* A, const double* B, double alpha, bool accumulate) {
  for (int q = threadIdx.x & 31; q < M * N; q += 32) {
    const int r = q / N, c = q % N;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const double av = TA ? A[j * LDA + r] : A[r * LDA + j];
      const double bv = TB ? B[c * LDB + j] : B[j * LDB + c];
      acc += av * bv;
    }
    C[r * N + c] = accumulate ? C[r * N + c] + alpha * acc : alpha * acc;
  }
  __syncwarp();
}

// riccati_factor_warp with compile-time (n_x, n_u) and A_k, B_k staged in shared memory once per step;
// the same operations in the same order, so the factors are identical.  Used by k_riccati_factor,
// which has shared memory to spare; the solver kernels keep riccati_factor_warp and its smaller
// scratch for their in-kernel refactorization.
constexpr int RIC_SCRATCH_STAGED = RIC_SCRATCH + 196 + 98;
template <int nx, int nu, typename Real>
__device__ void riccati_factor_staged(const Dev<Real>& D, int i, double rho, double* scr) {
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[i * NIS + IS_SLOT];
  const double* sa = D.slot[sl].arena + I.slot0;
  const double* arow = D.slot[sl].arow;
  const int lane = threadIdx.x & 31;
  double* P = scr;
  double* PA = P + 196;
  double* PB = PA + 196;
  double* Huu = PB + 98;
  double* Hux = Huu + 49;
  double* Nm = Hux + 98;
  double* Lm = Nm + 49;
  double* Q = Lm + 98;
  double* tmp = Q + 196;
  double* sA = tmp + 196;
  double* sB = sA + 196;
  auto build_Q = [&](int t) {
    for (int q = lane; q < nx * nx; q += 32) {
      int r = q / nx, c = q % nx;
      double v = (r == c) ? (2.0 * ar[L.Qx + r] + rho) : 0.0;
      for (int s = 0; s < I.rows_per_t; ++s) {
        long long rr = (long long)(t - 1) * I.rows_per_t + s;
        v += 0.5 * rho * arow[I.arow0 + rr * nx + r] * arow[I.arow0 + rr * nx + c];
      }
      Q[q] = v;
    }
    __syncwarp();
  };
  build_Q(I.T);
  for (int q = lane; q < nx * nx; q += 32) P[q] = Q[q];
  __syncwarp();
  for (int k = I.T - 1; k >= 0; --k) {
    const double* Ak = sa + SL.A + (long long)k * nx * nx;
    const double* Bk = sa + SL.B + (long long)k * nx * nu;
    for (int q = lane; q < nx * nx; q += 32) sA[q] = Ak[q];
    for (int q = lane; q < nx * nu; q += 32) sB[q] = Bk[q];
    __syncwarp();
    wmm_c<nx, nx, nx, false, false, nx, nx>(PA, P, sA, 1.0, false);
    wmm_c<nx, nu, nx, false, false, nx, nu>(PB, P, sB, 1.0, false);
    wmm_c<nu, nu, nx, true, false, nu, nu>(Huu, sB, PB, 1.0, false);
    wmm_c<nu, nx, nx, true, false, nu, nx>(Hux, sB, PA, 1.0, false);
    if (lane == 0) {
      for (int u = 0; u < nu; ++u) Huu[u * nu + u] += 2.0 * ar[L.Ru + u];
      if (I.n_groups > 0) {
        const int gpk = I.n_groups / I.T;
        for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
          const int2 gr = D.groups[I.grp0 + g];
          const int iu = D.rinfo[gr.x].z;
          Huu[iu * nu + iu] += 0.5 * rho * gr.y;
        }
      }
      double C[nu * nu];
      for (int q = 0; q < nu * nu; ++q) C[q] = Huu[q];
      chol_inplace(C, nu);
      for (int col = 0; col < nu; ++col) {
        double y[nu];
        for (int r = 0; r < nu; ++r) {
          double v = (r == col) ? 1.0 : 0.0;
          for (int s = 0; s < r; ++s) v -= C[r * nu + s] * y[s];
          y[r] = v / C[r * nu + r];
        }
        for (int r = nu - 1; r >= 0; --r) {
          double v = y[r];
          for (int s = r + 1; s < nu; ++s) v -= C[s * nu + r] * y[s];
          y[r] = v / C[r * nu + r];
        }
        for (int r = 0; r < nu; ++r) Nm[r * nu + col] = y[r];
      }
    }
    __syncwarp();
    wmm_c<nu, nx, nu, false, false, nu, nx>(Lm, Nm, Hux, -1.0, false);
    double* gL = ar + L.RicL + (long long)k * nu * nx;
    double* gAcl = ar + L.RicAcl + (long long)k * nx * nx;
    double* gN = ar + L.RicN + (long long)k * nu * nu;
    double* gM = ar + L.RicM + (long long)k * nu * nx;
    for (int q = lane; q < nu * nx; q += 32) gL[q] = Lm[q];
    for (int q = lane; q < nu * nu; q += 32) gN[q] = Nm[q];
    wmm_c<nu, nx, nu, false, true, nu, nu>(gM, Nm, sB, 1.0, false);
    for (int q = lane; q < nx * nx; q += 32) gAcl[q] = sA[q];
    __syncwarp();
    wmm_c<nx, nx, nu, false, false, nu, nx>(gAcl, sB, Lm, 1.0, true);
    {
      Real* pk = reinterpret_cast<Real*>(ar + L.RicPk) + (long long)k * pk_stride(nx, nu);
      const int oM = nu * nu, oL = oM + nu * nx, oA = oL + nu * nx, oB = oA + nx * nx;
      for (int q = lane; q < nu * nu; q += 32) pk[q] = (Real)Nm[q];
      for (int q = lane; q < nu * nx; q += 32) { pk[oM + q] = (Real)gM[q]; pk[oL + q] = (Real)Lm[q]; pk[oB + q] = (Real)sB[q]; }
      for (int q = lane; q < nx * nx; q += 32) pk[oA + q] = (Real)gAcl[q];
      __syncwarp();
    }
    if (k >= 1) {
      build_Q(k);
      wmm_c<nx, nx, nx, true, false, nx, nx>(tmp, sA, PA, 1.0, false);
      wmm_c<nx, nx, nu, true, false, nx, nx>(tmp, Hux, Lm, 1.0, true);
      for (int q = lane; q < nx * nx; q += 32) {
        int r = q / nx, c = q % nx;
        P[q] = Q[q] + 0.5 * (tmp[r * nx + c] + tmp[c * nx + r]);
      }
      __syncwarp();
    }
  }
}

template <typename Real>
__global__ void k_riccati_factor(Dev<Real> D, double rho0, int warm) {
  __shared__ double scr[RIC_SCRATCH_STAGED];
  const int kind = D.inst[blockIdx.x].kind;
  const double rho = start_rho(D.is, D.sc, blockIdx.x, warm, rho0);
  if (kind == KIND_UNICYCLE) riccati_factor_staged<3, 2, Real>(D, blockIdx.x, rho, scr);
  else if (kind == KIND_QUADCOPTER) riccati_factor_staged<12, 4, Real>(D, blockIdx.x, rho, scr);
  else riccati_factor_staged<14, 7, Real>(D, blockIdx.x, rho, scr);
}

// Dv_m[u][c] = 1/(1 + coef τ γ_u λ_c) for a new penalty (the eigen factors do not depend on it).
template <typename Real>
__device__ __noinline__ void gain_divisors(const Dev<Real>& D, int i, double coef) {
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  const int n = I.T * I.nu * I.nx;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const int m = q / (I.nu * I.nx), u = (q / I.nx) % I.nu, c = q % I.nx;
    ar[L.Dv + q] = 1.0 / (1.0 + coef * I.tau * ar[L.Gam + (long long)m * I.nu + u] * ar[L.SigL + (long long)m * I.nx + c]);
  }
}

// Gtᵀ_m = √τ K_m Ψ_mᵀ (nu×nx) for every step from a gain buffer; Gt_T = 0.  Block per instance.
template <typename Real>
__global__ void k_gain_to_gt(Dev<Real> D, int kbuf, int gtbuf) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  const int nx = I.nx, nu = I.nu;
  const double* K = ar + kbuf_off(L, kbuf);
  double* Gt = ar + (gtbuf == 0 ? L.Gt0 : L.Gt1);
  const int total = (I.T + 1) * nu * nx;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    int m = q / (nu * nx), u = (q / nx) % nu, c = q % nx;
    double acc = 0.0;
    if (m < I.T)
      for (int r = 0; r < nx; ++r)
        acc += K[(long long)m * nu * nx + u * nx + r] * ar[L.Psi + (long long)m * nx * nx + c * nx + r];
    Gt[q] = I.sqrt_tau * acc;
  }
}

// Merit of Problem 1 at the nominal of the selected slot with the gains in `kbuf` (Gtᵀ in `gtbuf`):
// φ = Σ_k (ū_k-u_ref)ᵀR_u(·) + Σ_{t≥1}(x̄_t-x_goal)ᵀQ_x(·) + Σ_k‖R_K K_k‖_F²
//     + w_p Σ_j max(0, g_j(x̄) + ‖Â_j k_v + b̂_j‖).
// Block per instance; writes sc[out_idx] and the cost to sc[SC_COST].  The row norms stream the
// ragged b̂, b rows once (warp per row) against the Gtᵀ table staged in shared memory; row values in
// the compute precision, sums in FP64.
template <int NX, int NU, typename Real>
__device__ void merit_rows(const Dev<Real>& D, const Inst& I, const double* Gt, const LinSlot<Real>& S,
                           Real* gts, double& vio, double& vmax) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = threadIdx.x; q < (I.T + 1) * NU * NX; q += blockDim.x) gts[q] = (Real)Gt[q];
  __syncthreads();
  for (int r = wid; r < I.n_sr + I.n_cr; r += nw) {
    const long long R = I.row0 + r;
    const int4 ri = D.rinfo[R];
    Real n2 = 0;
    if (r < I.n_sr) {
      const long long e0 = D.rent[R], b0 = D.rbent[R];
      const int len = (ri.x + 1) * NX;
      for (int e = lane; e < len; e += 32) {
        const int m = e / NX, c = e - m * NX;
        Real y = S.bhat[e0 + e];
#pragma unroll
        for (int u = 0; u < NU; ++u) y += gts[m * NU * NX + u * NX + c] * S.bvec[b0 + (long long)m * NU + u];
        n2 += y * y;
      }
    } else {
      for (int c = lane; c < NX; c += 32) {
        const Real y = gts[ri.x * NU * NX + ri.z * NX + c];
        n2 += y * y;
      }
    }
    n2 = warp_sum(n2);
    if (lane == 0) {
      const double v = S.g0[R] + sqrt((double)n2);
      vio += fmax(0.0, v);
      vmax = fmax(vmax, v);
    }
  }
}

template <typename Real>
__global__ void k_merit(Dev<Real> D, int slot_sel, int kbuf, int gtbuf, double w_p, int out_idx) {
  extern __shared__ __align__(16) char merit_smem[];
  const int i = blockIdx.x;
  const int slot = resolve_slot(D.is, i, slot_sel);
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const double* ar = D.arena + I.arena0;
  const double* sa = D.slot[slot].arena + I.slot0;
  const LinSlot<Real> S = D.slot[slot];
  const int nx = I.nx, nu = I.nu;
  const double* Gt = ar + (gtbuf == 0 ? L.Gt0 : L.Gt1);
  const double* K = ar + kbuf_off(L, kbuf);
  __shared__ double red[4 * 32];
  double cst = 0.0, vio = 0.0, z0 = 0.0, z1 = 0.0;
  double vmax = -INFINITY;   // no rows: every robust constraint holds trivially
  for (int q = threadIdx.x; q < I.T * nu; q += blockDim.x) {
    double d = sa[SL.u_hat + q] - ar[L.uref + q % nu];
    cst += ar[L.Ru + q % nu] * d * d;
  }
  for (int q = threadIdx.x; q < I.T * nx; q += blockDim.x) {
    double d = sa[SL.x_hat + nx + q] - ar[L.xg + q % nx];
    cst += ar[L.Qx + q % nx] * d * d;
  }
  for (int q = threadIdx.x; q < I.T * nu * nx; q += blockDim.x) {
    double kv = K[q] * ar[L.RK + (q / nx) % nu];
    cst += kv * kv;
  }
  Real* gts = reinterpret_cast<Real*>(merit_smem);
  if (I.kind == KIND_UNICYCLE) merit_rows<3, 2, Real>(D, I, Gt, S, gts, vio, vmax);
  else if (I.kind == KIND_QUADCOPTER) merit_rows<12, 4, Real>(D, I, Gt, S, gts, vio, vmax);
  else merit_rows<14, 7, Real>(D, I, Gt, S, gts, vio, vmax);
  block_sum4(cst, vio, z0, z1, red);
  vmax = block_max(vmax, red);
  if (threadIdx.x == 0) {
    D.sc[i * NSC + out_idx] = cst + w_p * vio;
    D.sc[i * NSC + SC_COST] = cst;
    if (out_idx == SC_PHI) {
      D.sc[i * NSC + SC_VIOL] = vmax;
      D.sc[i * NSC + SC_COST_ACC] = cst;
    } else {
      D.sc[i * NSC + SC_VIOLC] = vmax;
    }
  }
}

}  // namespace nrto
