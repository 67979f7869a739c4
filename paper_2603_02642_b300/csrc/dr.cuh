// NRTO-DR inner solve (Sec. II-B steps (4a)-(4c), Sec. III, Supplementary Sec. II) as one persistent
// kernel: a CTA owns an instance for all of its ADMM iterations (instances come from the work queue).
//
// ADMM on Problem 3 (the p = p̃ split), per iteration:
//   (4a) subproblem (7) in (k_v, p̃) by relaxed Douglas–Rachford.  Its state ξ̃ = (K̃, p̃̃, t̃, η̃) is
//        carried over from the previous ADMM iteration.  Per DR iteration (R_χ = r_χ I, R_s = σ I):
//          K = (Q_v + r_χ I + σ Σ_j Â_jᵀÂ_j)⁻¹ (r_χ K̃ + σ Σ_j Â_jᵀ(η̃_j - b̂_j))   (per-step Kronecker solve)
//          p̃_j = (r_χ p̃̃_j + ρ p_j + λ_j + σ t̃_j) / (ρ + r_χ + σ)
//          s_j = (p̃_j, Â_j k + b̂_j);  reflection 2 s_j - s̃_j;  projection onto the cone K_j
//          (Supplementary Sec. II-C);  s̃ += α(Π(2s - s̃) - s);  χ̃ += α(χ - χ̃);  r_dr = ‖Δs̃‖₂.
//        The Σ_j Â_jᵀ(η̃_j - b̂_j) of the next DR iteration is accumulated in the same row pass that
//        updates η̃ (Z'_m = Σ_j b_{j,m}(η̃_{j,m} - b̂_{j,m})ᵀ), so every DR iteration reads and
//        writes η̃ once.
//   (4b) subproblem 2, the exact minimizer over (δû, p): p_j = min(v_j, -g_j - b_jᵀδû) with
//        v = p̃ - λ/ρ leaves a strongly convex squared hinge in δû.  It is minimized by semismooth
//        Newton with Armijo backtracking.  Each Newton target is an LQ problem whose stage costs
//        carry ρ a_j a_jᵀ for the active rows, solved by a Riccati recursion (warp 0).  The trust
//        region ‖F_u δû‖ ≤ r is enforced by a multiplier μ ≥ 0, the root of ‖F_u δû(μ)‖² = r²
//        (bracket grown by 4, then Illinois regula falsi).
//   (4c) λ ← λ + ρ(p - p̃);  r_p = ‖p - p̃‖,  r_d = ρ‖p^l - p^{l-1}‖.
//
// Per-row storage in the DR path: p → D.p, λ (unscaled) → D.lamp, p̃ → D.pt, p̃̃ → D.w, t̃ → D.lamw,
// projection scale → D.s, b_jᵀδû → D.ell; D.ptn holds 2p̃ - t̃ during a DR pass and
// v_j + g_j during subproblem 2; D.dd / D.rnorm hold the Newton active weights and hinge values.
#pragma once
#include "fulladmm.cuh"

namespace nrto {

// ----------------------------------------------------------------------------------------------
// Subproblem 2 pieces (FP64).  x = (xu, xx): δû (T·NU) and the δx it generates ((T+1)·NX).
// ----------------------------------------------------------------------------------------------

// b_jᵀδû: ∇g_jᵀ δx_{t_j} for state rows, ±δu_{k,i} for control rows.
template <int NX, int NU, typename Real>
__device__ __forceinline__ double row_ell(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, int r,
                                          const double* xu, const double* xx) {
  const long long R = I.row0 + r;
  const int4 ri = D.rinfo[R];
  if (r < I.n_sr) {
    const double* a = S.arow + I.arow0 + (long long)r * NX;
    const double* x = xx + (long long)ri.x * NX;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < NX; ++c) v += a[c] * x[c];
    return v;
  }
  return ((ri.y == ROW_UHI) ? 1.0 : -1.0) * xu[(long long)ri.x * NU + ri.z];
}

// Riccati factorization of the Newton LQ problem: stage Hessians
//   Q_t = 2Q_x + μ I + Σ_{state rows j at t} w_j a_j a_jᵀ  (t = 1..T),
//   R_k = 2R_u + Σ_{control rows j at (k,i)} w_j e_i e_iᵀ,
// with w_j = ρ for active rows and 0 otherwise.  Stores L_k, Acl_k, N_k, M_k like the FullADMM
// block-2 factorization (same arena slots), so riccati_sweep solves it.  One warp.
template <int NX, int NU, typename Real>
__device__ __noinline__ void lq_factor_warp(const Dev<Real>& D, const Inst& I, double* ar, const Arena& L,
                                            const double* sa, const SlotL& SL, const LinSlot<Real>& S,
                                            const double* wrow, double mu, double* scr) {
  const int lane = threadIdx.x & 31;
  const int T = I.T;
  double* P = scr;
  double* PA = P + 196;
  double* PB = PA + 196;
  double* Huu = PB + 98;
  double* Hux = Huu + 49;
  double* Nm = Hux + 98;
  double* Lm = Nm + 49;
  double* Q = Lm + 98;
  double* tmp = Q + 196;
  const double* arow = S.arow + I.arow0;
  auto build_Q = [&](int t) {
    for (int q = lane; q < NX * NX; q += 32) {
      const int r = q / NX, c = q % NX;
      double v = (r == c) ? (2.0 * ar[L.Qx + r] + mu) : 0.0;
      for (int s = 0; s < I.rows_per_t; ++s) {
        const long long rr = (long long)(t - 1) * I.rows_per_t + s;
        v += wrow[I.row0 + rr] * arow[rr * NX + r] * arow[rr * NX + c];
      }
      Q[q] = v;
    }
    __syncwarp();
  };
  build_Q(T);
  for (int q = lane; q < NX * NX; q += 32) P[q] = Q[q];
  __syncwarp();
  for (int k = T - 1; k >= 0; --k) {
    const double* Ak = sa + SL.A + (long long)k * NX * NX;
    const double* Bk = sa + SL.B + (long long)k * NX * NU;
    wmm(PA, P, false, NX, Ak, false, NX, NX, NX, NX, 1.0, false);
    wmm(PB, P, false, NX, Bk, false, NU, NX, NU, NX, 1.0, false);
    wmm(Huu, Bk, true, NU, PB, false, NU, NU, NU, NX, 1.0, false);
    wmm(Hux, Bk, true, NU, PA, false, NX, NU, NX, NX, 1.0, false);
    if (lane == 0) {
      for (int u = 0; u < NU; ++u) Huu[u * NU + u] += 2.0 * ar[L.Ru + u];
      if (I.n_groups > 0) {
        const int gpk = I.n_groups / T;
        for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
          const int2 gr = D.groups[I.grp0 + g];
          const int iu = D.rinfo[gr.x].z;
          for (int q = 0; q < gr.y; ++q) Huu[iu * NU + iu] += wrow[gr.x + q];
        }
      }
      double C[49];
      for (int q = 0; q < NU * NU; ++q) C[q] = Huu[q];
      chol_inplace(C, NU);
      for (int col = 0; col < NU; ++col) {
        double y[7];
        for (int r = 0; r < NU; ++r) {
          double v = (r == col) ? 1.0 : 0.0;
          for (int s = 0; s < r; ++s) v -= C[r * NU + s] * y[s];
          y[r] = v / C[r * NU + r];
        }
        for (int r = NU - 1; r >= 0; --r) {
          double v = y[r];
          for (int s = r + 1; s < NU; ++s) v -= C[s * NU + r] * y[s];
          y[r] = v / C[r * NU + r];
        }
        for (int r = 0; r < NU; ++r) Nm[r * NU + col] = y[r];
      }
    }
    __syncwarp();
    wmm(Lm, Nm, false, NU, Hux, false, NX, NU, NX, NU, -1.0, false);
    double* gL = ar + L.RicL + (long long)k * NU * NX;
    double* gAcl = ar + L.RicAcl + (long long)k * NX * NX;
    double* gN = ar + L.RicN + (long long)k * NU * NU;
    double* gM = ar + L.RicM + (long long)k * NU * NX;
    for (int q = lane; q < NU * NX; q += 32) gL[q] = Lm[q];
    for (int q = lane; q < NU * NU; q += 32) gN[q] = Nm[q];
    wmm(gM, Nm, false, NU, Bk, true, NU, NU, NX, NU, 1.0, false);
    for (int q = lane; q < NX * NX; q += 32) gAcl[q] = Ak[q];
    __syncwarp();
    wmm(gAcl, Bk, false, NU, Lm, false, NX, NX, NX, NU, 1.0, true);
    if (k >= 1) {
      build_Q(k);
      wmm(tmp, Ak, true, NX, PA, false, NX, NX, NX, NX, 1.0, false);
      wmm(tmp, Hux, true, NX, Lm, false, NX, NX, NX, NU, 1.0, true);
      for (int q = lane; q < NX * NX; q += 32) {
        const int r = q / NX, c = q % NX;
        P[q] = Q[q] + 0.5 * (tmp[r * NX + c] + tmp[c * NX + r]);
      }
      __syncwarp();
    }
  }
}

// Squared norm of the gradient of the subproblem-2 objective at x (one warp, by the adjoint
// recursion): λ_t = 2Q_x(δx_t + x̂_t - x_g) + μ δx_t + Σ_{rows at t} w_j z_j a_j + A_tᵀλ_{t+1},
// ∂/∂δu_k = 2R_u(δu_k + û_k - u_ref) + Σ_{control rows at (k,i)} w_j σ_j z_j e_i + B_kᵀλ_{k+1}.
// With hinge = false the hinge terms are left out (then with x = 0, μ = 0 this is ‖c‖²).
template <int NX, int NU, typename Real>
__device__ __noinline__ double grad_norm2_warp(const Dev<Real>& D, const Inst& I, const double* ar, const Arena& L,
                                               const double* sa, const SlotL& SL, const LinSlot<Real>& S,
                                               const double* xu, const double* xx, double mu, bool hinge,
                                               double* lamv) {
  const int lane = threadIdx.x & 31;
  const int T = I.T;
  const double* arow = S.arow + I.arow0;
  const int gpk = (I.n_groups > 0) ? I.n_groups / T : 0;
  if (lane < NX) lamv[lane] = 0.0;   // λ_{T+1}
  __syncwarp();
  double g2 = 0.0;
  for (int t = T; t >= 1; --t) {
    double lt = 0.0;
    if (lane < NX) {
      const int c = lane;
      const double x = xx[(long long)t * NX + c];
      lt = 2.0 * ar[L.Qx + c] * (x + sa[SL.x_hat + (long long)t * NX + c] - ar[L.xg + c]) + mu * x;
      if (hinge)
        for (int s = 0; s < I.rows_per_t; ++s) {
          const long long rr = (long long)(t - 1) * I.rows_per_t + s;
          lt += D.dd[I.row0 + rr] * D.rnorm[I.row0 + rr] * arow[rr * NX + c];
        }
      if (t < T) {
        const double* At = sa + SL.A + (long long)t * NX * NX;
        for (int r = 0; r < NX; ++r) lt += At[r * NX + c] * lamv[r];
      }
    }
    __syncwarp();
    if (lane < NX) lamv[lane] = lt;
    __syncwarp();
    // gradient block k = t - 1 uses λ_t
    const int k = t - 1;
    if (lane < NU) {
      const int i = lane;
      double gk = 2.0 * ar[L.Ru + i] * (xu[(long long)k * NU + i] + sa[SL.u_hat + (long long)k * NU + i] - ar[L.uref + i]);
      if (hinge)
        for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
          const int2 gr = D.groups[I.grp0 + g];
          for (int q = 0; q < gr.y; ++q) {
            const int4 ri = D.rinfo[gr.x + q];
            if (ri.z == i) gk += D.dd[gr.x + q] * ((ri.y == ROW_UHI) ? 1.0 : -1.0) * D.rnorm[gr.x + q];
          }
        }
      const double* Bk = sa + SL.B + (long long)k * NX * NU;
      for (int r = 0; r < NX; ++r) gk += Bk[r * NU + i] * lamv[r];
      g2 += gk * gk;
    }
    __syncwarp();
  }
  return warp_sum(g2);
}

// Subproblem-2 objective at x + step·d (the constant is dropped):
//   Σ_k ‖δu_k‖²_{R_u} + 2(û_k - u_ref)ᵀR_u δu_k + Σ_{t≥1} ‖δx_t‖²_{Q_x} + 2(x̂_t - x_g)ᵀQ_x δx_t
//   + μ/2 ‖δx_t‖² + ρ/2 Σ_j max(0, w_j + b_jᵀδû)²,   w_j = v_j + g_j (in D.ptn).
// All threads; every thread returns the value.
template <int NX, int NU, typename Real>
__device__ double sub2_objective(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, const double* ar,
                                 const Arena& L, const double* sa, const SlotL& SL, const double* xu,
                                 const double* xx, const double* du_dir, const double* dx_dir, double step,
                                 double mu, double rho, double* red) {
  const int T = I.T, tid = threadIdx.x, NTt = blockDim.x;
  double f = 0.0, h = 0.0, z0 = 0.0, z1 = 0.0;
  for (int q = tid; q < T * NU; q += NTt) {
    const int i = q % NU;
    const double u = xu[q] + (du_dir ? step * du_dir[q] : 0.0);
    f += ar[L.Ru + i] * (u * u + 2.0 * (sa[SL.u_hat + q] - ar[L.uref + i]) * u);
  }
  for (int q = NX + tid; q < (T + 1) * NX; q += NTt) {
    const int c = q % NX;
    const double x = xx[q] + (dx_dir ? step * dx_dir[q] : 0.0);
    f += ar[L.Qx + c] * (x * x + 2.0 * (sa[SL.x_hat + q] - ar[L.xg + c]) * x) + 0.5 * mu * x * x;
  }
  const int n_rows = I.n_sr + I.n_cr;
  for (int r = tid; r < n_rows; r += NTt) {
    double e = row_ell<NX, NU, Real>(D, I, S, r, xu, xx);
    if (du_dir) e += step * row_ell<NX, NU, Real>(D, I, S, r, du_dir, dx_dir);
    const double z = D.ptn[I.row0 + r] + e;
    if (z > 0.0) h += z * z;
  }
  block_sum4(f, h, z0, z1, red);
  return f + 0.5 * rho * h;
}

// Σ_{t≥1} ‖δx_t‖² of x (all threads).
__device__ inline double traj_norm2(const double* xx, int T, int nx, double* red) {
  double s = 0.0, z0 = 0.0, z1 = 0.0, z2 = 0.0;
  for (int q = nx + threadIdx.x; q < (T + 1) * nx; q += blockDim.x) s += xx[q] * xx[q];
  block_sum4(s, z0, z1, z2, red);
  return s;
}

__device__ inline void copy_vec(double* dst, const double* src, int n) {
  for (int q = threadIdx.x; q < n; q += blockDim.x) dst[q] = src ? src[q] : 0.0;
  __syncthreads();
}

// Semismooth Newton for min f_μ(δû) from the iterate already in (xu, xx); result left there.
// (tu, tx) receive each Newton target (the LQ solution for the current active set).
template <int NX, int NU, typename Real>
__device__ void sub2_ssn(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, double* ar, const Arena& L,
                         const double* sa, const SlotL& SL, double* xu, double* xx, double mu, double rho,
                         double cnorm, double* red, double* vec, double* scr, int* s_int) {
  const int T = I.T, tid = threadIdx.x, warp = tid >> 5;
  const int n_rows = I.n_sr + I.n_cr;
  double* tu = ar + L.du;
  double* tx = ar + L.dx;
  const int gpk = (I.n_groups > 0) ? I.n_groups / T : 0;
  for (int it = 0; it < 100; ++it) {
    // hinge values and active weights at x
    for (int r = tid; r < n_rows; r += blockDim.x) {
      const long long R = I.row0 + r;
      const double z = D.ptn[R] + row_ell<NX, NU, Real>(D, I, S, r, xu, xx);
      D.rnorm[R] = z;
      D.dd[R] = (z > 0.0) ? rho : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      const double g2 = grad_norm2_warp<NX, NU, Real>(D, I, ar, L, sa, SL, S, xu, xx, mu, true, vec);
      if (tid == 0) red[0] = g2;
    }
    __syncthreads();
    const double gn = sqrt(red[0]);
    __syncthreads();
    if (gn <= 1e-13 * (1.0 + cnorm)) break;
    // Newton target: LQ problem with the active set of x
    if (warp == 0) lq_factor_warp<NX, NU, Real>(D, I, ar, L, sa, SL, S, D.dd, mu, scr);
    for (int q = tid; q < T * NX; q += blockDim.x) {
      const int t = q / NX + 1, c = q % NX;
      double v = 2.0 * ar[L.Qx + c] * (sa[SL.x_hat + (long long)t * NX + c] - ar[L.xg + c]);
      for (int s2 = 0; s2 < I.rows_per_t; ++s2) {
        const long long rr = (long long)(t - 1) * I.rows_per_t + s2;
        v += D.dd[I.row0 + rr] * D.ptn[I.row0 + rr] * S.arow[I.arow0 + rr * NX + c];
      }
      ar[L.qv + (long long)t * NX + c] = v;
    }
    for (int q = tid; q < T * NU; q += blockDim.x) {
      const int k = q / NU, iu = q % NU;
      double v = 2.0 * ar[L.Ru + iu] * (sa[SL.u_hat + q] - ar[L.uref + iu]);
      for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
        const int2 gr = D.groups[I.grp0 + g];
        for (int qq = 0; qq < gr.y; ++qq) {
          const int4 ri = D.rinfo[gr.x + qq];
          if (ri.z == iu) v += D.dd[gr.x + qq] * ((ri.y == ROW_UHI) ? 1.0 : -1.0) * D.ptn[gr.x + qq];
        }
      }
      ar[L.rv + q] = v;
    }
    __syncthreads();
    if (warp == 0) riccati_sweep<NX, NU, double>(ar, L, sa, SL, T, vec);
    __syncthreads();
    // direction d = target - x (kept in the target arrays)
    for (int q = tid; q < T * NU; q += blockDim.x) tu[q] -= xu[q];
    for (int q = tid; q < (T + 1) * NX; q += blockDim.x) tx[q] -= xx[q];
    __syncthreads();
    // directional derivative gradᵀd and f(x)
    double gd = 0.0, z0 = 0.0, z1 = 0.0, z2 = 0.0;
    for (int q = tid; q < T * NU; q += blockDim.x) {
      const int i = q % NU;
      gd += 2.0 * ar[L.Ru + i] * (xu[q] + sa[SL.u_hat + q] - ar[L.uref + i]) * tu[q];
    }
    for (int q = NX + tid; q < (T + 1) * NX; q += blockDim.x) {
      const int c = q % NX;
      gd += (2.0 * ar[L.Qx + c] * (xx[q] + sa[SL.x_hat + q] - ar[L.xg + c]) + mu * xx[q]) * tx[q];
    }
    for (int r = tid; r < n_rows; r += blockDim.x) {
      const long long R = I.row0 + r;
      if (D.dd[R] > 0.0) gd += D.dd[R] * D.rnorm[R] * row_ell<NX, NU, Real>(D, I, S, r, tu, tx);
    }
    block_sum4(gd, z0, z1, z2, red);
    const double f0 = sub2_objective<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, nullptr, nullptr, 0.0, mu, rho, red);
    double step = 1.0;
    for (int bt = 0; bt < 64; ++bt) {
      const double f1 = sub2_objective<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, tu, tx, step, mu, rho, red);
      if (f1 > f0 + 1e-4 * step * gd && step > 1e-12) step *= 0.5;
      else break;
    }
    for (int q = tid; q < T * NU; q += blockDim.x) xu[q] += step * tu[q];
    for (int q = tid; q < (T + 1) * NX; q += blockDim.x) xx[q] += step * tx[q];
    __syncthreads();
    int changed = 0;
    for (int r = tid; r < n_rows; r += blockDim.x) {
      const long long R = I.row0 + r;
      const double z = D.ptn[R] + row_ell<NX, NU, Real>(D, I, S, r, xu, xx);
      if ((z > 0.0) != (D.dd[R] > 0.0)) changed = 1;
    }
    changed = __syncthreads_or(changed);
    if (step == 1.0 && !changed) break;
  }
  (void)s_int;
}

// Subproblem 2 (exact) with w_j = v_j + g_j already in D.ptn: δû, δx into the arena (du, dx),
// ℓ_j = b_jᵀδû into D.ell.  Shared by NRTO-DR (v = p̃ - λ/ρ) and the as-written FullADMM block 2a
// (v = p̃ - λ_p, scaled dual).
template <int NX, int NU, typename Real>
__device__ __noinline__ void sub2_solve_w(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, double* ar,
                                          const Arena& L, const double* sa, const SlotL& SL, double rho,
                                          double r_trust, double* red, double* vec, double* scr, int* s_int) {
  const int T = I.T, tid = threadIdx.x, warp = tid >> 5;
  const int n_rows = I.n_sr + I.n_cr;
  __syncthreads();
  double* xu = ar + L.du_prev;
  double* xx = ar + L.dx_prev;
  double* hu = ar + L.Ws1;
  double* hx = ar + L.Ws2;
  const int nu_t = T * NU, nx_t = (T + 1) * NX;
  // ‖c‖ = ‖∇f_0(0)‖ without the hinge
  copy_vec(xu, nullptr, nu_t);
  copy_vec(xx, nullptr, nx_t);
  if (warp == 0) {
    const double c2 = grad_norm2_warp<NX, NU, Real>(D, I, ar, L, sa, SL, S, xu, xx, 0.0, false, vec);
    if (tid == 0) red[0] = c2;
  }
  __syncthreads();
  const double cnorm = sqrt(red[0]);
  __syncthreads();
  sub2_ssn<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, 0.0, rho, cnorm, red, vec, scr, s_int);
  const double r2 = r_trust * r_trust;
  // φ(μ) = ‖F̃ δû(μ)‖² - r², decreasing in μ: the trust multiplier is its root when φ(0) > 0
  double fa = traj_norm2(xx, T, NX, red) - r2;
  if (fa > 0.0) {
    // bracket [lo, hi] with φ(lo) > 0 >= φ(hi), growing hi by 4
    double lo = 0.0, hi = 1.0;
    sub2_ssn<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, hi, rho, cnorm, red, vec, scr, s_int);
    double fb = traj_norm2(xx, T, NX, red) - r2;
    for (int grow = 0; grow < 64 && fb > 0.0; ++grow) {
      lo = hi;
      fa = fb;
      hi *= 4.0;
      sub2_ssn<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, hi, rho, cnorm, red, vec, scr, s_int);
      fb = traj_norm2(xx, T, NX, red) - r2;
    }
    copy_vec(hu, xu, nu_t);
    copy_vec(hx, xx, nx_t);
    // Illinois regula falsi (a bracketing secant; the endpoint kept twice in a row has its φ
    // halved), each point solved from the feasible end's solution; the feasible end is returned
    // once the bracket is 1e-14 relative
    int side = 0;
    for (int it = 0; it < 200; ++it) {
      double mc = hi - fb * (hi - lo) / (fb - fa);
      if (!(lo < mc && mc < hi)) mc = 0.5 * (lo + hi);
      copy_vec(xu, hu, nu_t);
      copy_vec(xx, hx, nx_t);
      sub2_ssn<NX, NU, Real>(D, I, S, ar, L, sa, SL, xu, xx, mc, rho, cnorm, red, vec, scr, s_int);
      const double fc = traj_norm2(xx, T, NX, red) - r2;
      if (fc > 0.0) {
        lo = mc;
        fa = fc;
        if (side == -1) fb *= 0.5;
        side = -1;
      } else {
        hi = mc;
        fb = fc;
        copy_vec(hu, xu, nu_t);
        copy_vec(hx, xx, nx_t);
        if (side == 1) fa *= 0.5;
        side = 1;
      }
      if (hi - lo <= 1e-14 * hi || fc == 0.0) break;
    }
    copy_vec(xu, hu, nu_t);
    copy_vec(xx, hx, nx_t);
  }
  copy_vec(ar + L.du, xu, nu_t);
  copy_vec(ar + L.dx, xx, nx_t);
  for (int r = tid; r < n_rows; r += blockDim.x)
    D.ell[I.row0 + r] = row_ell<NX, NU, Real>(D, I, S, r, ar + L.du, ar + L.dx);
  __syncthreads();
}

// Subproblem 2 of NRTO-DR: v = p̃ - λ/ρ (unscaled λ).
template <int NX, int NU, typename Real>
__device__ __forceinline__ void sub2_solve(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, double* ar,
                                           const Arena& L, const double* sa, const SlotL& SL, double rho,
                                           double r_trust, double* red, double* vec, double* scr, int* s_int) {
  for (int r = threadIdx.x; r < I.n_sr + I.n_cr; r += blockDim.x) {
    const long long R = I.row0 + r;
    D.ptn[R] = (D.pt[R] - D.lamp[R] / rho) + S.g0[R];   // w_j = v_j + g_j
  }
  sub2_solve_w<NX, NU, Real>(D, I, S, ar, L, sa, SL, rho, r_trust, red, vec, scr, s_int);
}

// ----------------------------------------------------------------------------------------------
// One instance
// ----------------------------------------------------------------------------------------------
template <int NX, int NU, typename Real>
__device__ void dr_instance(const Dev<Real>& D, const SolveParams& sp, int inst, FASmem<NX, NU, Real>& sm,
                            uint64_t* bars, uint32_t* phase, int* s_flag, double* ric_scr) {
  using C = FACfg<NX, NU, Real>;
  constexpr int NT = C::NT, PAIRS = C::PAIRS, NWR_MAX = C::NWR_MAX, W = C::W;
  const Inst I = D.inst[inst];
  const Arena L = arena_layout(NX, NU, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(NX, NU, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[inst * NIS + IS_SLOT];
  const LinSlot<Real> S = D.slot[sl];
  const double* sa = S.arena + I.slot0;
  const int T = I.T;
  const int tid = threadIdx.x, lane = tid & 31;
  const double rho = sp.rho, rc = sp.r_chi, sg = sp.sigma, alpha = sp.alpha;
  const int n_rows = I.n_sr + I.n_cr;
  Real* lam = D.lam;   // η̃
  double* sc = D.sc + (long long)inst * NSC;
  int* isr = D.is + inst * NIS;
  const ChunkInfo* chunks = D.chunks + I.cb0;
  PhaseTimer tm;
  tm.start(D.phase_cycles != nullptr);

  const ColMap cm = col_map<NX, NU, Real>(I.T, FASmem<NX, NU, Real>::zcap(sp.chunk, sp.max_rows, I.T));
  const int grp = cm.grp, NG = cm.ng, NWR = cm.nwr, ck = cm.ck;
  const int gwarp = (tid - (grp < NG ? grp : 0) * NWR * 32) >> 5;
  const int mk[PAIRS] = {cm.mk[0], cm.mk[1]};

  // ---- initialization: ξ̃ = 0, p = λ = 0 (a warm start sets K̃ = K, p̃̃ = p = p̃ and keeps λ) ----
  for (long long e = tid; e < I.n_ent; e += NT) lam[I.ent0 + e] = (Real)0;
  for (int r = tid; r < n_rows; r += NT) {
    const long long R = I.row0 + r;
    if (!sp.warm) { D.p[R] = 0.0; D.pt[R] = 0.0; D.lamp[R] = 0.0; D.w[R] = 0.0; }
    else { D.p[R] = D.pt[R]; D.w[R] = D.pt[R]; }
    D.lamw[R] = 0.0; D.s[R] = 1.0; D.ell[R] = 0.0;
  }
  for (int q = tid; q < T * NU; q += NT) ar[L.du + q] = 0.0;
  for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.dx + q] = 0.0;
  for (int q = tid; q < T * NU * NX; q += NT) {
    if (!sp.warm) ar[L.K1 + q] = 0.0;
    ar[L.Kt + q] = ar[L.K1 + q];
  }
  for (int q = tid; q < (T + 1) * NU * NX; q += NT) ar[L.Gt1 + q] = 0.0;
  __syncthreads();
  tm.mark(PH_INIT);

  int status = ST_MAXITER, iters = 0, dr_total = 0;
  double r_p = 0.0, r_d = 0.0, r_dr = 0.0;
  const int Lmax = sp.max_iter;
  const int gpk = (I.n_groups > 0) ? I.n_groups / T : 0;
  (void)gpk;

  // Row pass over all rows.  zonly: only Z' = Σ_j b_j (η̃_j - b̂_j)ᵀ of the current η̃ (start of a
  // cold solve); otherwise one DR step on every row (projection of the reflection, η̃ and t̃
  // relaxation), accumulating Z' of the new η̃ and Σ‖Δs̃‖².  Returns Σ‖Δs̃‖² (all threads).
  auto row_pass = [&](bool zonly) -> double {
    Real gc[PAIRS][NU][W], z[PAIRS][NU][W];
    load_gt_regs<NX, NU, Real, PAIRS, W>(ar + L.Gt1, T, mk, ck, gc);
#pragma unroll
    for (int k = 0; k < PAIRS; ++k)
#pragma unroll
      for (int u = 0; u < NU; ++u)
#pragma unroll
        for (int w = 0; w < W; ++w) z[k][u][w] = (Real)0;
    double rdr = 0.0;
    __syncthreads();
    if (tid == 0) {
      fence_proxy_async();
      for (int c0 = 0; c0 < 2 && c0 < I.n_chunks; ++c0) issue_chunk<NX, NU, Real>(D, S, I, chunks[c0], sm.buf[c0], &bars[c0]);
    }
    bool ok = true;
    for (int ch = 0; ch < I.n_chunks; ++ch) {
      const int bi = ch & 1;
      typename FASmem<NX, NU, Real>::Buf& bf = sm.buf[bi];
      const ChunkInfo cki = chunks[ch];
      const int nr = cki.r1 - cki.r0;
      if (tid == 0) *s_flag = mbar_wait_bounded(&bars[bi], phase[bi]) ? 1 : 0;
      __syncthreads();
      phase[bi] ^= 1u;
      if (*s_flag == 0) { ok = false; break; }   // uniform: s_flag is shared
      if (!zonly) {
        // sub-pass 1: ‖2(Â_j k + b̂_j) - η̃_j‖ per row
        for (int q = grp; q < nr; q += NG) {
          const RowMeta rm = bf.meta[q];
          Real pn = 0;
          bool act = false;
#pragma unroll
          for (int k = 0; k < PAIRS; ++k) {
            if (mk[k] <= rm.t) {
              act = true;
              const int e = rm.off + mk[k] * NX + ck;
              Real bv[NU], yb[W], l[W];
              ld_vec<NU, Real>(bf.bb + rm.boff + mk[k] * NU, bv);
              ld_vec<W, Real>(bf.bhat + e, yb);
              ld_vec<W, Real>(bf.lam + e, l);
#pragma unroll
              for (int w = 0; w < W; ++w) {
                Real y = yb[w];
#pragma unroll
                for (int u = 0; u < NU; ++u) y += gc[k][u][w] * bv[u];
                const Real er = (Real)2 * y - l[w];
                pn += er * er;
              }
            }
          }
          if (__any_sync(0xffffffffu, act)) pn = warp_sum(pn);
          if (lane == 0) sm.rowpart[q * NWR_MAX + gwarp] = pn;
        }
        __syncthreads();
        // projection of (2p̃ - t̃, 2η - η̃) onto K_j; t̃ relaxation
        for (int q = tid; q < nr; q += NT) {
          Real a2 = 0;
          for (int w = 0; w < NWR; ++w) a2 += sm.rowpart[q * NWR_MAX + w];
          const long long R = I.row0 + bf.meta[q].pad;
          double snew, tpi;
          soc_case(D.ptn[R], sqrt((double)a2), snew, tpi);
          sm.snew[q] = (Real)snew;
          D.s[R] = snew;
          const double tt = D.lamw[R];
          const double ttn = tt + alpha * (tpi - D.pt[R]);
          rdr += (ttn - tt) * (ttn - tt);
          D.lamw[R] = ttn;
        }
        __syncthreads();
      }
      {
        // sub-pass 2: η̃ relaxation and Z' of the new η̃
        for (int q = grp; q < nr; q += NG) {
          const RowMeta rm = bf.meta[q];
          const Real sn = zonly ? (Real)0 : sm.snew[q];
#pragma unroll
          for (int k = 0; k < PAIRS; ++k) {
            if (mk[k] <= rm.t) {
              const int e = rm.off + mk[k] * NX + ck;
              Real bv[NU], yb[W], l[W];
              ld_vec<NU, Real>(bf.bb + rm.boff + mk[k] * NU, bv);
              ld_vec<W, Real>(bf.bhat + e, yb);
              ld_vec<W, Real>(bf.lam + e, l);
              if (!zonly) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                  Real y = yb[w];
#pragma unroll
                  for (int u = 0; u < NU; ++u) y += gc[k][u][w] * bv[u];
                  const Real er = (Real)2 * y - l[w];
                  const Real ln = l[w] + (Real)alpha * (sn * er - y);
                  rdr += (double)((ln - l[w]) * (ln - l[w]));
                  l[w] = ln;
                }
                st_vec<W, Real>(lam + cki.e0 + e, l);
              }
              if (mk[k] < rm.t) {
#pragma unroll
                for (int w = 0; w < W; ++w) {
                  const Real wv = l[w] - yb[w];
#pragma unroll
                  for (int u = 0; u < NU; ++u) z[k][u][w] += bv[u] * wv;
                }
              }
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0 && ch + 2 < I.n_chunks) {
        fence_proxy_async();
        issue_chunk<NX, NU, Real>(D, S, I, chunks[ch + 2], bf, &bars[bi]);
      }
    }
    if (!ok) return -1.0;
    // Z' = Σ over row groups (fixed order)
    if (NG == 1) {
#pragma unroll
      for (int k = 0; k < PAIRS; ++k)
        if (mk[k] < T)
#pragma unroll
          for (int u = 0; u < NU; ++u)
#pragma unroll
            for (int w = 0; w < W; ++w) ar[L.Zp + (long long)mk[k] * NU * NX + u * NX + ck + w] = (double)z[k][u][w];
    } else {
      Real* part = sm.buf[0].lam;
      const int nz = T * NU * NX;
#pragma unroll
      for (int k = 0; k < PAIRS; ++k)
        if (mk[k] < T)
#pragma unroll
          for (int u = 0; u < NU; ++u)
#pragma unroll
            for (int w = 0; w < W; ++w) part[grp * nz + mk[k] * NU * NX + u * NX + ck + w] = z[k][u][w];
      __syncthreads();
      for (int q = tid; q < nz; q += NT) {
        Real acc = 0;
        for (int g2 = 0; g2 < NG; ++g2) acc += part[g2 * nz + q];
        ar[L.Zp + q] = (double)acc;
      }
    }
    __syncthreads();
    // control rows (one block each; b = ±e_i, b̂ = 0); thread per (k, i) group, rows in order
    for (int g = tid; g < I.n_groups; g += NT) {
      const int2 gr = D.groups[I.grp0 + g];
      for (int q = 0; q < gr.y; ++q) {
        const long long R = gr.x + q;
        const int4 ri = D.rinfo[R];
        const int k = ri.x, iu = ri.z;
        const Real sgn = (ri.y == ROW_UHI) ? (Real)1 : (Real)-1;
        const long long e0 = D.rent[R];
        Real y[NX], l[NX];
        Real an = 0;
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          y[c] = sgn * (Real)ar[L.Gt1 + (long long)k * NU * NX + iu * NX + c];
          l[c] = lam[e0 + c];
          const Real er = (Real)2 * y[c] - l[c];
          an += er * er;
        }
        if (!zonly) {
          double snew, tpi;
          soc_case(D.ptn[R], sqrt((double)an), snew, tpi);
          D.s[R] = snew;
          const double tt = D.lamw[R];
          const double ttn = tt + alpha * (tpi - D.pt[R]);
          rdr += (ttn - tt) * (ttn - tt);
          D.lamw[R] = ttn;
#pragma unroll
          for (int c = 0; c < NX; ++c) {
            const Real er = (Real)2 * y[c] - l[c];
            const Real ln = l[c] + (Real)alpha * ((Real)snew * er - y[c]);
            rdr += (double)((ln - l[c]) * (ln - l[c]));
            l[c] = ln;
            lam[e0 + c] = ln;
          }
        }
#pragma unroll
        for (int c = 0; c < NX; ++c) ar[L.Zp + (long long)k * NU * NX + iu * NX + c] += (double)(sgn * l[c]);
      }
    }
    double z1 = 0.0, z2 = 0.0, z3 = 0.0;
    block_sum4(rdr, z1, z2, z3, sm.red);
    return rdr;
  };

  // Z' of the initial η̃ (zero) for the first gain solve
  if (row_pass(true) < 0.0) { status = ST_TIMEOUT; goto done; }
  tm.mark(PH_ROWS);

  for (int a = 1; a <= Lmax; ++a) {
    // ---------------- (4a) subproblem (7) by relaxed DR ----------------
    for (int d = 1; d <= sp.max_dr; ++d) {
      gain_solve<NX, NU, Real>(ar, L, T, I.sqrt_tau, sg * I.sqrt_tau, rc, ar + L.K1, ar + L.Gt1);
      tm.mark(PH_GAIN);
      for (int r = tid; r < n_rows; r += NT) {
        const long long R = I.row0 + r;
        const double pt = (rc * D.w[R] + rho * D.p[R] + D.lamp[R] + sg * D.lamw[R]) / (rho + rc + sg);
        D.pt[R] = pt;
        D.ptn[R] = 2.0 * pt - D.lamw[R];
      }
      __syncthreads();
      const double rdr2 = row_pass(false);
      if (rdr2 < 0.0) { status = ST_TIMEOUT; goto done; }
      tm.mark(PH_ROWS);
      for (int q = tid; q < T * NU * NX; q += NT) ar[L.Kt + q] += alpha * (ar[L.K1 + q] - ar[L.Kt + q]);
      for (int r = tid; r < n_rows; r += NT) {
        const long long R = I.row0 + r;
        D.w[R] += alpha * (D.pt[R] - D.w[R]);
      }
      __syncthreads();
      r_dr = sqrt(rdr2);
      ++dr_total;
      if (sp.check && r_dr <= sp.eps_dr) break;
    }
    // ---------------- (4b) subproblem 2 ----------------
    sub2_solve<NX, NU, Real>(D, I, S, ar, L, sa, SL, rho, sc[SC_RTRUST], sm.red, sm.vec, ric_scr, s_flag);
    tm.mark(PH_RICCATI);
    // ---------------- (4c) p, dual update, residuals ----------------
    double a_rp = 0.0, a_rd = 0.0, z2 = 0.0, z3 = 0.0;
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const double pt = D.pt[R];
      const double v = pt - D.lamp[R] / rho;
      const double pn = fmin(v, -S.g0[R] - D.ell[R]);
      a_rp += (pn - pt) * (pn - pt);
      a_rd += (pn - D.p[R]) * (pn - D.p[R]);
      D.lamp[R] += rho * (pn - pt);
      D.p[R] = pn;
    }
    block_sum4(a_rp, a_rd, z2, z3, sm.red);
    tm.mark(PH_DUALS);
    r_p = sqrt(a_rp);
    r_d = rho * sqrt(a_rd);
    iters = a;
    if (!(r_p == r_p) || !(r_d == r_d) || isinf(r_p) || isinf(r_d)) { status = ST_NUMERIC; break; }
    if (sp.check && r_p <= sp.eps_p && r_d <= sp.eps_d) { status = ST_CONVERGED; break; }
    if (a == Lmax) { status = ST_MAXITER; break; }
  }
done:
  if (status == ST_TIMEOUT && tid == 0) {
    for (int k = 0; k < 2; ++k) (void)mbar_wait_bounded(&bars[k], phase[k]);
  }
  if (tid == 0) {
    sc[SC_RP] = r_p; sc[SC_RD] = r_d; sc[SC_RPP] = r_p; sc[SC_RDP] = r_d; sc[SC_RDR] = r_dr; sc[SC_RHO] = rho;
    isr[IS_STATUS] = status; isr[IS_ITERS] = iters; isr[IS_CUMITERS] += iters; isr[IS_DRITERS] = dr_total;
  }
  tm.flush(D.phase_cycles);
  __syncthreads();
}

template <int NX, int NU, typename Real>
__global__ void __launch_bounds__(FACfg<NX, NU, Real>::NT, FACfg<NX, NU, Real>::MINB) k_dr(Dev<Real> D, SolveParams sp) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_next, s_flag;
  __shared__ double ric_scr[RIC_SCRATCH];
  FASmem<NX, NU, Real> sm;
  sm.carve(smem_raw, sp.chunk, sp.max_rows);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t ph[2] = {0u, 0u};
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(D.queue + sp.queue_idx, 1);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= sp.n_order) break;
    const int inst = D.order[sp.order0 + q];
    dr_instance<NX, NU, Real>(D, sp, inst, sm, bars, ph, &s_flag, ric_scr);
    if (D.is[inst * NIS + IS_STATUS] == ST_TIMEOUT) break;
  }
}

}  // namespace nrto
