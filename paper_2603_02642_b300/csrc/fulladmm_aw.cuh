// NRTO-FullADMM with block 2a as the paper states it (Sec. IV, Algorithm 1): per iteration,
//   (a) block 1: (ν_j, p̃_j) = Π_SOC(Â_j k + b̂_j + λ_ν,j, p_j + λ_p,j) for every row;
//   (c) block 2b: k = M ρ Σ_j Â_jᵀ(ν_j - b̂_j - λ_ν,j) (the Kronecker gain solve);
//   (b) block 2a: (δû, p) = argmin Q_û(δû) + ρ/2‖p - p̃ + λ_p‖² subject to the linearized robust
//       constraints g_j + b_jᵀδû + p_j ≤ 0 and the trust region ‖F_u δû‖ ≤ r: no slack variables, the
//       same QP as NRTO-DR's subproblem 2 with v = p̃ - λ_p, solved exactly in FP64 (semismooth
//       Newton over Riccati solves, the trust multiplier by Illinois regula falsi);
//   (d) λ_p += p - p̃, λ_ν += Â_j k + b̂_j - ν_j (the λ_ν update fused into the next row pass, as in
//       the lifted kernel), full residuals r_p = ‖(p - p̃, Âk + b̂ - ν)‖, r_d = ρ‖(Δp, Δ(Âk + b̂))‖.
// The row pass and the control rows are the lifted kernel's; the per-row arrays D.w (p̃ of the
// iteration) and D.ptn (w_j = v_j + g_j during block 2a) are scratch here.  Fixed ρ.
#pragma once
#include "dr.cuh"

namespace nrto {

template <int NX, int NU, typename Real>
__device__ void fulladmm_aw_instance(const Dev<Real>& D, const SolveParams& sp, int inst, FASmem<NX, NU, Real>& sm,
                                     uint64_t* bars, uint32_t* phase, int* s_flag, double* ric_scr) {
  using C = FACfg<NX, NU, Real>;
  constexpr int NT = C::NT;
  const Inst I = D.inst[inst];
  const Arena L = arena_layout(NX, NU, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(NX, NU, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[inst * NIS + IS_SLOT];
  const LinSlot<Real> S = D.slot[sl];
  const double* sa = S.arena + I.slot0;
  const int T = I.T;
  const int tid = threadIdx.x;
  const double rho = sp.rho;
  const int n_rows = I.n_sr + I.n_cr;
  Real* lam = D.lam;
  double* sc = D.sc + (long long)inst * NSC;
  int* isr = D.is + inst * NIS;
  PhaseTimer tm;
  tm.start(D.phase_cycles != nullptr);
  const ColMap cm = col_map<NX, NU, Real>(I.T, FASmem<NX, NU, Real>::zcap(sp.chunk, sp.max_rows, I.T));

  // ---- initialization (Algorithm 1): λ_p, λ_ν, k, p <- 0 ----
  for (long long e = tid; e < I.n_ent; e += NT) lam[I.ent0 + e] = (Real)0;
  for (int r = tid; r < n_rows; r += NT) {
    const long long R = I.row0 + r;
    D.p[R] = 0.0; D.pt[R] = 0.0; D.lamp[R] = 0.0; D.w[R] = 0.0;
    D.s[R] = 1.0; D.sr[R] = (Real)1; D.ell[R] = 0.0;
  }
  for (int q = tid; q < T * NU; q += NT) ar[L.du + q] = 0.0;
  for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.dx + q] = 0.0;
  for (int q = tid; q < T * NU * NX; q += NT) ar[L.K1 + q] = 0.0;
  for (int q = tid; q < (T + 1) * NU * NX; q += NT) { ar[L.Gt1 + q] = 0.0; ar[L.Gt0 + q] = 0.0; }
  if (tid == 0) { sc[SC_SCAL_RP] = 0; sc[SC_SCAL_RD] = 0; sc[SC_SCAL_RPP] = 0; sc[SC_SCAL_RDP] = 0; }
  __syncthreads();
  tm.mark(PH_INIT);
  int gsel = 1;
  const int Lmax = sp.max_iter;
  int status = ST_MAXITER, iters = 0;
  double r_p = 0, r_d = 0;

  for (int b = 1; b <= Lmax + 1 && Lmax > 0; ++b) {
    const bool first = (b == 1);
    const bool block1 = (b <= Lmax);
    const double* gtc_arena = ar + (gsel ? L.Gt1 : L.Gt0);
    const double* gto_arena = ar + (gsel ? L.Gt0 : L.Gt1);
    Real arp = 0, ard = 0;
    unsigned long long* const wc = tm.on ? &tm.acc[PH_WAIT] : nullptr;
    const bool rows_ok =
        first ? fa_row_pass<NX, NU, Real, true>(D, S, I, sm, bars, phase, s_flag, cm, gtc_arena, gto_arena, ar + L.Zp,
                                                block1, (Real)1, &arp, &ard, wc)
              : fa_row_pass<NX, NU, Real, false>(D, S, I, sm, bars, phase, s_flag, cm, gtc_arena, gto_arena, ar + L.Zp,
                                                 block1, (Real)1, &arp, &ard, wc);
    if (!rows_ok) {
      status = ST_TIMEOUT;
      goto done;
    }
    __syncthreads();
    tm.mark(PH_ROWS);
    double prp = (double)arp, prd = (double)ard;
    fa_control_rows<NX, NU, Real>(D, I, ar, L, gtc_arena, gto_arena, first, block1, (Real)1, prp, prd);
    {
      double z2 = 0.0, z3 = 0.0;
      block_sum4(prp, prd, z2, z3, sm.red);
    }
    tm.mark(PH_CTRL);
    // ---------------- convergence test of iteration b-1 ----------------
    if (!first) {
      r_p = sqrt(sc[SC_SCAL_RP] + prp);
      r_d = rho * sqrt(sc[SC_SCAL_RD] + prd);
      iters = b - 1;
      const bool bad = !(r_p == r_p) || !(r_d == r_d) || isinf(r_p) || isinf(r_d);
      if (bad) { status = ST_NUMERIC; break; }
      if (sp.check && r_p <= sp.eps_p && r_d <= sp.eps_d) { status = ST_CONVERGED; break; }
      if (b - 1 == Lmax) { status = ST_MAXITER; break; }
    }
    // ---------------- (c) block 2b: K^b and its Gtᵀ table (replaces the previous table) ----------------
    {
      double* gt_new = ar + (gsel ? L.Gt0 : L.Gt1);
      gain_solve_warps<NX, NU, Real>(ar, L, T, I.sqrt_tau, rho * I.sqrt_tau, ar + L.K1, gt_new, 0,
                                     GainScratch<NX, NU, Real>::warps(C::NW - 1), sm.rowpart);
      __syncthreads();
      gsel ^= 1;
    }
    tm.mark(PH_GAIN);
    // ---------------- (b) block 2a: the constrained (δû, p) QP with v = p̃ - λ_p ----------------
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const double ptn = D.ptn[R];               // p̃ of this iteration (block 1)
      D.w[R] = ptn;
      D.ptn[R] = (ptn - D.lamp[R]) + S.g0[R];    // w_j = v_j + g_j
    }
    sub2_solve_w<NX, NU, Real>(D, I, S, ar, L, sa, SL, rho, sc[SC_RTRUST], sm.red, sm.vec, ric_scr, s_flag);
    tm.mark(PH_RICCATI);
    // ---------------- (d) p, λ_p, scalar residual parts of iteration b ----------------
    double a_rp = 0, a_rd = 0, a_rpp = 0, a_rdp = 0;
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const double ptn = D.w[R];
      const double v = ptn - D.lamp[R];
      const double pn = fmin(v, -S.g0[R] - D.ell[R]);
      const double dp = pn - D.p[R];
      a_rp += (pn - ptn) * (pn - ptn);
      a_rd += dp * dp;
      a_rpp += (pn - ptn) * (pn - ptn);
      a_rdp += (ptn - D.pt[R]) * (ptn - D.pt[R]);
      D.lamp[R] += pn - ptn;
      D.p[R] = pn;
      D.pt[R] = ptn;
    }
    block_sum4(a_rp, a_rd, a_rpp, a_rdp, sm.red);
    if (tid == 0) { sc[SC_SCAL_RP] = a_rp; sc[SC_SCAL_RD] = a_rd; sc[SC_SCAL_RPP] = a_rpp; sc[SC_SCAL_RDP] = a_rdp; }
    __syncthreads();
    tm.mark(PH_DUALS);
  }
done:
  if (status == ST_TIMEOUT && tid == 0) {
    for (int k = 0; k < 2; ++k) (void)mbar_wait_bounded(&bars[k], phase[k]);
  }
  if (tid == 0) {
    sc[SC_RP] = r_p; sc[SC_RD] = r_d;
    sc[SC_RPP] = sqrt(sc[SC_SCAL_RPP]); sc[SC_RDP] = rho * sqrt(sc[SC_SCAL_RDP]);
    sc[SC_RHO] = rho;
    sc[SC_RHOD] = rho;
    isr[IS_STATUS] = status; isr[IS_ITERS] = iters; isr[IS_CUMITERS] += iters;
    isr[IS_MOVED] = 0;
  }
  tm.flush(D.phase_cycles);
  __syncthreads();
}

template <int NX, int NU, typename Real>
__global__ void __launch_bounds__(FACfg<NX, NU, Real>::NT, FACfg<NX, NU, Real>::MINB) k_fulladmm_aw(Dev<Real> D, SolveParams sp) {
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
    if (threadIdx.x == 0) D.is[inst * NIS + IS_FALLBACK] = 0;
    fulladmm_aw_instance<NX, NU, Real>(D, sp, inst, sm, bars, ph, &s_flag, ric_scr);
    if (D.is[inst * NIS + IS_STATUS] == ST_TIMEOUT) break;
  }
}

}  // namespace nrto
