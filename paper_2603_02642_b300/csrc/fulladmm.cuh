// NRTO-FullADMM inner loop (Sec. IV, Algorithm 1, Supplementary Sec. III) as one persistent
// kernel: a CTA owns an instance for all its iterations (instances come from a work queue, largest
// first).  Per iteration, over the ragged rows of the instance:
//   (a) Block 1: per row, η̂_j = Â_j k + b̂_j + λ_ν,j, t̂_j = p_j + λ_p,j, SOC projection
//       (ν_j, p̃_j) = Π(η̂_j, t̂_j) = (s_j η̂_j, p̃_j); lifted slacks w (orthant) and e (ball);
//   (c) gain update k = M ρ Σ_j Â_jᵀ(ν_j - b̂_j - λ_ν,j): the Σ is accumulated per step m as
//       Z'_m = Σ_j b_{j,m} w_{j,m}ᵀ, then K_m is solved with the per-step eigen factors;
//   (b) Block 2 (δû, p): Riccati backward/forward sweep with the factorization fixed per outer step;
//   (d) duals λ_p, λ_ν, λ_w, λ_e and the primal/dual residual reductions.
// Row state kept between iterations is λ_ν only (plus one scale s_j per row): ν^l = s^l(y^{l-1}+λ^{l-1})
// is recomputed from the gains, so the λ_ν update of iteration l is done during the row pass of
// iteration l+1 (which also yields the row parts of iteration l's residuals).  Termination at
// iteration l therefore happens after that pass; iteration l+1's block-1 results are discarded.
#pragma once
#include "linearize.cuh"

namespace nrto {

struct SolveParams {
  double rho, eps_p, eps_d;
  double alpha, r_chi, sigma, eps_dr;   // DR
  int max_iter, check, warm, max_dr;
  int chunk, max_rows, tmax, n_order;   // chunk entries, rows per chunk, max T of the launch, instances
  int order0, queue_idx;
};

template <int NX, int NU>
struct FACfg {
  static constexpr int NT = 512;
  static constexpr int NW = NT / 32;
  static constexpr int GS = NU * NX + 1;  // padded Gtᵀ step stride
  static constexpr int TMAXC = (NX == 3) ? 256 : (NX == 12 ? 160 : 128);
  static constexpr int PAIRS = ((TMAXC + 1) * NX + NT - 1) / NT;
};

// Supplementary Sec. II-C closed form: (t̂, η̂) ↦ (p̃, s·η̂)
__device__ __forceinline__ void soc_case(double tt, double a, double& s_new, double& pt_new) {
  if (a <= tt) { s_new = 1.0; pt_new = tt; }
  else if (a <= -tt) { s_new = 0.0; pt_new = 0.0; }
  else { pt_new = 0.5 * (tt + a); s_new = pt_new / a; }
}

// Shared-memory carve for one CTA (sizes must match fa_smem_bytes on the host).
template <int NX, int NU, typename Real>
struct FASmem {
  Real* gtA; Real* gtB; Real* eta; Real* uu; Real* bb; Real* rowS; int* rowOff; int* rowBOff; int* rowT;
  double* red; double* vec;
  NRTO_HD static size_t bytes(int tmax, int chunk, int max_rows) {
    size_t g = (size_t)(tmax + 1) * FACfg<NX, NU>::GS;
    size_t nb = (size_t)chunk / NX * NU + NU;
    size_t b = 2 * g * sizeof(Real) + 2 * (size_t)chunk * sizeof(Real) + nb * sizeof(Real) + max_rows * sizeof(Real);
    b = (b + 15) & ~(size_t)15;
    b += 3 * (size_t)max_rows * sizeof(int);
    b = (b + 15) & ~(size_t)15;
    b += (4 * FACfg<NX, NU>::NW + 4 * 16) * sizeof(double);
    return b;
  }
  __device__ void carve(char* base, int tmax, int chunk, int max_rows) {
    size_t g = (size_t)(tmax + 1) * FACfg<NX, NU>::GS;
    size_t nb = (size_t)chunk / NX * NU + NU;
    Real* r = reinterpret_cast<Real*>(base);
    gtA = r; r += g; gtB = r; r += g; eta = r; r += chunk; uu = r; r += chunk; bb = r; r += nb; rowS = r; r += max_rows;
    char* c = reinterpret_cast<char*>(r);
    c = base + ((c - base + 15) & ~(size_t)15);
    int* ip = reinterpret_cast<int*>(c);
    rowOff = ip; ip += max_rows; rowBOff = ip; ip += max_rows; rowT = ip; ip += max_rows;
    c = reinterpret_cast<char*>(ip);
    c = base + ((c - base + 15) & ~(size_t)15);
    red = reinterpret_cast<double*>(c);
    vec = red + 4 * FACfg<NX, NU>::NW;
  }
};

// Per-step gain solve (FullADMM: coefA = ρ√τ on Z', no K̃ term; DR adds r_χ K̃):
//   X = (Pfᵀ (coefA Z' Φ + coefK K̃ U)) ⊙ Dv,  K = Pf X Uᵀ,  Gtᵀ = √τ Pf X Φᵀ.
template <int NX, int NU, typename Real>
__device__ void gain_solve_step(const double* ar, const Arena& L, int m, double sqrt_tau, double coefA, double coefK,
                                const double* Kt, double* Kout, Real* gt_smem, double* gt_glob) {
  constexpr int GS = FACfg<NX, NU>::GS;
  Real Z[NU][NX], Y[NU][NX];
  const double* Zp = ar + L.Zp + (long long)m * NU * NX;
  const double* Pf = ar + L.Pf + (long long)m * NU * NU;
  const double* Phi = ar + L.Phi + (long long)m * NX * NX;
  const double* U = ar + L.SigU + (long long)m * NX * NX;
  const double* Dv = ar + L.Dv + (long long)m * NU * NX;
#pragma unroll
  for (int u = 0; u < NU; ++u)
#pragma unroll
    for (int c = 0; c < NX; ++c) Z[u][c] = (Real)Zp[u * NX + c];
  for (int u = 0; u < NU; ++u)
    for (int c = 0; c < NX; ++c) {
      Real acc = 0;
      for (int r = 0; r < NX; ++r) acc += Z[u][r] * (Real)Phi[r * NX + c];
      acc *= (Real)coefA;
      if (coefK != 0.0) {
        Real a2 = 0;
        for (int r = 0; r < NX; ++r) a2 += (Real)Kt[(long long)m * NU * NX + u * NX + r] * (Real)U[r * NX + c];
        acc += (Real)coefK * a2;
      }
      Y[u][c] = acc;
    }
  // X = (Pfᵀ Y) ⊙ Dv  (into Z)
  for (int u = 0; u < NU; ++u)
    for (int c = 0; c < NX; ++c) {
      Real acc = 0;
      for (int v = 0; v < NU; ++v) acc += (Real)Pf[v * NU + u] * Y[v][c];
      Z[u][c] = acc * (Real)Dv[u * NX + c];
    }
  // PX = Pf X  (into Y)
  for (int u = 0; u < NU; ++u)
    for (int c = 0; c < NX; ++c) {
      Real acc = 0;
      for (int v = 0; v < NU; ++v) acc += (Real)Pf[u * NU + v] * Z[v][c];
      Y[u][c] = acc;
    }
  for (int u = 0; u < NU; ++u)
    for (int c = 0; c < NX; ++c) {
      Real k = 0, g = 0;
      for (int r = 0; r < NX; ++r) {
        k += Y[u][r] * (Real)U[c * NX + r];
        g += Y[u][r] * (Real)Phi[c * NX + r];
      }
      Kout[(long long)m * NU * NX + u * NX + c] = (double)k;
      g *= (Real)sqrt_tau;
      gt_smem[m * GS + u * NX + c] = g;
      gt_glob[(long long)m * NU * NX + u * NX + c] = (double)g;
    }
}

// Block-2 (δû) LQ sweep with fixed factors (warp 0 only).  Linear terms q_t (t = 0..T, index t
// of qv; q_0 unused) and r_k in the arena.  Writes du, dx.  Arithmetic in Real.
template <int NX, int NU, typename Real>
__device__ void riccati_sweep(double* ar, const Arena& L, const double* sa, const SlotL& SL, int T, double* pv) {
  const int lane = threadIdx.x & 31;
  // backward: l_k = -(N_k r_k + M_k p_{k+1}),  p_k = q_k + Acl_kᵀ p_{k+1} + L_kᵀ r_k
  if (lane < NX) pv[lane] = ar[L.qv + (long long)T * NX + lane];
  __syncwarp();
  for (int k = T - 1; k >= 0; --k) {
    const double* N = ar + L.RicN + (long long)k * NU * NU;
    const double* M = ar + L.RicM + (long long)k * NU * NX;
    const double* Lk = ar + L.RicL + (long long)k * NU * NX;
    const double* Acl = ar + L.RicAcl + (long long)k * NX * NX;
    const double* r = ar + L.rv + (long long)k * NU;
    Real lv = 0, pn = 0;
    if (lane < NU) {
      for (int v = 0; v < NU; ++v) lv += (Real)N[lane * NU + v] * (Real)r[v];
      for (int c = 0; c < NX; ++c) lv += (Real)M[lane * NX + c] * (Real)pv[c];
      ar[L.du + (long long)k * NU + lane] = -(double)lv;   // l_k stored in du until the forward pass
    }
    if (lane < NX && k >= 1) {
      pn = (Real)ar[L.qv + (long long)k * NX + lane];
      for (int c = 0; c < NX; ++c) pn += (Real)Acl[c * NX + lane] * (Real)pv[c];
      for (int v = 0; v < NU; ++v) pn += (Real)Lk[v * NX + lane] * (Real)r[v];
    }
    __syncwarp();
    if (lane < NX && k >= 1) pv[lane] = (double)pn;
    __syncwarp();
  }
  // forward: δx_0 = 0, δu_k = L_k δx_k + l_k, δx_{k+1} = A_k δx_k + B_k δu_k
  double* dx = ar + L.dx;
  double* du = ar + L.du;
  if (lane < NX) dx[lane] = 0.0;
  __syncwarp();
  for (int k = 0; k < T; ++k) {
    const double* Lk = ar + L.RicL + (long long)k * NU * NX;
    const double* A = sa + SL.A + (long long)k * NX * NX;
    const double* B = sa + SL.B + (long long)k * NX * NU;
    Real u = 0;
    if (lane < NU) {
      u = (Real)du[(long long)k * NU + lane];
      for (int c = 0; c < NX; ++c) u += (Real)Lk[lane * NX + c] * (Real)dx[(long long)k * NX + c];
    }
    __syncwarp();
    if (lane < NU) du[(long long)k * NU + lane] = (double)u;
    __syncwarp();
    if (lane < NX) {
      Real x = 0;
      for (int c = 0; c < NX; ++c) x += (Real)A[lane * NX + c] * (Real)dx[(long long)k * NX + c];
      for (int v = 0; v < NU; ++v) x += (Real)B[lane * NU + v] * (Real)du[(long long)k * NU + v];
      dx[(long long)(k + 1) * NX + lane] = (double)x;
    }
    __syncwarp();
  }
}

template <int NX, int NU, typename Real>
__device__ void fulladmm_instance(const Dev<Real>& D, const SolveParams& sp, int inst, FASmem<NX, NU, Real>& sm) {
  using C = FACfg<NX, NU>;
  constexpr int NT = C::NT, NW = C::NW, GS = C::GS, PAIRS = C::PAIRS;
  const Inst I = D.inst[inst];
  const Arena L = arena_layout(NX, NU, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(NX, NU, I.T);
  double* ar = D.arena + I.arena0;
  const int sl = D.is[inst * NIS + IS_SLOT];
  const LinSlot<Real> S = D.slot[sl];
  const double* sa = S.arena + I.slot0;
  const int T = I.T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double rho = sp.rho;
  const int n_rows = I.n_sr + I.n_cr;
  Real* lam = D.lam;
  double* sc = D.sc + (long long)inst * NSC;
  int* isr = D.is + inst * NIS;

  // ---- initialization (Algorithm 1): λ_p, λ_ν, k, p <- 0 (or a warm start of k, p̃, λ_p) ----
  for (long long e = tid; e < I.n_ent; e += NT) lam[I.ent0 + e] = (Real)0;
  for (int r = tid; r < n_rows; r += NT) {
    const long long R = I.row0 + r;
    if (!sp.warm) { D.p[R] = 0.0; D.pt[R] = 0.0; D.lamp[R] = 0.0; }
    else { D.p[R] = D.pt[R]; }
    D.w[R] = 0.0; D.lamw[R] = 0.0; D.s[R] = 1.0; D.ell[R] = 0.0;
  }
  for (int q = tid; q < T * NU; q += NT) { ar[L.du + q] = 0.0; }
  for (int q = tid; q < (T + 1) * NX; q += NT) { ar[L.dx + q] = 0.0; ar[L.e + q] = 0.0; ar[L.lam_e + q] = 0.0; }
  if (!sp.warm)
    for (int q = tid; q < T * NU * NX; q += NT) ar[L.K1 + q] = 0.0;
  __syncthreads();
  // Gtᵀ of the initial gains
  for (int q = tid; q < (T + 1) * NU * NX; q += NT) {
    int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    double acc = 0.0;
    if (m < T)
      for (int r = 0; r < NX; ++r) acc += ar[L.K1 + (long long)m * NU * NX + u * NX + r] * ar[L.Psi + (long long)m * NX * NX + c * NX + r];
    ar[L.Gt1 + q] = I.sqrt_tau * acc;
    sm.gtB[m * GS + u * NX + c] = (Real)(I.sqrt_tau * acc);
  }
  if (tid == 0) { sc[SC_SCAL_RP] = 0; sc[SC_SCAL_RD] = 0; sc[SC_SCAL_RPP] = 0; sc[SC_SCAL_RDP] = 0; }
  __syncthreads();
  Real* gtOld = sm.gtA;   // Gtᵀ of k^{b-2}
  Real* gtCur = sm.gtB;   // Gtᵀ of k^{b-1}
  const int Lmax = sp.max_iter;
  int status = ST_MAXITER, iters = 0;
  double r_p = 0, r_d = 0;

  for (int b = 1; b <= Lmax + 1 && Lmax > 0; ++b) {
    const bool first = (b == 1);
    const bool block1 = (b <= Lmax);
    double prp = 0.0, prd = 0.0;
    Real acc[PAIRS][NU];
#pragma unroll
    for (int k = 0; k < PAIRS; ++k)
#pragma unroll
      for (int u = 0; u < NU; ++u) acc[k][u] = (Real)0;

    // ---------------- row pass over state rows, chunk by chunk ----------------
    for (int ch = 0; ch < I.n_chunks; ++ch) {
      const int r0 = D.cbound[I.cb0 + ch], r1 = D.cbound[I.cb0 + ch + 1];
      const long long ec0 = D.rent[I.row0 + r0];
      const long long bc0 = D.rbent[I.row0 + r0];
      // sub-pass 1: warp per row
      for (int r = r0 + warp; r < r1; r += NW) {
        const long long R = I.row0 + r;
        const int t = D.rinfo[R].x;
        const long long e0 = D.rent[R], b0 = D.rbent[R];
        const int len = (t + 1) * NX;
        const int loc = (int)(e0 - ec0), bloc = (int)(b0 - bc0);
        const Real sold = (Real)D.s[R];
        Real arp = 0, ard = 0, an = 0;
        for (int e = lane; e < len; e += 32) {
          const int m = e / NX, c = e - m * NX;
          Real bvv[NU];
#pragma unroll
          for (int u = 0; u < NU; ++u) bvv[u] = S.bvec[b0 + (long long)m * NU + u];
          const Real yb = S.bhat[e0 + e];
          Real y = yb;
          const Real* gc = gtCur + m * GS + c;
#pragma unroll
          for (int u = 0; u < NU; ++u) y += gc[u * NX] * bvv[u];
          Real l = lam[e0 + e];
          if (!first) {
            Real yo = yb;
            const Real* go = gtOld + m * GS + c;
#pragma unroll
            for (int u = 0; u < NU; ++u) yo += go[u * NX] * bvv[u];
            const Real nu = sold * (yo + l);
            const Real ln = l + y - nu;
            arp += (y - nu) * (y - nu);
            ard += (y - yo) * (y - yo);
            l = ln;
            lam[e0 + e] = l;
          }
          if (block1) {
            const Real et = y + l;
            an += et * et;
            sm.eta[loc + e] = et;
            sm.uu[loc + e] = -yb - l;
            if (c < NU) sm.bb[bloc + m * NU + c] = S.bvec[b0 + (long long)m * NU + c];
          }
        }
        arp = warp_sum(arp); ard = warp_sum(ard); an = warp_sum(an);
        if (lane == 0) {
          prp += (double)arp; prd += (double)ard;
          if (block1) {
            double snew, ptn;
            soc_case(D.p[R] + D.lamp[R], sqrt((double)an), snew, ptn);
            D.s[R] = snew; D.ptn[R] = ptn;
            sm.rowS[r - r0] = (Real)snew; sm.rowOff[r - r0] = loc; sm.rowBOff[r - r0] = bloc; sm.rowT[r - r0] = t;
          }
        }
      }
      __syncthreads();
      // sub-pass 2: Z'_m += Σ_j b_{j,m} w_{j,m}ᵀ, thread per (m, c) pairs, rows of the chunk
      if (block1) {
        const int nr = r1 - r0;
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) {
          const int P = tid + k * NT;
          const int m = P / NX, c = P - m * NX;
          if (m < T) {
            int lo = 0, hi = nr;
            while (lo < hi) { int mid = (lo + hi) >> 1; if (sm.rowT[mid] > m) hi = mid; else lo = mid + 1; }
            for (int q = lo; q < nr; ++q) {
              const int off = sm.rowOff[q] + m * NX + c;
              const Real wv = sm.rowS[q] * sm.eta[off] + sm.uu[off];
              const Real* bq = sm.bb + sm.rowBOff[q] + m * NU;
#pragma unroll
              for (int u = 0; u < NU; ++u) acc[k][u] += bq[u] * wv;
            }
          }
        }
      }
      __syncthreads();
    }
    if (block1) {
#pragma unroll
      for (int k = 0; k < PAIRS; ++k) {
        const int P = tid + k * NT;
        const int m = P / NX, c = P - m * NX;
        if (m < T)
#pragma unroll
          for (int u = 0; u < NU; ++u) ar[L.Zp + (long long)m * NU * NX + u * NX + c] = (double)acc[k][u];
      }
    }
    __syncthreads();
    // ---------------- control rows (one block each; b = ±e_i, b̂ = 0) ----------------
    const int gpk = (I.n_groups > 0) ? I.n_groups / T : 0;
    for (int g = tid; g < I.n_groups; g += NT) {
      const int2 gr = D.groups[I.grp0 + g];
      for (int q = 0; q < gr.y; ++q) {
        const long long R = gr.x + q;
        const int4 ri = D.rinfo[R];
        const int k = ri.x, iu = ri.z;
        const Real sg = (ri.y == ROW_UHI) ? (Real)1 : (Real)-1;
        const long long e0 = D.rent[R];
        const Real sold = (Real)D.s[R];
        Real et[NX], lv[NX];
        Real an = 0;
        double lrp = 0, lrd = 0;
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          const Real y = sg * gtCur[k * GS + iu * NX + c];
          Real l = lam[e0 + c];
          if (!first) {
            const Real yo = sg * gtOld[k * GS + iu * NX + c];
            const Real nu = sold * (yo + l);
            const Real ln = l + y - nu;
            lrp += (double)((y - nu) * (y - nu));
            lrd += (double)((y - yo) * (y - yo));
            l = ln;
            lam[e0 + c] = l;
          }
          lv[c] = l;
          et[c] = y + l;
          an += et[c] * et[c];
        }
        prp += lrp; prd += lrd;
        if (block1) {
          double snew, ptn;
          soc_case(D.p[R] + D.lamp[R], sqrt((double)an), snew, ptn);
          D.s[R] = snew; D.ptn[R] = ptn;
#pragma unroll
          for (int c = 0; c < NX; ++c)
            ar[L.Zp + (long long)k * NU * NX + iu * NX + c] += (double)(sg * ((Real)snew * et[c] - lv[c]));
        }
      }
    }
    double z2 = 0.0, z3 = 0.0;
    block_sum4(prp, prd, z2, z3, sm.red);

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

    // ---------------- Block 1, scalar parts: w (orthant) and e (ball) ----------------
    double en = 0.0, z4 = 0.0, z5 = 0.0, z6 = 0.0;
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const double g0 = S.g0[R];
      const double wn = fmax(0.0, -(g0 + D.ell[R] + D.p[R] + D.lamw[R]));
      D.w[R] = wn;
      D.dd[R] = D.ptn[R] - D.lamp[R] + g0 + wn + D.lamw[R];
    }
    for (int q = tid; q < T * NX; q += NT) {
      const double v = ar[L.dx + NX + q] + ar[L.lam_e + NX + q];
      en += v * v;
    }
    block_sum4(en, z4, z5, z6, sm.red);
    const double escale = (sqrt(en) <= sc[SC_RTRUST]) ? 1.0 : sc[SC_RTRUST] / sqrt(en);
    for (int q = tid; q < T * NX; q += NT) ar[L.e + NX + q] = escale * (ar[L.dx + NX + q] + ar[L.lam_e + NX + q]);
    __syncthreads();

    // ---------------- (c) gain update: K^b from Z' (thread per step) ----------------
    for (int m = tid; m < T; m += NT)
      gain_solve_step<NX, NU, Real>(ar, L, m, I.sqrt_tau, rho * I.sqrt_tau, 0.0, nullptr, ar + L.K1, gtOld, ar + L.Gt1);
    // Riccati linear terms: q_t = 2Q_x(x̂_t - x_g) - ρ(e_t - λ_e,t) + (ρ/2) Σ_{rows at t} d_j a_j
    for (int q = tid; q < T * NX; q += NT) {
      const int t = q / NX + 1, c = q % NX;
      double v = 2.0 * ar[L.Qx + c] * (sa[SL.x_hat + (long long)t * NX + c] - ar[L.xg + c])
                 - rho * (ar[L.e + (long long)t * NX + c] - ar[L.lam_e + (long long)t * NX + c]);
      for (int s2 = 0; s2 < I.rows_per_t; ++s2) {
        const long long rr = (long long)(t - 1) * I.rows_per_t + s2;
        v += 0.5 * rho * D.dd[I.row0 + rr] * S.arow[I.arow0 + rr * NX + c];
      }
      ar[L.qv + (long long)t * NX + c] = v;
    }
    //   r_k = 2R_u(û_k - u_ref) + (ρ/2) Σ_{control rows at (k,i)} σ_j d_j e_i
    for (int q = tid; q < T * NU; q += NT) {
      const int k = q / NU, iu = q % NU;
      double v = 2.0 * ar[L.Ru + iu] * (sa[SL.u_hat + q] - ar[L.uref + iu]);
      if (gpk > 0) {
        for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
          const int2 gr = D.groups[I.grp0 + g];
          for (int qq = 0; qq < gr.y; ++qq) {
            const int4 ri = D.rinfo[gr.x + qq];
            if (ri.z == iu) v += 0.5 * rho * ((ri.y == ROW_UHI) ? 1.0 : -1.0) * D.dd[gr.x + qq];
          }
        }
      }
      ar[L.rv + q] = v;
    }
    for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.dx_prev + q] = ar[L.dx + q];
    __syncthreads();
    { Real* t2 = gtOld; gtOld = gtCur; gtCur = t2; }
    // ---------------- (b) Block 2: Riccati sweep (warp 0) ----------------
    if (warp == 0) riccati_sweep<NX, NU, Real>(ar, L, sa, SL, T, sm.vec);
    __syncthreads();
    // ---------------- (d) p, scalar duals, scalar residual parts of iteration b ----------------
    double a_rp = 0, a_rd = 0, a_rpp = 0, a_rdp = 0;
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const int4 ri = D.rinfo[R];
      double eln;
      if (r < I.n_sr) {
        eln = 0.0;
        for (int c = 0; c < NX; ++c) eln += S.arow[I.arow0 + (long long)r * NX + c] * ar[L.dx + (long long)ri.x * NX + c];
      } else {
        eln = ((ri.y == ROW_UHI) ? 1.0 : -1.0) * ar[L.du + (long long)ri.x * NU + ri.z];
      }
      const double g0 = S.g0[R], ptn = D.ptn[R], wv = D.w[R];
      const double pn = 0.5 * ((ptn - D.lamp[R]) - (g0 + eln + wv + D.lamw[R]));
      const double dp = pn - D.p[R];
      const double c3 = g0 + eln + pn + wv;
      a_rp += (pn - ptn) * (pn - ptn) + c3 * c3;
      a_rd += dp * dp + (eln - D.ell[R] + dp) * (eln - D.ell[R] + dp);
      a_rpp += (pn - ptn) * (pn - ptn);
      a_rdp += (ptn - D.pt[R]) * (ptn - D.pt[R]);
      D.lamp[R] += pn - ptn;
      D.lamw[R] += c3;
      D.p[R] = pn; D.pt[R] = ptn; D.ell[R] = eln;
    }
    for (int q = tid; q < T * NX; q += NT) {
      const double dxv = ar[L.dx + NX + q], ev = ar[L.e + NX + q];
      a_rp += (dxv - ev) * (dxv - ev);
      ar[L.lam_e + NX + q] += dxv - ev;
    }
    for (int q = tid; q < (T + 1) * NX; q += NT) {
      const double d = ar[L.dx + q] - ar[L.dx_prev + q];
      a_rd += d * d;
    }
    block_sum4(a_rp, a_rd, a_rpp, a_rdp, sm.red);
    if (tid == 0) { sc[SC_SCAL_RP] = a_rp; sc[SC_SCAL_RD] = a_rd; sc[SC_SCAL_RPP] = a_rpp; sc[SC_SCAL_RDP] = a_rdp; }
    __syncthreads();
  }
  if (tid == 0) {
    sc[SC_RP] = r_p; sc[SC_RD] = r_d;
    sc[SC_RPP] = sqrt(sc[SC_SCAL_RPP]); sc[SC_RDP] = rho * sqrt(sc[SC_SCAL_RDP]);
    isr[IS_STATUS] = status; isr[IS_ITERS] = iters; isr[IS_CUMITERS] += iters;
  }
  __syncthreads();
}

template <int NX, int NU, typename Real>
__global__ void __launch_bounds__(FACfg<NX, NU>::NT, 1) k_fulladmm(Dev<Real> D, SolveParams sp) {
  extern __shared__ __align__(16) char smem_raw[];
  FASmem<NX, NU, Real> sm;
  sm.carve(smem_raw, sp.tmax, sp.chunk, sp.max_rows);
  __shared__ int s_next;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(D.queue + sp.queue_idx, 1);
    __syncthreads();
    const int q = s_next;
    __syncthreads();
    if (q >= sp.n_order) break;
    fulladmm_instance<NX, NU, Real>(D, sp, D.order[sp.order0 + q], sm);
  }
}

}  // namespace nrto
