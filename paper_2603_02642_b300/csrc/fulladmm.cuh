// NRTO-FullADMM inner loop (Sec. IV, Algorithm 1, Supplementary Sec. III) as one persistent
// kernel: a CTA owns an instance for all its iterations (instances come from a work queue, largest
// first).  Per iteration, over the ragged rows of the instance:
//   (a) Block 1: per row, η̂_j = Â_j k + b̂_j + λ_ν,j, t̂_j = p_j + λ_p,j, SOC projection
//       (ν_j, p̃_j) = Π(η̂_j, t̂_j) = (s_j η̂_j, p̃_j); lifted slacks w (orthant) and e (ball);
//   (c) gain update k = M ρ Σ_j Â_jᵀ(ν_j - b̂_j - λ_ν,j): the Σ is accumulated per step m as
//       Z'_m = Σ_j b_{j,m} w_{j,m}ᵀ, then K_m is solved with the per-step eigen factors;
//   (b) Block 2 (δû, p): Riccati backward/forward sweep with the factorization fixed per outer step;
//   (d) duals λ_p, λ_ν, λ_w, λ_e and the primal/dual residual reductions.
//
// Row state kept between iterations is λ_ν only (plus one scale s_j per row): ν^l = s^l(y^{l-1}+λ^{l-1})
// is recomputed from the gains (y = Â_j k + b̂_j), so the λ_ν update of iteration l is done during the
// row pass of iteration l+1, which also yields the row parts of iteration l's residuals.  Termination
// at iteration l therefore happens after that pass; iteration l+1's block-1 results are discarded.
//
// Row pass data flow: the rows are cut into chunks of whole rows; each chunk's λ, b̂, b ranges and its
// row metadata arrive in shared memory by bulk copies (double buffered, mbarrier completion).  Thread
// `tid` owns the (block m, component c) columns P = tid + k·NT of the ζ-layout for every row, and keeps
// the gain tables Gtᵀ_m[:, c] (= √τ K_m Ψ_mᵀ) of the current and previous iterate and its Z'_m[:, c]
// accumulators in registers across all rows, so the row data is read from shared memory once per
// sub-pass and the gain tables are never re-read.  Row norms are reduced by warp shuffles and a
// fixed-order sum over warps (deterministic).
#pragma once
#include "linearize.cuh"
#include "tma.cuh"

namespace nrto {

struct SolveParams {
  int kv_pcg_iters;                     // k_v update by Jacobi-PCG with this cap (0: exact per-step solve)
  double kv_pcg_tol;
  double rho, eps_p, eps_d;
  double alpha, r_chi, sigma, eps_dr;   // DR
  int max_iter, check, warm, max_dr;
  int chunk, max_rows, tmax, n_order;   // chunk entries, rows per chunk, max T of the launch, instances
  int order0, queue_idx;
  int adapt_every, stall_every;         // residual balancing / stall stop periods (0 = off)
  int fallback;                         // warm start: rerun cold when the warm-started run stalls
  double adapt_mu, adapt_tau, rho_min, rho_max, stall_ratio;
  double stall_budget;                  // budget stop factor at the stall checkpoints (0 = off)
};

// Solver CTA shape for the compute precision float (threads, resident CTAs per SM); FP64 uses 512 × 1.
#ifndef NRTO_FA_NT_F32
#define NRTO_FA_NT_F32 512
#endif
#ifndef NRTO_FA_EM
#define NRTO_FA_EM 1
#endif
#ifndef NRTO_FA_RB
#define NRTO_FA_RB 4
#endif
#ifndef NRTO_FA_MINB_F32
#define NRTO_FA_MINB_F32 1
#endif
// consecutive components of a ζ-block per thread in the quadcopter's row pass (2, 3 or 4; 12 = NCG·W)
#ifndef NRTO_FA_W_QUAD
#define NRTO_FA_W_QUAD 2
#endif

// The unicycle's CTA shape in the compute precision float (its rows need at most 128 threads per row
// group up to T = 254, so two 256-thread CTAs can share an SM).
#ifndef NRTO_FA_NT_UNI
#define NRTO_FA_NT_UNI NRTO_FA_NT_F32
#endif
#ifndef NRTO_FA_MINB_UNI
#define NRTO_FA_MINB_UNI NRTO_FA_MINB_F32
#endif

template <int NX, int NU, typename Real>
struct FACfg {
  static constexpr bool UNI32 = sizeof(Real) == 4 && NX == 3;
  static constexpr int NT = UNI32 ? NRTO_FA_NT_UNI : (sizeof(Real) == 4 ? NRTO_FA_NT_F32 : 512);
  static constexpr int MINB = UNI32 ? NRTO_FA_MINB_UNI : (sizeof(Real) == 4 ? NRTO_FA_MINB_F32 : 1);   // resident CTAs per SM
  static constexpr int NW = NT / 32;
  static constexpr int TMAXC = (NX == 3) ? 256 : (NX == 12 ? 160 : 128);
  static constexpr int W = (NX == 3) ? 3 : (NX == 12 ? NRTO_FA_W_QUAD : 2);   // components of a block per thread
  static constexpr int NCG = NX / W;                     // column groups per ζ-block
  static constexpr int PAIRS = 2;                        // a thread owns blocks m and T - m
  static constexpr int NPAIR_MAX = TMAXC / 2 + 1;        // block pairs of the longest horizon
  static constexpr int TPG_MAX = (NPAIR_MAX * NCG + 31) / 32 * 32;   // threads of one row group
  static constexpr int NWR_MAX = TPG_MAX / 32;           // warps of a row group (partial row norms)
  static constexpr int RB = NRTO_FA_RB;                  // rows per warp reduction in sub-pass 1
  // Sub-pass 1 with a warp per row and lanes over the row's entries, the two gain tables in shared
  // memory ([m][c][u], u padded to NUP), for small blocks (n_x·n_u ≤ 8: the unicycle).  Its rows are
  // short and many per chunk, so warps stay balanced and the tables are small.  With n_x = 12 it
  // measured 9% slower than the column-owned pass (62 KB of tables shrink the chunks, and a chunk's
  // ~10 rows of 24..1932 entries leave warps idle), and 38% slower with rows split into segments.
  static constexpr int NUP = NU <= 2 ? 2 : (NU <= 4 ? 4 : 8);
  static constexpr bool EM = NRTO_FA_EM && NX * NU <= 8;
  static constexpr int GT_COUNT = EM ? 2 * (TMAXC + 1) * NX * NUP : 0;   // values of the two tables
};

// Column ownership in the row pass for an instance of horizon T.  Rows at time t hold blocks
// m = 0..t; thread lt of a row group owns components c .. c+W-1 of block m1 = lt / NCG and of its
// mirror m2 = T - m1, so that over rows of all lengths every thread has about the same work.  A
// row group is tpg = roundup32(npair·NCG) threads; ng groups work on different rows of a chunk.
struct ColMap {
  int grp, ng, nwr, ck;
  int mk[2];
};
template <int NX, int NU, typename Real>
__device__ __forceinline__ ColMap col_map(int T, int zcap) {
  using C = FACfg<NX, NU, Real>;
  ColMap cm;
  const int npair = T / 2 + 1;
  const int tpg = (npair * C::NCG + 31) / 32 * 32;
  int ng = C::NT / tpg;
  if (ng < 1) ng = 1;
  if (ng > zcap) ng = zcap > 0 ? zcap : 1;
  cm.ng = ng;
  cm.nwr = tpg / 32;
  const int tid = threadIdx.x;
  cm.grp = tid / tpg;
  const int lt = tid - cm.grp * tpg;
  constexpr int OFF = 1 << 20;   // no row reaches this block index
  if (cm.grp >= ng || lt >= npair * C::NCG) {
    cm.mk[0] = OFF; cm.mk[1] = OFF; cm.ck = 0;
    if (cm.grp >= ng) cm.grp = OFF;   // idle thread: no rows
  } else {
    const int m1 = lt / C::NCG;
    cm.ck = (lt - m1 * C::NCG) * C::W;
    cm.mk[0] = m1;
    cm.mk[1] = (T - m1 != m1) ? T - m1 : OFF;
  }
  return cm;
}

// Sums RB per-lane values over the warp in one butterfly: the first log2(RB) levels halve the set
// of values each lane carries (a lane keeps the half selected by its lane bit and sends the other),
// the remaining levels are a plain butterfly.  Lanes [r·32/RB, (r+1)·32/RB) return the sum of
// v[r]; every sum uses the same pairing tree as warp_sum.
template <int RB, typename T>
__device__ __forceinline__ T warp_sum_rows(const T (&v)[RB], int lane) {
  static_assert(RB == 1 || RB == 2 || RB == 4, "RB must be 1, 2 or 4");
  if constexpr (RB == 1) {
    return warp_sum(v[0]);
  } else if constexpr (RB == 2) {
    const bool hi = (lane & 16) != 0;
    T a = hi ? v[1] : v[0];
    a += __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[1], 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  } else {
    const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
    T a0 = h4 ? v[2] : v[0], a1 = h4 ? v[3] : v[1];
    a0 += __shfl_xor_sync(0xffffffffu, h4 ? v[0] : v[2], 16);
    a1 += __shfl_xor_sync(0xffffffffu, h4 ? v[1] : v[3], 16);
    T a = h3 ? a1 : a0;
    a += __shfl_xor_sync(0xffffffffu, h3 ? a0 : a1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    return a;
  }
}

// Supplementary Sec. II-C closed form: (t̂, η̂) ↦ (p̃, s·η̂), a = ‖η̂‖
__device__ __forceinline__ void soc_case(double tt, double a, double& s_new, double& pt_new) {
  if (a <= tt) { s_new = 1.0; pt_new = tt; }
  else if (a <= -tt) { s_new = 0.0; pt_new = 0.0; }
  else { pt_new = 0.5 * (tt + a); s_new = pt_new / a; }
}
template <typename Real>
__device__ __forceinline__ void soc_case_r(Real tt, Real a, Real& s_new, Real& pt_new) {
  if (a <= tt) { s_new = (Real)1; pt_new = tt; }
  else if (a <= -tt) { s_new = (Real)0; pt_new = (Real)0; }
  else { pt_new = (Real)0.5 * (tt + a); s_new = pt_new / a; }
}

// Per-warp shared scratch of the FullADMM gain solve (gain_solve_warps): the step's operands and
// two intermediates, in compute precision.
template <int NX, int NU, typename Real>
struct GainScratch {
  static constexpr int NE = NU * NX;
  static constexpr int oPhi = 0, oU = NX * NX, oPf = 2 * NX * NX, oDv = oPf + NU * NU, oZ = oDv + NE;
  static constexpr int oY = oZ + NE, oX = oY + NE, PER_WARP = (oX + NE + 3) / 4 * 4;   // values per warp
  // gain warps whose scratch fits in about 32 KB (at least one)
  static constexpr int warps(int avail) {
    const int cap = (int)((32 * 1024) / (PER_WARP * sizeof(Real)));
    const int w = avail < cap ? avail : cap;
    return w > 0 ? w : 1;
  }
};

// Shared memory of one CTA: two chunk buffers plus per-chunk scratch.  Host and device use the
// same size function.
template <int NX, int NU, typename Real>
struct FASmem {
  struct Buf {
    Real* lam; Real* bhat; Real* bb; RowMeta* meta;
    Real* so;   // the chunk's row scales s_j (storage order) from a 16-byte-aligned window
  };
  // elements of the row-scale window in front of a chunk's first row
  static constexpr int SO_ALIGN = 16 / (int)sizeof(Real);
  Buf buf[2];
  Real* rowpart;   // [max_rows][NWR_MAX] warp partial norms; in block 2 the gain solve's per-warp scratch
  Real* snew;      // [max_rows]
  Real* gts;       // the gain tables of an entry-major sub-pass 1 (FACfg::GT_COUNT values)
  double* red;     // block reductions
  double* vec;     // Riccati sweep vector

  NRTO_HD static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
  NRTO_HD static size_t rowpart_count(int max_rows) {
    using G = GainScratch<NX, NU, Real>;
    const size_t a = (size_t)max_rows * FACfg<NX, NU, Real>::NWR_MAX;
    const size_t g = (size_t)G::warps(FACfg<NX, NU, Real>::NW - 1) * G::PER_WARP;
    return a > g ? a : g;
  }
  NRTO_HD static size_t buf_bytes(int chunk, int max_rows) {
    size_t b = 0;
    b += align16((size_t)(chunk + 4) * sizeof(Real));            // lam
    b += align16((size_t)(chunk + 4) * sizeof(Real));            // bhat
    b += align16((size_t)(chunk / NX * NU + 8) * sizeof(Real));  // b
    b += align16((size_t)max_rows * sizeof(RowMeta));            // meta
    b += align16((size_t)(max_rows + 2 * SO_ALIGN) * sizeof(Real));   // row scales
    return b;
  }
  NRTO_HD static size_t bytes(int chunk, int max_rows) {
    size_t b = 2 * buf_bytes(chunk, max_rows);
    b += align16(rowpart_count(max_rows) * sizeof(Real));
    b += align16((size_t)max_rows * sizeof(Real));
    b += align16((size_t)FACfg<NX, NU, Real>::GT_COUNT * sizeof(Real));
    b += (4 * FACfg<NX, NU, Real>::NW + 4 * 16) * sizeof(double);
    return b;
  }
  // Row groups whose Z' partials fit in the (then idle) chunk buffers for horizon T.
  NRTO_HD static int zcap(int chunk, int max_rows, int T) {
    return (int)(2 * buf_bytes(chunk, max_rows) / sizeof(Real) / ((size_t)T * NU * NX));
  }
  __device__ void carve(char* base, int chunk, int max_rows) {
    char* c = base;
    auto take = [&](size_t bytes) { char* r = c; c += align16(bytes); return r; };
    for (int k = 0; k < 2; ++k) {
      buf[k].lam = reinterpret_cast<Real*>(take((size_t)(chunk + 4) * sizeof(Real)));
      buf[k].bhat = reinterpret_cast<Real*>(take((size_t)(chunk + 4) * sizeof(Real)));
      buf[k].bb = reinterpret_cast<Real*>(take((size_t)(chunk / NX * NU + 8) * sizeof(Real)));
      buf[k].meta = reinterpret_cast<RowMeta*>(take((size_t)max_rows * sizeof(RowMeta)));
      buf[k].so = reinterpret_cast<Real*>(take((size_t)(max_rows + 2 * SO_ALIGN) * sizeof(Real)));
    }
    rowpart = reinterpret_cast<Real*>(take(rowpart_count(max_rows) * sizeof(Real)));
    snew = reinterpret_cast<Real*>(take((size_t)max_rows * sizeof(Real)));
    gts = reinterpret_cast<Real*>(take((size_t)FACfg<NX, NU, Real>::GT_COUNT * sizeof(Real)));
    red = reinterpret_cast<double*>(c);
    vec = red + 4 * FACfg<NX, NU, Real>::NW;
  }
};

// Issue the bulk copies of one chunk into a buffer (one thread): the entry ranges of λ and b̂,
// the b range, the chunk's row metadata (state rows in storage order, logical index in .pad) and
// its row scales.  The row scales are kept in storage order; their window starts at the 16-byte
// boundary at or before the chunk's first row (so_offset() elements earlier) and is rounded up to a
// 16-byte multiple, which stays inside the array's 4-element tail padding.
template <int NX, int NU, typename Real>
__device__ __forceinline__ int so_offset(const Inst& I, const ChunkInfo& ck) {
  return (int)((I.row0 + ck.r0) & (FASmem<NX, NU, Real>::SO_ALIGN - 1));
}
template <int NX, int NU, typename Real>
__device__ void issue_chunk(const Dev<Real>& D, const LinSlot<Real>& S, const Inst& I, const ChunkInfo& ck,
                            const typename FASmem<NX, NU, Real>::Buf& bf, uint64_t* bar) {
  constexpr int A = FASmem<NX, NU, Real>::SO_ALIGN;
  const int nr = ck.r1 - ck.r0, so0 = so_offset<NX, NU, Real>(I, ck);
  const uint32_t bl = (uint32_t)(ck.ne * sizeof(Real)), bbb = (uint32_t)(ck.nb * sizeof(Real));
  const uint32_t bm = (uint32_t)(nr * sizeof(RowMeta));
  const uint32_t bs = (uint32_t)(((so0 + nr + A - 1) & ~(A - 1)) * sizeof(Real));
  mbar_arrive_expect_tx(bar, 2 * bl + bbb + bm + bs);
  // the row streams are read once per pass: first to leave L2
  const uint64_t pol = l2_policy_evict_first();
  bulk_g2s_hint(bf.lam, D.lam + ck.e0, bl, bar, pol);
  bulk_g2s_hint(bf.bhat, S.bhat + ck.e0, bl, bar, pol);
  bulk_g2s_hint(bf.bb, S.bvec + ck.b0, bbb, bar, pol);
  bulk_g2s(bf.meta, D.rmeta + I.row0 + ck.r0, bm, bar);
  bulk_g2s(bf.so, D.sr + (I.row0 + ck.r0 - so0), bs, bar);
}

// Per-step gain solve, parallel over (m, u, c) in four phases through arena scratch:
//   Y = coefA Z' Φ + coefK K̃ U;  X = (Pfᵀ Y) ⊙ Dv;  PX = Pf X;  K = PX Uᵀ;  Gtᵀ = √τ PX Φᵀ.
// (FullADMM: coefA = ρ√τ, coefK = 0; DR: coefA = σ√τ, coefK = r_χ.)  All threads of the block.
// Threads t0 .. t0+nthr-1 take part; they synchronize with barrier `bar_id` (0: the whole block).
__device__ __forceinline__ void group_sync(int bar_id, int nthr) {
  if (bar_id == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
}

template <int NX, int NU, typename Real>
__device__ __noinline__ void gain_solve(double* ar, const Arena& L, int T, double sqrt_tau, double coefA, double coefK,
                           double* Kout, double* gt_out, int t0 = 0, int nthr = 0, int bar_id = 0) {
  const int n = T * NU * NX;
  if (nthr == 0) nthr = blockDim.x;
  const int me = threadIdx.x - t0;
  for (int q = me; q < n; q += nthr) {
    const int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    const double* Zp = ar + L.Zp + (long long)m * NU * NX + u * NX;
    const double* Phi = ar + L.Phi + (long long)m * NX * NX;
    Real acc = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r) acc += (Real)Zp[r] * (Real)Phi[r * NX + c];
    acc *= (Real)coefA;
    if (coefK != 0.0) {
      const double* Kt = ar + L.Kt + (long long)m * NU * NX + u * NX;
      const double* U = ar + L.SigU + (long long)m * NX * NX;
      Real a2 = 0;
#pragma unroll
      for (int r = 0; r < NX; ++r) a2 += (Real)Kt[r] * (Real)U[r * NX + c];
      acc += (Real)coefK * a2;
    }
    ar[L.Ws1 + q] = (double)acc;
  }
  group_sync(bar_id, nthr);
  for (int q = me; q < n; q += nthr) {
    const int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    const double* Pf = ar + L.Pf + (long long)m * NU * NU;
    const double* Y = ar + L.Ws1 + (long long)m * NU * NX;
    Real acc = 0;
#pragma unroll
    for (int v = 0; v < NU; ++v) acc += (Real)Pf[v * NU + u] * (Real)Y[v * NX + c];
    ar[L.Ws2 + q] = (double)(acc * (Real)ar[L.Dv + q]);
  }
  group_sync(bar_id, nthr);
  for (int q = me; q < n; q += nthr) {
    const int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    const double* Pf = ar + L.Pf + (long long)m * NU * NU;
    const double* X = ar + L.Ws2 + (long long)m * NU * NX;
    Real acc = 0;
#pragma unroll
    for (int v = 0; v < NU; ++v) acc += (Real)Pf[u * NU + v] * (Real)X[v * NX + c];
    ar[L.Ws1 + q] = (double)acc;
  }
  group_sync(bar_id, nthr);
  for (int q = me; q < n; q += nthr) {
    const int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    const double* PX = ar + L.Ws1 + (long long)m * NU * NX + u * NX;
    const double* U = ar + L.SigU + (long long)m * NX * NX + c * NX;
    const double* Phi = ar + L.Phi + (long long)m * NX * NX + c * NX;
    Real k = 0, g = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      const Real px = (Real)PX[r];
      k += px * (Real)U[r];
      g += px * (Real)Phi[r];
    }
    Kout[q] = (double)k;
    gt_out[q] = (double)(g * (Real)sqrt_tau);
  }
  for (int q = me; q < NU * NX; q += nthr) gt_out[(long long)T * NU * NX + q] = 0.0;
  group_sync(bar_id, nthr);
}

// The FullADMM gain solve (coefK = 0) with one warp per step: warps w0 .. w0+nw-1 take steps
// m = w - w0, w - w0 + nw, ...  A warp first stages its step's operands (Z', Φ, U = Σ_U, P_f, D_v)
// into its shared scratch as compute-precision values with coalesced, independent loads, then runs
// the four products of gain_solve from shared memory, so no block-wide barrier separates them and
// each operand costs one memory latency per step.  Every element is summed in the same order as in
// gain_solve from the same compute-precision values, so the results are identical.

template <int NX, int NU, typename Real>
__device__ __forceinline__ void gain_solve_warps(const double* ar, const Arena& L, int T, double sqrt_tau, double coefA,
                                                 double* Kout, double* gt_out, int w0, int nw, Real* scr) {
  using G = GainScratch<NX, NU, Real>;
  constexpr int NE = G::NE, EPL = (NE + 31) / 32;
  const int lane = threadIdx.x & 31, wv = (int)(threadIdx.x >> 5) - w0;
  if (wv < 0 || wv >= nw) return;
  Real* const sw = scr + (size_t)wv * G::PER_WARP;
  Real* const sPhi = sw + G::oPhi;
  Real* const sU = sw + G::oU;
  Real* const sPf = sw + G::oPf;
  Real* const sDv = sw + G::oDv;
  Real* const sZ = sw + G::oZ;
  Real* const Y = sw + G::oY;   // Y, then PX
  Real* const X = sw + G::oX;
  const Real cA = (Real)coefA, st = (Real)sqrt_tau;
  for (int m = wv; m < T; m += nw) {
    {
      const double* Phi = ar + L.Phi + (long long)m * NX * NX;
      const double* U = ar + L.SigU + (long long)m * NX * NX;
      const double* Pf = ar + L.Pf + (long long)m * NU * NU;
      const double* Dv = ar + L.Dv + (long long)m * NE;
      const double* Zp = ar + L.Zp + (long long)m * NE;
      for (int q = lane; q < NX * NX; q += 32) { sPhi[q] = (Real)Phi[q]; sU[q] = (Real)U[q]; }
      for (int q = lane; q < NU * NU; q += 32) sPf[q] = (Real)Pf[q];
      for (int q = lane; q < NE; q += 32) { sDv[q] = (Real)Dv[q]; sZ[q] = (Real)Zp[q]; }
    }
    __syncwarp();
    // Y = coefA Z' Φ
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = lane + 32 * i;
      if (e < NE) {
        const int u = e / NX, c = e - u * NX;
        Real acc = 0;
#pragma unroll
        for (int r = 0; r < NX; ++r) acc += sZ[u * NX + r] * sPhi[r * NX + c];
        acc *= cA;
        Y[e] = acc;
      }
    }
    __syncwarp();
    // X = (P_fᵀ Y) ⊙ D_v
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = lane + 32 * i;
      if (e < NE) {
        const int u = e / NX, c = e - u * NX;
        Real acc = 0;
#pragma unroll
        for (int v = 0; v < NU; ++v) acc += sPf[v * NU + u] * Y[v * NX + c];
        X[e] = acc * sDv[e];
      }
    }
    __syncwarp();
    // PX = P_f X (into Y)
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = lane + 32 * i;
      if (e < NE) {
        const int u = e / NX, c = e - u * NX;
        Real acc = 0;
#pragma unroll
        for (int v = 0; v < NU; ++v) acc += sPf[u * NU + v] * X[v * NX + c];
        Y[e] = acc;
      }
    }
    __syncwarp();
    // K = PX Uᵀ,  Gtᵀ = √τ PX Φᵀ
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = lane + 32 * i;
      if (e < NE) {
        const int u = e / NX, c = e - u * NX;
        Real k = 0, g = 0;
#pragma unroll
        for (int r = 0; r < NX; ++r) {
          const Real px = Y[u * NX + r];
          k += px * sU[c * NX + r];
          g += px * sPhi[c * NX + r];
        }
        Kout[(long long)m * NE + e] = (double)k;
        gt_out[(long long)m * NE + e] = (double)(g * st);
      }
    }
    __syncwarp();
  }
  if (wv == 0)
    for (int q = lane; q < NE; q += 32) gt_out[(long long)T * NE + q] = 0.0;
}

// The k_v update by matrix-free Jacobi-preconditioned conjugate gradients (Sec. IV: the k_v update
// by PCG), run by threads 32 .. blockDim-1 with named barrier 1 while warp 0 runs the block-2 sweep.
// System: (H X)_m = 2 R_KᵀR_K X_m + ρτ G_m X_m Σ_m = R_m = ρ√τ Z'_m Ψ_m (the same right-hand side as
// the exact per-step solve); preconditioner: the diagonal 2 (R_K)_u² + ρτ (G_m)_uu (Σ_m)_cc.  Starts
// from the gains in Kout, stops before an iteration when ‖R - H X‖ ≤ tol ‖R‖ or after max_iter
// iterations, leaves X in Kout and its table √τ X_m Ψ_mᵀ in gt_out.  FP64.  Returns the iterations.
struct PcgArgs {
  int max_iter;
  double tol, rho, tau;
  const double* Gm;      // slot arena's G_m blocks (T × nu × nu)
  double* red;           // shared scratch: 3 × (warps) doubles
};

template <int NX, int NU>
__device__ __noinline__ int gain_pcg_group(double* ar, const Arena& L, int T, double sqrt_tau, const PcgArgs& pa,
                                           double* Kout, double* gt_out) {
  constexpr int NE = NU * NX;
  const int me = threadIdx.x - 32, ng = blockDim.x - 32, n = T * NE;
  const int lane = threadIdx.x & 31, gw = me >> 5, nwg = ng >> 5;
  double* x = Kout;
  double* r = ar + L.Ws1;
  double* p = ar + L.Ws2;
  double* Ap = ar + L.Pc1;
  const double* Sig = ar + L.Sigma;
  const double* RK = ar + L.RK;
  const double ct = pa.rho * pa.tau;
  auto hop = [&](const double* v, int q) {
    const int m = q / NE, u = (q / NX) % NU, c = q % NX;
    const double* vm = v + (long long)m * NE;
    const double* G = pa.Gm + (long long)m * NU * NU + u * NU;
    const double* S = Sig + (long long)m * NX * NX;
    double acc = 0.0;
    for (int w = 0; w < NU; ++w) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < NX; ++k) t += vm[w * NX + k] * S[k * NX + c];
      acc += G[w] * t;
    }
    return 2.0 * RK[u] * RK[u] * v[q] + ct * acc;
  };
  auto dinv = [&](int q) {
    const int m = q / NE, u = (q / NX) % NU, c = q % NX;
    return 1.0 / (2.0 * RK[u] * RK[u] + ct * pa.Gm[(long long)m * NU * NU + u * NU + u] * Sig[(long long)m * NX * NX + c * NX + c]);
  };
  auto gsum3 = [&](double& a, double& b, double& c) {
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    if (lane == 0) { pa.red[3 * gw] = a; pa.red[3 * gw + 1] = b; pa.red[3 * gw + 2] = c; }
    group_sync(1, ng);
    a = b = c = 0.0;
    for (int w = 0; w < nwg; ++w) { a += pa.red[3 * w]; b += pa.red[3 * w + 1]; c += pa.red[3 * w + 2]; }
    group_sync(1, ng);
  };
  // r = R - H x,  p = D⁻¹ r
  double rn0 = 0.0, rz = 0.0, rr = 0.0;
  for (int q = me; q < n; q += ng) {
    const int m = q / NE, u = (q / NX) % NU, c = q % NX;
    const double* Zp = ar + L.Zp + (long long)m * NE + u * NX;
    const double* Ps = ar + L.Psi + (long long)m * NX * NX;
    double R = 0.0;
#pragma unroll
    for (int k = 0; k < NX; ++k) R += Zp[k] * Ps[k * NX + c];
    R *= pa.rho * sqrt_tau;
    const double rq = R - hop(x, q);
    const double zq = dinv(q) * rq;
    r[q] = rq;
    p[q] = zq;
    rn0 += R * R; rz += rq * zq; rr += rq * rq;
  }
  gsum3(rn0, rz, rr);
  rn0 = sqrt(rn0);
  int it = 0;
  while (it < pa.max_iter && !(sqrt(rr) <= pa.tol * rn0)) {
    double pap = 0.0, z0 = 0.0, z1 = 0.0;
    for (int q = me; q < n; q += ng) {
      const double a = hop(p, q);
      Ap[q] = a;
      pap += p[q] * a;
    }
    gsum3(pap, z0, z1);
    const double alpha = rz / pap;
    double rzn = 0.0, rrn = 0.0, z2 = 0.0;
    for (int q = me; q < n; q += ng) {
      x[q] += alpha * p[q];
      const double rq = r[q] - alpha * Ap[q];
      r[q] = rq;
      rzn += rq * dinv(q) * rq;
      rrn += rq * rq;
    }
    gsum3(rzn, rrn, z2);
    const double beta = rzn / rz;
    for (int q = me; q < n; q += ng) p[q] = dinv(q) * r[q] + beta * p[q];
    group_sync(1, ng);
    rz = rzn;
    rr = rrn;
    ++it;
  }
  // the gain table of the new gains for the row pass: √τ X_m Ψ_mᵀ
  for (int q = me; q < n; q += ng) {
    const int m = q / NE, u = (q / NX) % NU, c = q % NX;
    const double* xm = x + (long long)m * NE + u * NX;
    const double* Ps = ar + L.Psi + (long long)m * NX * NX + c * NX;
    double g = 0.0;
#pragma unroll
    for (int k = 0; k < NX; ++k) g += xm[k] * Ps[k];
    gt_out[q] = sqrt_tau * g;
  }
  for (int q = me; q < NE; q += ng) gt_out[(long long)T * NE + q] = 0.0;
  return it;
}

// Block-2 (δû) LQ sweep with fixed factors (warp 0 only).  Linear terms q_t (t = 0..T, index t
// of qv; q_0 unused) and r_k in the arena.  Writes du, dx.  Arithmetic in Real.
// Each lane keeps the factor rows it needs for one step in registers and loads the next step's rows
// before the current step's dependent arithmetic, so the 2T dependent steps do not each wait for L2.
template <int NX, int NU, typename Real>
__device__ __noinline__ void riccati_sweep(double* ar, const Arena& L, const double* sa, const SlotL& SL, int T, double* pv) {
  const int lane = threadIdx.x & 31;
  // lane j < NX: column j of Acl_k and of L_k, q_k[j];   lane j < NU: row j of N_k and of M_k, r_k
  Real acl[NX], lk[NU], nrow[NU], mrow[NX], rr[NU];
  Real qk = 0;
  auto load_back = [&](int k) {
    const double* N = ar + L.RicN + (long long)k * NU * NU;
    const double* M = ar + L.RicM + (long long)k * NU * NX;
    const double* Lk = ar + L.RicL + (long long)k * NU * NX;
    const double* Acl = ar + L.RicAcl + (long long)k * NX * NX;
    const double* r = ar + L.rv + (long long)k * NU;
#pragma unroll
    for (int v = 0; v < NU; ++v) rr[v] = (Real)r[v];
    if (lane < NX) {
#pragma unroll
      for (int c = 0; c < NX; ++c) acl[c] = (Real)Acl[c * NX + lane];
#pragma unroll
      for (int v = 0; v < NU; ++v) lk[v] = (Real)Lk[v * NX + lane];
      qk = (Real)ar[L.qv + (long long)k * NX + lane];
    }
    if (lane < NU) {
#pragma unroll
      for (int v = 0; v < NU; ++v) nrow[v] = (Real)N[lane * NU + v];
#pragma unroll
      for (int c = 0; c < NX; ++c) mrow[c] = (Real)M[lane * NX + c];
    }
  };
  // backward: l_k = -(N_k r_k + M_k p_{k+1}),  p_k = q_k + Acl_kᵀ p_{k+1} + L_kᵀ r_k
  if (lane < NX) pv[lane] = ar[L.qv + (long long)T * NX + lane];
  load_back(T - 1);
  __syncwarp();
  for (int k = T - 1; k >= 0; --k) {
    Real acl_c[NX], lk_c[NU], n_c[NU], m_c[NX], r_c[NU];
    const Real q_c = qk;
#pragma unroll
    for (int c = 0; c < NX; ++c) { acl_c[c] = acl[c]; m_c[c] = mrow[c]; }
#pragma unroll
    for (int v = 0; v < NU; ++v) { lk_c[v] = lk[v]; n_c[v] = nrow[v]; r_c[v] = rr[v]; }
    if (k >= 1) load_back(k - 1);
    Real p_in[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) p_in[c] = (Real)pv[c];
    if (lane < NU) {
      Real lv = 0;
#pragma unroll
      for (int v = 0; v < NU; ++v) lv += n_c[v] * r_c[v];
#pragma unroll
      for (int c = 0; c < NX; ++c) lv += m_c[c] * p_in[c];
      ar[L.du + (long long)k * NU + lane] = -(double)lv;   // l_k stored in du until the forward pass
    }
    Real pn = q_c;
    if (lane < NX && k >= 1) {
#pragma unroll
      for (int c = 0; c < NX; ++c) pn += acl_c[c] * p_in[c];
#pragma unroll
      for (int v = 0; v < NU; ++v) pn += lk_c[v] * r_c[v];
    }
    __syncwarp();
    if (lane < NX && k >= 1) pv[lane] = (double)pn;
    __syncwarp();
  }
  // forward: δx_0 = 0, δu_k = L_k δx_k + l_k, δx_{k+1} = A_k δx_k + B_k δu_k
  double* dx = ar + L.dx;
  double* du = ar + L.du;
  // lane j < NU: row j of L_k, l_k[j];   lane j < NX: row j of A_k and of B_k
  Real lrow[NX], arow[NX], brow[NU];
  Real lkv = 0;
  auto load_fwd = [&](int k) {
    const double* Lk = ar + L.RicL + (long long)k * NU * NX;
    const double* A = sa + SL.A + (long long)k * NX * NX;
    const double* B = sa + SL.B + (long long)k * NX * NU;
    if (lane < NU) {
#pragma unroll
      for (int c = 0; c < NX; ++c) lrow[c] = (Real)Lk[lane * NX + c];
      lkv = (Real)du[(long long)k * NU + lane];
    }
    if (lane < NX) {
#pragma unroll
      for (int c = 0; c < NX; ++c) arow[c] = (Real)A[lane * NX + c];
#pragma unroll
      for (int v = 0; v < NU; ++v) brow[v] = (Real)B[lane * NU + v];
    }
  };
  Real xk[NX];
#pragma unroll
  for (int c = 0; c < NX; ++c) xk[c] = 0;
  if (lane < NX) dx[lane] = 0.0;
  load_fwd(0);
  for (int k = 0; k < T; ++k) {
    Real l_c[NX], a_c[NX], b_c[NU];
    const Real lk0 = lkv;
#pragma unroll
    for (int c = 0; c < NX; ++c) { l_c[c] = lrow[c]; a_c[c] = arow[c]; }
#pragma unroll
    for (int v = 0; v < NU; ++v) b_c[v] = brow[v];
    if (k + 1 < T) load_fwd(k + 1);
    // every lane holds the full δx_k (xk); δu_k is formed by lanes < NU and broadcast by shuffles
    Real u = lk0;
    if (lane < NU) {
#pragma unroll
      for (int c = 0; c < NX; ++c) u += l_c[c] * xk[c];
      du[(long long)k * NU + lane] = (double)u;
    }
    Real uk[NU];
#pragma unroll
    for (int v = 0; v < NU; ++v) uk[v] = __shfl_sync(0xffffffffu, u, v);
    Real xn = 0;
    if (lane < NX) {
#pragma unroll
      for (int c = 0; c < NX; ++c) xn += a_c[c] * xk[c];
#pragma unroll
      for (int v = 0; v < NU; ++v) xn += b_c[v] * uk[v];
      dx[(long long)(k + 1) * NX + lane] = (double)xn;
    }
#pragma unroll
    for (int c = 0; c < NX; ++c) xk[c] = __shfl_sync(0xffffffffu, xn, c);
  }
  __syncwarp();
}

// Shared-memory areas of the block-2 sweep, cut from the chunk buffers (idle after the row pass):
// linear terms q_t (t = 0..T) and r_k, feed-forward l_k, c_k / d_k, the costates p_t or states δx_t,
// and a two-half ring of packed factor records (pk_stride values per step) that bulk copies fill
// ahead of the serial recursions.
template <int NX, int NU, typename Real>
struct B2Smem {
  Real* qs;    // (T+1)·NX
  Real* rs;    // T·NU
  Real* ls;    // T·NU
  Real* cd;    // T·NX: c_k (backward), then d_k (forward)
  Real* px;    // (T+1)·NX: p_t (backward), then δx_t (forward)
  Real* ring;
  int nbs;     // steps per ring half
  __device__ void carve(char* base, size_t bytes, int T) {
    auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    char* c = base;
    qs = reinterpret_cast<Real*>(c); c += a16((size_t)(T + 1) * NX * sizeof(Real));
    rs = reinterpret_cast<Real*>(c); c += a16((size_t)T * NU * sizeof(Real));
    ls = reinterpret_cast<Real*>(c); c += a16((size_t)T * NU * sizeof(Real));
    cd = reinterpret_cast<Real*>(c); c += a16((size_t)T * NX * sizeof(Real));
    px = reinterpret_cast<Real*>(c); c += a16((size_t)(T + 1) * NX * sizeof(Real));
    ring = reinterpret_cast<Real*>(c);
    const size_t used = (size_t)(c - base);
    const size_t rec = (size_t)pk_stride(NX, NU) * sizeof(Real);
    nbs = used < bytes ? (int)((bytes - used) / (2 * rec)) : 0;
  }
  NRTO_HD static size_t fixed_bytes(int T) {
    auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    return a16((size_t)(T + 1) * NX * sizeof(Real)) + 2 * a16((size_t)T * NU * sizeof(Real)) +
           a16((size_t)T * NX * sizeof(Real)) + a16((size_t)(T + 1) * NX * sizeof(Real));
  }
};

// Block-2 (δû) solve with the fixed factorization and the gain solve (independent of block 2).
// Only the A_cl products are serial in k, so everything else runs in parallel passes over k:
//   c_k = q_k + L_kᵀ r_k                                     (all threads)
//   p_T = q_T,  p_k = c_k + A_cl,kᵀ p_{k+1}                   (warp 0; warps 1.. solve for the gains)
//   l_k = -(N_k r_k + M_k p_{k+1}),  d_k = B_k l_k             (all threads)
//   δx_0 = 0,  δx_{k+1} = A_cl,k δx_k + d_k                    (warp 0)
//   δu_k = L_k δx_k + l_k                                     (all threads)
// which is the Riccati backward/forward sweep (δx_{k+1} = A_k δx_k + B_k δu_k) reordered.  The
// records for the serial passes stream through the ring by bulk copies (lane 0 of warp 0, mbarriers
// `bars` with phases `phase`); the parallel passes read the records from global memory.  Returns
// false if a copy did not arrive.
template <int NX, int NU, typename Real>
__device__ __noinline__ bool block2_sweep_and_gain(double* ar, const Arena& L, int T, const B2Smem<NX, NU, Real> b2,
                                                   uint64_t* bars, uint32_t* phase, int* s_flag, Real* gscr,
                                                   const double* gargs, double* Kout, double* gt_out,
                                                   const PcgArgs& pcg, int* pcg_iters) {
  constexpr int BW = pk_stride(NX, NU);
  constexpr int oM = NU * NU, oL = oM + NU * NX, oA = oL + NU * NX, oB = oA + NX * NX;
  const int tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
  const Real* pk = reinterpret_cast<const Real*>(ar + L.RicPk);
  const int nbs = b2.nbs;
  const int nblk = (T + nbs - 1) / nbs;
  // one block of records [lo, hi] into ring half h (lane 0 of warp 0)
  auto issue = [&](int lo, int hi, int h) {
    const uint32_t bytes = (uint32_t)((hi - lo + 1) * BW * sizeof(Real));
    mbar_arrive_expect_tx(&bars[h], bytes);
    bulk_g2s(b2.ring + (size_t)h * nbs * BW, pk + (size_t)lo * BW, bytes, &bars[h]);
  };
  auto wait = [&](int h) {
    int got = 1;
    if (lane == 0) got = mbar_wait_bounded(&bars[h], phase[h]) ? 1 : 0;
    got = __shfl_sync(0xffffffffu, got, 0);
    phase[h] ^= 1u;
    return got != 0;
  };
  auto bwd_lo = [&](int j) { const int hi = T - 1 - j * nbs; return hi - nbs + 1 > 0 ? hi - nbs + 1 : 0; };
  if (tid == 0) {
    // the ring reuses chunk-buffer memory last written by generic stores
    fence_proxy_async();
    issue(bwd_lo(0), T - 1, 0);
    if (nblk > 1) issue(bwd_lo(1), T - 1 - nbs, 1);
  }
  // ---- c_k = q_k + L_kᵀ r_k ----
  for (int q = tid; q < T * NX; q += nthr) {
    const int k = q / NX, j = q - k * NX;
    const Real* f = pk + (size_t)k * BW;
    Real v = b2.qs[(size_t)k * NX + j];
#pragma unroll
    for (int u = 0; u < NU; ++u) v += f[oL + u * NX + j] * b2.rs[(size_t)k * NU + u];
    b2.cd[q] = v;
  }
  __syncthreads();
  bool ok = true;
  if (tid >= 32) {
    if (pcg.max_iter > 0) {
      const int it = gain_pcg_group<NX, NU>(ar, L, T, gargs[0], pcg, Kout, gt_out);
      if (tid == 32) *pcg_iters += it;
    } else {
      gain_solve_warps<NX, NU, Real>(ar, L, T, gargs[0], gargs[1], Kout, gt_out, 1,
                                     GainScratch<NX, NU, Real>::warps(nthr / 32 - 1), gscr);
    }
  } else {
    // ---- backward: p_k = c_k + A_cl,kᵀ p_{k+1}; lane j < NX owns p_j ----
    Real p = (lane < NX) ? b2.qs[(size_t)T * NX + lane] : (Real)0;
    if (lane < NX) b2.px[(size_t)T * NX + lane] = p;
    for (int j = 0; j < nblk && ok; ++j) {
      const int h = j & 1, hi = T - 1 - j * nbs, lo = bwd_lo(j);
      if (!wait(h)) { ok = false; break; }
      const Real* base = b2.ring + (size_t)h * nbs * BW;
      for (int k = hi; k >= lo; --k) {
        const Real* A = base + (size_t)(k - lo) * BW + oA;
        Real pc[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) pc[c] = __shfl_sync(0xffffffffu, p, c);
        if (k >= 1) {
          Real s0 = (lane < NX) ? b2.cd[(size_t)k * NX + lane] : (Real)0, s1 = 0;
          if (lane < NX) {
#pragma unroll
            for (int c = 0; c < NX; c += 2) {
              s0 += A[c * NX + lane] * pc[c];
              if (c + 1 < NX) s1 += A[(c + 1) * NX + lane] * pc[c + 1];
            }
          }
          p = s0 + s1;
          if (lane < NX) b2.px[(size_t)k * NX + lane] = p;
        }
      }
      __syncwarp();
      if (lane == 0 && j + 2 < nblk) {
        fence_proxy_async();
        issue(bwd_lo(j + 2), T - 1 - (j + 2) * nbs, h);
      }
    }
    if (lane == 0) *s_flag = ok ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  // forward records into the ring while l_k and d_k are formed
  if (tid == 0) {
    fence_proxy_async();
    issue(0, nbs - 1 < T - 1 ? nbs - 1 : T - 1, 0);
    if (nblk > 1) issue(nbs, 2 * nbs - 1 < T - 1 ? 2 * nbs - 1 : T - 1, 1);
  }
  // ---- l_k = -(N_k r_k + M_k p_{k+1}) ----
  for (int q = tid; q < T * NU; q += nthr) {
    const int k = q / NU, u = q - k * NU;
    const Real* f = pk + (size_t)k * BW;
    Real v = 0;
#pragma unroll
    for (int w = 0; w < NU; ++w) v += f[u * NU + w] * b2.rs[(size_t)k * NU + w];
#pragma unroll
    for (int c = 0; c < NX; ++c) v += f[oM + u * NX + c] * b2.px[(size_t)(k + 1) * NX + c];
    b2.ls[q] = -v;
  }
  __syncthreads();
  // ---- d_k = B_k l_k ----
  for (int q = tid; q < T * NX; q += nthr) {
    const int k = q / NX, j = q - k * NX;
    const Real* f = pk + (size_t)k * BW;
    Real v = 0;
#pragma unroll
    for (int u = 0; u < NU; ++u) v += f[oB + j * NU + u] * b2.ls[(size_t)k * NU + u];
    b2.cd[q] = v;
  }
  __syncthreads();
  if (tid < 32) {
    // ---- forward: δx_{k+1} = A_cl,k δx_k + d_k; lane j < NX owns δx_j ----
    Real x = 0;
    if (lane < NX) b2.px[lane] = (Real)0;
    for (int j = 0; j < nblk && ok; ++j) {
      const int h = j & 1, lo = j * nbs, hi = lo + nbs - 1 < T - 1 ? lo + nbs - 1 : T - 1;
      if (!wait(h)) { ok = false; break; }
      const Real* base = b2.ring + (size_t)h * nbs * BW;
      for (int k = lo; k <= hi; ++k) {
        const Real* A = base + (size_t)(k - lo) * BW + oA;
        Real xc[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) xc[c] = __shfl_sync(0xffffffffu, x, c);
        Real s0 = (lane < NX) ? b2.cd[(size_t)k * NX + lane] : (Real)0, s1 = 0;
        if (lane < NX) {
#pragma unroll
          for (int c = 0; c < NX; c += 2) {
            s0 += A[lane * NX + c] * xc[c];
            if (c + 1 < NX) s1 += A[lane * NX + c + 1] * xc[c + 1];
          }
        }
        x = s0 + s1;
        if (lane < NX) b2.px[(size_t)(k + 1) * NX + lane] = x;
      }
      __syncwarp();
      if (lane == 0 && j + 2 < nblk) {
        fence_proxy_async();
        const int lo2 = (j + 2) * nbs;
        issue(lo2, lo2 + nbs - 1 < T - 1 ? lo2 + nbs - 1 : T - 1, h);
      }
    }
    if (lane == 0) *s_flag = ok ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag == 0) return false;
  // ---- δu_k = L_k δx_k + l_k, and δx to global memory ----
  double* du = ar + L.du;
  double* dx = ar + L.dx;
  for (int q = tid; q < T * NU; q += nthr) {
    const int k = q / NU, u = q - k * NU;
    const Real* f = pk + (size_t)k * BW;
    Real v = b2.ls[q];
#pragma unroll
    for (int c = 0; c < NX; ++c) v += f[oL + u * NX + c] * b2.px[(size_t)k * NX + c];
    du[q] = (double)v;
  }
  for (int q = tid; q < (T + 1) * NX; q += nthr) dx[q] = (double)b2.px[q];
  __syncthreads();
  return true;
}

template <int NX, int NU, typename Real, int PAIRS, int W>
__device__ __forceinline__ void load_gt_regs(const double* gt, int T, const int (&mk)[PAIRS], int ck,
                                             Real (&g)[PAIRS][NU][W]) {
#pragma unroll
  for (int k = 0; k < PAIRS; ++k)
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int w = 0; w < W; ++w)
        g[k][u][w] = (mk[k] < T) ? (Real)gt[(long long)mk[k] * NU * NX + u * NX + ck + w] : (Real)0;
}

// Vector loads/stores of W consecutive shared-memory values (8- or 16-byte aligned by the layout:
// row offsets within a chunk are multiples of NX, block offsets of NU, and W divides NX).
template <int N, typename Real>
__device__ __forceinline__ void ld_vec(const Real* p, Real (&v)[N]) {
  if constexpr (N == 2 && sizeof(Real) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(p); v[0] = t.x; v[1] = t.y;
  } else if constexpr (N == 4 && sizeof(Real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (N == 2 && sizeof(Real) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p); v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}
template <int N, typename Real>
__device__ __forceinline__ void st_vec(Real* p, const Real (&v)[N]) {
  if constexpr (N == 2 && sizeof(Real) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else if constexpr (N == 4 && sizeof(Real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (N == 2 && sizeof(Real) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

// Two FP32 values in one 64-bit register pair, and the paired FP32 arithmetic of sm_100-family
// GPUs (PTX .f32x2) on them: each half is rounded as the scalar instruction would round it.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2_pack(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2p v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p f2_fma(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2p f2_add(f2p a, f2p b) {
  f2p d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p f2_sub(f2p a, f2p b) {
  f2p d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p f2_mul(f2p a, f2p b) {
  f2p d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p f2_neg(f2p a) { return a ^ 0x8000000080000000ull; }
// 8-byte shared-memory load / store of a pair (8-byte aligned by the chunk layout when W = 2)
__device__ __forceinline__ f2p f2_ld(const float* p) { return *reinterpret_cast<const f2p*>(p); }
__device__ __forceinline__ void f2_st(float* p, f2p v) { *reinterpret_cast<f2p*>(p) = v; }

// Global store of N consecutive values with an L2 cache policy (the λ stream of the row pass is
// written once per pass and marked first to evict).
template <int N, typename Real>
__device__ __forceinline__ void st_vec_stream(Real* p, const Real (&v)[N], uint64_t pol) {
  if constexpr (N == 2 && sizeof(Real) == 4) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"((float)v[0]), "f"((float)v[1]), "l"(pol)
                 : "memory");
  } else if constexpr (N == 4 && sizeof(Real) == 4) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"((float)v[0]), "f"((float)v[1]),
                 "f"((float)v[2]), "f"((float)v[3]), "l"(pol)
                 : "memory");
  } else if constexpr (sizeof(Real) == 4) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p + i), "f"((float)v[i]), "l"(pol) : "memory");
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i)
      asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p + i), "d"((double)v[i]), "l"(pol) : "memory");
  }
}

__device__ __forceinline__ void f2_st_stream(float* p, f2p v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}

// Phase timer: thread 0 accumulates the SM cycles between consecutive marks (taken right after block
// barriers) and adds them to the global counters at the end of the instance.
struct PhaseTimer {
  unsigned long long acc[NPHASE];
  long long last;
  bool on;
  __device__ void start(bool enable) {
    on = enable && threadIdx.x == 0;
    for (int k = 0; k < NPHASE; ++k) acc[k] = 0;
    last = clock64();
  }
  __device__ __forceinline__ void mark(int ph) {
    if (on) { const long long t = clock64(); acc[ph] += (unsigned long long)(t - last); last = t; }
  }
  __device__ void flush(unsigned long long* out) {
    if (on && out)
      for (int k = 0; k < NPHASE; ++k) atomicAdd(out + k, acc[k]);
  }
};

// Row pass of one FullADMM iteration over the state rows: chunks arrive by bulk copies (double
// buffered); sub-pass 1 applies the λ_ν update of the previous iteration and forms the row norms of
// η̂ = Â_j k + b̂_j + λ_ν,j, the projection gives each row's scale s_j and p̃_j, and sub-pass 2
// accumulates Z'_m = Σ_j b_{j,m} w_{j,m}ᵀ.  Pointers are hoisted into registers and the chunk
// buffer descriptors copied per chunk, so the loops touch only registers and shared memory besides
// the row data.  `first` (iteration 1: no λ update) is a template parameter so that the common path
// carries no code or registers of the other.  Returns false if a chunk copy timed out.
template <int NX, int NU, typename Real, bool first>
__device__ __forceinline__ bool fa_row_pass(const Dev<Real>& D, const LinSlot<Real>& S, const Inst& I,
                                         FASmem<NX, NU, Real>& sm, uint64_t* bars, uint32_t* phase, int* s_flag,
                                         const ColMap cm, const double* gtc, const double* gto, double* Zp,
                                         bool block1, Real lscale, Real* arp_out, Real* ard_out,
                                         unsigned long long* wait_cycles) {
  using C = FACfg<NX, NU, Real>;
  constexpr int NT = C::NT, PAIRS = C::PAIRS, NWR_MAX = C::NWR_MAX, W = C::W, RB = C::RB;
  const int T = I.T, tid = threadIdx.x, lane = tid & 31;
  const int grp = cm.grp, NG = cm.ng, NWR = cm.nwr, ck = cm.ck;
  const int gwarp = (tid - (grp < NG ? grp : 0) * NWR * 32) >> 5;
  const int mk[PAIRS] = {cm.mk[0], cm.mk[1]};
  const long long row0 = I.row0;
  const ChunkInfo* chunks = D.chunks + I.cb0;
  Real* const lam = D.lam;
  Real* const sr = D.sr;
  double* const sarr = D.s;
  const double* const parr = D.p;
  const double* const lamparr = D.lamp;
  double* const ptnarr = D.ptn;
  Real* const rowpart = sm.rowpart;
  Real* const snew_s = sm.snew;
  Real gc[PAIRS][NU][W], go[PAIRS][NU][W], z[PAIRS][NU][W];
  load_gt_regs<NX, NU, Real, PAIRS, W>(gtc, T, mk, ck, gc);
  load_gt_regs<NX, NU, Real, PAIRS, W>(gto, T, mk, ck, go);
  // FP32 with two components per thread: sub-pass 1 runs on component pairs (paired FP32 ops), the
  // gain tables packed once per pass
  constexpr bool PK = sizeof(Real) == 4 && W == 2 && !C::EM;
  [[maybe_unused]] f2p gcp[PAIRS][NU], gop[PAIRS][NU];
  if constexpr (PK) {
#pragma unroll
    for (int k = 0; k < PAIRS; ++k)
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        gcp[k][u] = f2_pack(gc[k][u][0], gc[k][u][1]);
        gop[k][u] = f2_pack(go[k][u][0], go[k][u][1]);
      }
  }
#pragma unroll
  for (int k = 0; k < PAIRS; ++k)
#pragma unroll
    for (int u = 0; u < NU; ++u)
#pragma unroll
      for (int w = 0; w < W; ++w) z[k][u][w] = (Real)0;
  Real arp = 0, ard = 0;
  const uint64_t spol = l2_policy_evict_first();
  constexpr int NUP = C::NUP;
  const int TB = (T + 1) * NX * NUP;   // offset of the previous-gains table
  if constexpr (C::EM) {
    // Gtᵀ tables ([m][u][c] in the arena) into shared memory as [m][c][u], u padded to NUP
    Real* const gts = sm.gts;
    for (int q = tid; q < (T + 1) * NX * NUP; q += NT) {
      const int u = q % NUP, mc = q / NUP, m = mc / NX, c = mc - m * NX;
      const long long a = (long long)m * NU * NX + u * NX + c;
      gts[q] = (u < NU) ? (Real)gtc[a] : (Real)0;
      gts[TB + q] = (u < NU && !first) ? (Real)gto[a] : (Real)0;
    }
  }
  // ---------------- row pass over state rows, chunk by chunk (bulk copies, double buffered) --------
  // Thread 0 waits for a chunk's copies before the block barrier that precedes its use: for chunk 0
  // here, for chunk ch+1 at the end of chunk ch, where that barrier also frees chunk ch's buffer.
  auto wait_chunk = [&](int c) {
    if (tid == 0) {
      const long long tw = clock64();
      *s_flag = mbar_wait_bounded(&bars[c & 1], phase[c & 1]) ? 1 : 0;
      if (wait_cycles) *wait_cycles += (unsigned long long)(clock64() - tw);
    }
  };
  __syncthreads();
  if (tid == 0) {
    fence_proxy_async();
    if (I.n_chunks > 0) issue_chunk<NX, NU, Real>(D, S, I, chunks[0], sm.buf[0], &bars[0]);
    if (I.n_chunks > 1) issue_chunk<NX, NU, Real>(D, S, I, chunks[1], sm.buf[1], &bars[1]);
  }
  if (I.n_chunks > 0) {
    wait_chunk(0);
    __syncthreads();
    phase[0] ^= 1u;
    if (*s_flag == 0) return false;
  }
  for (int ch = 0; ch < I.n_chunks; ++ch) {
    const int bi = ch & 1;
    // selected with constant indices: a run-time index would move the descriptors to local memory
    // and the compiler would lose that they point to shared memory
    const typename FASmem<NX, NU, Real>::Buf bf = bi ? sm.buf[1] : sm.buf[0];
    const ChunkInfo cki = chunks[ch];
    const int nr = cki.r1 - cki.r0;
    const Real* const so_s = bf.so + so_offset<NX, NU, Real>(I, cki);
    if constexpr (C::EM) {
      // sub-pass 1, entry-major: warp w takes rows w, w+NW, ...; lanes stride over the row's entries,
      // whose (m, c) gains come from the shared tables.  The warp holds the row's whole norm, so its
      // lane 0 projects the row at once.
      const int warp = tid >> 5;
      const Real* const gts = sm.gts;
      for (int q = warp; q < nr; q += NT / 32) {
        const RowMeta rm = bf.meta[q];
        const int len = (rm.t + 1) * NX;
        const Real so = so_s[q];
        const long long R = row0 + rm.pad;
        // t̂ = p + λ_p of this row, loaded now so that its latency overlaps the row
        double tpre = 0.0;
        if (block1 && lane == 0) tpre = parr[R] + lamparr[R];
        Real pn = 0;
#pragma unroll 2
        for (int p = lane; p < len; p += 32) {
          const int m = p / NX, c = p - m * NX;
          const int e = rm.off + p;
          Real bv[NU], g[NUP];
          ld_vec<NU, Real>(bf.bb + rm.boff + m * NU, bv);
          ld_vec<NUP, Real>(gts + (m * NX + c) * NUP, g);
          const Real yb = bf.bhat[e];
          Real l = bf.lam[e];
          Real y = yb;
#pragma unroll
          for (int u = 0; u < NU; ++u) y += g[u] * bv[u];
          if (!first) {
            Real go_[NUP];
            ld_vec<NUP, Real>(gts + TB + (m * NX + c) * NUP, go_);
            Real yo = yb;
#pragma unroll
            for (int u = 0; u < NU; ++u) yo += go_[u] * bv[u];
            const Real nu = so * (yo + l);
            const Real ln = l + y - nu;
            arp += (y - nu) * (y - nu);
            ard += (y - yo) * (y - yo);
            l = ln * lscale;
            const Real lg[1] = {l};
            st_vec_stream<1, Real>(lam + cki.e0 + e, lg, spol);
          }
          const Real et = y + l;
          pn += et * et;
          if (block1) {
            bf.lam[e] = et;         // η̂, kept for sub-pass 2
            bf.bhat[e] = yb + l;    // b̂ + λ, kept for sub-pass 2
          }
        }
        if (block1) {
          pn = warp_sum(pn);
          if (lane == 0) {
            // SOC projection (Supplementary Sec. II-C) with t̂ = p + λ_p, in the compute precision
            Real snew, ptn;
            soc_case_r<Real>((Real)tpre, sqrt(pn), snew, ptn);
            snew_s[q] = snew;
            sarr[R] = (double)snew;
            sr[row0 + cki.r0 + q] = snew;
            ptnarr[R] = (double)ptn;
          }
        }
      }
    } else {
      // sub-pass 1: λ update of iteration b-1, η̂ of iteration b and row norms.  Row group `grp` takes
      // rows grp, grp+NG, ...; a warp runs RB rows back to back and reduces their partial norms together
      // (one transposing butterfly), so the rows' reduction latencies overlap.
      for (int q0 = grp; q0 < nr; q0 += RB * NG) {
        Real pnv[RB];
  #pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int q = q0 + r * NG;
          pnv[r] = (Real)0;
          if (q >= nr) continue;
          const RowMeta rm = bf.meta[q];
          const Real so = so_s[q];
          Real pn = 0;
  #pragma unroll
          for (int k = 0; k < PAIRS; ++k) {
            if (mk[k] <= rm.t) {
              const int e = rm.off + mk[k] * NX + ck;
              Real bv[NU], yb[W], l[W], lg[W];
              ld_vec<NU, Real>(bf.bb + rm.boff + mk[k] * NU, bv);
              if constexpr (PK) {
                // the scalar steps below on the pair (components ck, ck+1); the norm and residual
                // sums stay scalar, in the same order
                const f2p yb2 = f2_ld(bf.bhat + e);
                f2p l2 = f2_ld(bf.lam + e);
                f2p bd[NU];
  #pragma unroll
                for (int u = 0; u < NU; ++u) bd[u] = f2_pack(bv[u], bv[u]);
                f2p y2 = yb2;
  #pragma unroll
                for (int u = 0; u < NU; ++u) y2 = f2_fma(gcp[k][u], bd[u], y2);
                if (!first) {
                  f2p yo2 = yb2;
  #pragma unroll
                  for (int u = 0; u < NU; ++u) yo2 = f2_fma(gop[k][u], bd[u], yo2);
                  const f2p nu2 = f2_mul(f2_pack(so, so), f2_add(yo2, l2));
                  const f2p ln2 = f2_sub(f2_add(l2, y2), nu2);
                  float d0, d1, e0, e1;
                  f2_unpack(f2_sub(y2, nu2), d0, d1);
                  f2_unpack(f2_sub(y2, yo2), e0, e1);
                  arp = fmaf(d0, d0, arp);
                  arp = fmaf(d1, d1, arp);
                  ard = fmaf(e0, e0, ard);
                  ard = fmaf(e1, e1, ard);
                  l2 = f2_mul(ln2, f2_pack(lscale, lscale));
                  f2_st_stream(lam + cki.e0 + e, l2, spol);
                }
                const f2p et2 = f2_add(y2, l2);
                float t0, t1;
                f2_unpack(et2, t0, t1);
                pn = fmaf(t0, t0, pn);
                pn = fmaf(t1, t1, pn);
                if (block1) {
                  f2_st(bf.lam + e, et2);               // η̂, kept for sub-pass 2
                  f2_st(bf.bhat + e, f2_add(yb2, l2));  // b̂ + λ, kept for sub-pass 2
                }
                continue;
              }
              ld_vec<W, Real>(bf.bhat + e, yb);
              ld_vec<W, Real>(bf.lam + e, l);
  #pragma unroll
              for (int w = 0; w < W; ++w) {
                Real y = yb[w];
  #pragma unroll
                for (int u = 0; u < NU; ++u) y += gc[k][u][w] * bv[u];
                if (!first) {
                  Real yo = yb[w];
  #pragma unroll
                  for (int u = 0; u < NU; ++u) yo += go[k][u][w] * bv[u];
                  const Real nu = so * (yo + l[w]);
                  const Real ln = l[w] + y - nu;
                  arp += (y - nu) * (y - nu);
                  ard += (y - yo) * (y - yo);
                  l[w] = ln * lscale;
                }
                const Real et = y + l[w];
                pn += et * et;
                lg[w] = l[w];
                yb[w] += l[w];     // b̂ + λ, kept for sub-pass 2
                l[w] = et;         // η̂, kept for sub-pass 2
              }
              if (!first) st_vec_stream<W, Real>(lam + cki.e0 + e, lg, spol);
              if (block1) {
                st_vec<W, Real>(bf.lam + e, l);
                st_vec<W, Real>(bf.bhat + e, yb);
              }
            }
          }
          pnv[r] = pn;
        }
        if (block1) {
          // lanes [r·32/RB, (r+1)·32/RB) end with the warp's sum for row q0 + r·NG
          const Real tot = warp_sum_rows<RB>(pnv, lane);
          const int r = lane / (32 / RB);
          const int q = q0 + r * NG;
          if ((lane & (32 / RB - 1)) == 0 && q < nr) rowpart[q * NWR_MAX + gwarp] = tot;
        }
      }
    }
    __syncthreads();
    if (block1) {
      if constexpr (!C::EM) {
        // SOC projection per row (Supplementary Sec. II-C) with t̂ = p + λ_p
        for (int q = tid; q < nr; q += NT) {
          Real a2 = 0;
          for (int w = 0; w < NWR; ++w) a2 += rowpart[q * NWR_MAX + w];
          const long long R = row0 + bf.meta[q].pad;
          Real snew, ptn;   // in the compute precision (FP32 cones in mixed mode)
          soc_case_r<Real>((Real)(parr[R] + lamparr[R]), sqrt(a2), snew, ptn);
          snew_s[q] = snew;
          sarr[R] = (double)snew;
          sr[row0 + cki.r0 + q] = snew;   // storage order: the next iteration's chunk copy brings it
          ptnarr[R] = (double)ptn;
        }
        __syncthreads();
      }
      // sub-pass 2: Z'_m[:, c] += b_{j,m} w_{j,m}[c], w = ν - b̂ - λ = s η̂ - (b̂ + λ), from the η̂ and
      // b̂ + λ that sub-pass 1 left in the chunk buffer (λ_ν itself was stored to global memory)
      for (int q = grp; q < nr; q += NG) {
        const RowMeta rm = bf.meta[q];
        const Real sn = snew_s[q];
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) {
          if (mk[k] < rm.t) {
            const int e = rm.off + mk[k] * NX + ck;
            Real bv[NU], bl[W], et[W];
            ld_vec<NU, Real>(bf.bb + rm.boff + mk[k] * NU, bv);
            ld_vec<W, Real>(bf.bhat + e, bl);   // b̂ + λ
            ld_vec<W, Real>(bf.lam + e, et);    // η̂ = y + λ
#pragma unroll
            for (int w = 0; w < W; ++w) {
              const Real wv = sn * et[w] - bl[w];
#pragma unroll
              for (int u = 0; u < NU; ++u) z[k][u][w] += bv[u] * wv;
            }
          }
        }
      }
    }
    if (ch + 1 < I.n_chunks) wait_chunk(ch + 1);
    __syncthreads();
    if (ch + 1 < I.n_chunks) {
      phase[bi ^ 1] ^= 1u;
      if (*s_flag == 0) return false;
    }
    if (tid == 0 && ch + 2 < I.n_chunks) {
      fence_proxy_async();
      issue_chunk<NX, NU, Real>(D, S, I, chunks[ch + 2], bf, &bars[bi]);
    }
  }
  if (block1) {
    // Z' = Σ over row groups (fixed order) of the register accumulators; the idle chunk buffers
    // hold the per-group partials when there is more than one group.
    if (NG == 1) {
#pragma unroll
      for (int k = 0; k < PAIRS; ++k)
        if (mk[k] < T)
#pragma unroll
          for (int u = 0; u < NU; ++u)
#pragma unroll
            for (int w = 0; w < W; ++w) Zp[(long long)mk[k] * NU * NX + u * NX + ck + w] = (double)z[k][u][w];
    } else {
      Real* part = sm.buf[0].lam;   // NG × T × NU × NX values (NG is capped so that they fit)
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
        Zp[q] = (double)acc;
      }
    }
  }
  __syncthreads();
  *arp_out = arp;
  *ard_out = ard;
  return true;
}

// Control rows of one FullADMM iteration (block 1 for the rows b_j = ±e_i, b̂_j = 0): the λ_ν update of
// the previous iteration (first: none), η̂, the cone in the compute precision, Z' and the residual
// sums prp, prd.  Shared by the lifted and the as-written iterations.
template <int NX, int NU, typename Real>
__device__ __forceinline__ void fa_control_rows(const Dev<Real>& D, const Inst& I, double* ar, const Arena& L,
                                                const double* gtc_arena, const double* gto_arena, bool first,
                                                bool block1, Real lscale, double& prp, double& prd) {
  constexpr int NT = FACfg<NX, NU, Real>::NT;
  const int tid = threadIdx.x;
  Real* lam = D.lam;
  // ---------------- control rows (one block each; b = ±e_i, b̂ = 0) ----------------
  // A group holds the rows of one (k, i), upper before lower bound, which update the same Z'
  // elements; a thread takes whole groups.  For the common two-row group the loads of both rows
  // are issued together, in few dependent rounds: each round trip costs a full memory latency while
  // the row streams keep the memory system loaded.  Both paths update Z' and the residual sums row
  // after row, in the same order.
  auto ctrl_row = [&](long long R, const int4 ri, long long e0, Real sold, Real tt, Real (&l)[NX], const Real (&gcv)[NX],
                      const Real (&gov)[NX], Real& snew, Real (&et)[NX], Real (&lv)[NX]) {
    const Real sg = (ri.y == ROW_UHI) ? (Real)1 : (Real)-1;
    Real an = 0, lrp = 0, lrd = 0;   // per-row sums in the compute precision, like the state rows
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      const Real y = sg * gcv[c];
      Real lc = l[c];
      if (!first) {
        const Real yo = sg * gov[c];
        const Real nu = sold * (yo + lc);
        const Real ln = lc + y - nu;
        lrp += (y - nu) * (y - nu);
        lrd += (y - yo) * (y - yo);
        lc = ln * lscale;
        lam[e0 + c] = lc;
      }
      lv[c] = lc;
      et[c] = y + lc;
      an += et[c] * et[c];
    }
    prp += (double)lrp; prd += (double)lrd;
    if (block1) {
      // the cone in the compute precision (FP32 cones in mixed mode), as for the state rows
      Real ptn;
      soc_case_r<Real>(tt, sqrt(an), snew, ptn);
      D.s[R] = (double)snew; D.ptn[R] = (double)ptn;
    }
  };
  for (int g = tid; g < I.n_groups; g += NT) {
    const int2 gr = D.groups[I.grp0 + g];
    if (gr.y == 2) {
      const long long RA = gr.x, RB = (long long)gr.x + 1;
      const int4 riA = D.rinfo[RA], riB = D.rinfo[RB];
      const long long eA = D.rent[RA], eB = D.rent[RB];
      const Real sA = (Real)D.s[RA], sB = (Real)D.s[RB];
      const Real tA = block1 ? (Real)(D.p[RA] + D.lamp[RA]) : (Real)0;
      const Real tB = block1 ? (Real)(D.p[RB] + D.lamp[RB]) : (Real)0;
      const long long gofs = (long long)riA.x * NU * NX + riA.z * NX;   // the group's (k, i)
      Real gcv[NX], gov[NX], lA[NX], lB[NX];
#pragma unroll
      for (int c = 0; c < NX; ++c) {
        gcv[c] = (Real)gtc_arena[gofs + c];
        gov[c] = first ? (Real)0 : (Real)gto_arena[gofs + c];
        lA[c] = lam[eA + c];
        lB[c] = lam[eB + c];
      }
      Real snA = 1, snB = 1, etA[NX], etB[NX], lvA[NX], lvB[NX];
      ctrl_row(RA, riA, eA, sA, tA, lA, gcv, gov, snA, etA, lvA);
      ctrl_row(RB, riB, eB, sB, tB, lB, gcv, gov, snB, etB, lvB);
      if (block1) {
        const Real sgA = (riA.y == ROW_UHI) ? (Real)1 : (Real)-1, sgB = (riB.y == ROW_UHI) ? (Real)1 : (Real)-1;
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          double z = ar[L.Zp + gofs + c];
          z += (double)(sgA * (snA * etA[c] - lvA[c]));
          z += (double)(sgB * (snB * etB[c] - lvB[c]));
          ar[L.Zp + gofs + c] = z;
        }
      }
    } else {
      for (int q = 0; q < gr.y; ++q) {
        const long long R = gr.x + q;
        const int4 ri = D.rinfo[R];
        const long long e0 = D.rent[R];
        const long long gofs = (long long)ri.x * NU * NX + ri.z * NX;
        Real gcv[NX], gov[NX], l[NX];
#pragma unroll
        for (int c = 0; c < NX; ++c) {
          gcv[c] = (Real)gtc_arena[gofs + c];
          gov[c] = first ? (Real)0 : (Real)gto_arena[gofs + c];
          l[c] = lam[e0 + c];
        }
        Real sn = 1, et[NX], lv[NX];
        ctrl_row(R, ri, e0, (Real)D.s[R], block1 ? (Real)(D.p[R] + D.lamp[R]) : (Real)0, l, gcv, gov, sn, et, lv);
        if (block1) {
          const Real sg = (ri.y == ROW_UHI) ? (Real)1 : (Real)-1;
#pragma unroll
          for (int c = 0; c < NX; ++c) ar[L.Zp + gofs + c] += (double)(sg * (sn * et[c] - lv[c]));
        }
      }
    }
  }
}

template <int NX, int NU, typename Real>
__device__ void fulladmm_instance(const Dev<Real>& D, const SolveParams& sp, int inst, FASmem<NX, NU, Real>& sm,
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
  const int tid = threadIdx.x, warp = tid >> 5;
  double rho = sp.rho;        // penalty of the current iteration (residual balancing may change it)
  double rho_done = rho;      // penalty of the last iteration whose residuals were checked
  double rp_mark = 0.0;       // r_p at the previous stall checkpoint
  const int n_rows = I.n_sr + I.n_cr;
  Real* lam = D.lam;
  double* sc = D.sc + (long long)inst * NSC;
  int* isr = D.is + inst * NIS;
  const ChunkInfo* chunks = D.chunks + I.cb0;
  PhaseTimer tm;
  tm.start(D.phase_cycles != nullptr);

  // this thread's row group and its two column groups (blocks m and T - m, components ck .. ck+W-1)
  const ColMap cm = col_map<NX, NU, Real>(I.T, FASmem<NX, NU, Real>::zcap(sp.chunk, sp.max_rows, I.T));
  // block-2 sweep areas in the chunk buffers (checked on the host to hold a ring of >= 1 step)
  B2Smem<NX, NU, Real> b2;
  b2.carve(reinterpret_cast<char*>(sm.buf[0].lam), 2 * FASmem<NX, NU, Real>::buf_bytes(sp.chunk, sp.max_rows), I.T);

  // ---- initialization (Algorithm 1): λ_p, λ_ν, k, p <- 0.  winit 1: a learned warm start of k, p̃,
  // λ_p (p = p̃).  winit 2 (inner-state carry): the previous inner solve's final state is kept — k,
  // p, p̃, λ_p, λ_ν, λ_w, λ_e and the penalty they are scaled for; δû, δx, e and ℓ too unless the
  // nominal moved to û + δû since (then the previous solution is δû = 0 in the new coordinates).
  // A previous solve that ended on a non-finite residual or a copy timeout is not carried. ----
  const bool carry = carry_applies(D.is, inst, sp.warm);
  const int winit = carry ? 2 : (sp.warm == 1 ? 1 : 0);
  // lifted warm start (with winit 1): λ_w, δû and λ_e are given as well, λ_ν follows from the
  // per-row factors θ (in D.dd) and the warm gains, δx = F_u δû and ℓ from δû
  const bool lifted = winit == 1 && isr[IS_WLIFT] != 0;
  const bool keep_dx = carry && isr[IS_MOVED] == 0;
  if (tid == 0) isr[IS_PCG] = 0;
  if (winit != 2)
    for (long long e = tid; e < I.n_ent; e += NT) lam[I.ent0 + e] = (Real)0;
  for (int r = tid; r < n_rows; r += NT) {
    const long long R = I.row0 + r;
    if (winit == 0) { D.p[R] = 0.0; D.pt[R] = 0.0; D.lamp[R] = 0.0; }
    else if (winit == 1) { D.p[R] = D.pt[R]; }
    if (winit != 2 && !lifted) D.lamw[R] = 0.0;
    if (!keep_dx) D.ell[R] = 0.0;
    D.w[R] = 0.0; D.s[R] = 1.0; D.sr[R] = (Real)1;
  }
  if (!keep_dx) {
    if (!lifted)
      for (int q = tid; q < T * NU; q += NT) ar[L.du + q] = 0.0;
    for (int q = tid; q < (T + 1) * NX; q += NT) { ar[L.dx + q] = 0.0; ar[L.e + q] = 0.0; }
  }
  if (winit != 2 && !lifted)
    for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.lam_e + q] = 0.0;
  if (winit == 0)
    for (int q = tid; q < T * NU * NX; q += NT) ar[L.K1 + q] = 0.0;
  if (winit == 2) {
    // start at the penalty the carried duals are scaled for; the factor kernels launched before
    // this solve factored block 2 and the gain divisors for it (start_rho)
    rho = sc[SC_RHOD];
    rho_done = rho;
  } else if (lifted && sc[SC_RHOW] > 0.0) {
    rho = sc[SC_RHOW];   // the lifted warm start's penalty (start_rho, as for the factors)
    rho_done = rho;
  }
  __syncthreads();
  if (lifted) {
    // δx_0 = 0, δx_{k+1} = A_k δx_k + B_k δu_k (warp 0; lane j < NX owns δx_j)
    if (warp == 0) {
      double x = 0.0;
      const int lane = tid & 31;
      for (int k = 0; k < T; ++k) {
        double xn = 0.0;
        const double* A = sa + SL.A + (long long)k * NX * NX;
        const double* B = sa + SL.B + (long long)k * NX * NU;
        for (int j = 0; j < NX; ++j) {
          const double xj = __shfl_sync(0xffffffffu, x, j);
          if (lane < NX) xn += A[lane * NX + j] * xj;
        }
        if (lane < NX) {
          for (int u = 0; u < NU; ++u) xn += B[lane * NU + u] * ar[L.du + (long long)k * NU + u];
          ar[L.dx + (long long)(k + 1) * NX + lane] = xn;
        }
        x = xn;
      }
    }
    __syncthreads();
    // ℓ_j = b_jᵀδû: a_j · δx_t for state rows, ±δu_{k,i} for control rows
    for (int r = tid; r < n_rows; r += NT) {
      const long long R = I.row0 + r;
      const int4 ri = D.rinfo[R];
      double eln = 0.0;
      if (r < I.n_sr) {
        for (int c = 0; c < NX; ++c) eln += S.arow[I.arow0 + (long long)r * NX + c] * ar[L.dx + (long long)ri.x * NX + c];
      } else {
        eln = ((ri.y == ROW_UHI) ? 1.0 : -1.0) * ar[L.du + (long long)ri.x * NU + ri.z];
      }
      D.ell[R] = eln;
    }
    if (tid == 0) isr[IS_WLIFT] = 0;
  }
  // Gtᵀ of the initial gains into Gt1 ("current"); Gt0 is the "previous" table
  for (int q = tid; q < (T + 1) * NU * NX; q += NT) {
    const int m = q / (NU * NX), u = (q / NX) % NU, c = q % NX;
    double acc = 0.0;
    if (m < T)
      for (int r = 0; r < NX; ++r) acc += ar[L.K1 + (long long)m * NU * NX + u * NX + r] * ar[L.Psi + (long long)m * NX * NX + c * NX + r];
    ar[L.Gt1 + q] = I.sqrt_tau * acc;
    ar[L.Gt0 + q] = 0.0;
  }
  if (tid == 0) { sc[SC_SCAL_RP] = 0; sc[SC_SCAL_RD] = 0; sc[SC_SCAL_RPP] = 0; sc[SC_SCAL_RDP] = 0; }
  __syncthreads();
  if (lifted) {
    // λ_ν,j = θ_j (Â_j k + b̂_j) from the warm gains' table (a warp per row, lanes over its entries)
    const int lane = tid & 31;
    for (int r = warp; r < n_rows; r += NT / 32) {
      const long long R = I.row0 + r;
      const double th = D.dd[R];
      if (!(th > 0.0)) continue;
      const int4 ri = D.rinfo[R];
      const long long e0 = D.rent[R];
      if (r < I.n_sr) {
        const long long b0 = D.rbent[R];
        for (int q = lane; q < (ri.x + 1) * NX; q += 32) {
          const int m = q / NX, c = q - m * NX;
          double y = (double)S.bhat[e0 + q];
          for (int u = 0; u < NU; ++u) y += ar[L.Gt1 + (long long)m * NU * NX + u * NX + c] * (double)S.bvec[b0 + (long long)m * NU + u];
          lam[e0 + q] = (Real)(th * y);
        }
      } else {
        const double sg = (ri.y == ROW_UHI) ? 1.0 : -1.0;
        for (int c = lane; c < NX; c += 32)
          lam[e0 + c] = (Real)(th * sg * ar[L.Gt1 + (long long)ri.x * NU * NX + ri.z * NX + c]);
      }
    }
    __syncthreads();
  }
  tm.mark(PH_INIT);
  int gsel = 1;           // arena table holding Gtᵀ of the current gains (other one: previous)
  const int Lmax = sp.max_iter;
  int status = ST_MAXITER, iters = 0;
  double r_p = 0, r_d = 0;
  const int gpk = (I.n_groups > 0) ? I.n_groups / T : 0;

  for (int b = 1; b <= Lmax + 1 && Lmax > 0; ++b) {
    const bool first = (b == 1);
    const bool block1 = (b <= Lmax);
    const double* gtc_arena = ar + (gsel ? L.Gt1 : L.Gt0);
    const double* gto_arena = ar + (gsel ? L.Gt0 : L.Gt1);
    Real arp = 0, ard = 0;
    const double rho_prev = rho;   // penalty of iteration b-1
    Real lscale = (Real)1;         // rescale of the scaled dual λ_ν^{b-1} when ρ changes for iteration b

    // ---------------- residual balancing at the start of iteration b (uses iteration b-2) ----------------
    if (block1 && sp.adapt_every > 0 && b >= 3 && b > sp.adapt_every && (b - 1) % sp.adapt_every == 0) {
      double rn = rho;
      if (r_p > sp.adapt_mu * r_d) rn = fmin(rho * sp.adapt_tau, sp.rho_max);
      else if (r_d > sp.adapt_mu * r_p) rn = fmax(rho / sp.adapt_tau, sp.rho_min);
      if (rn != rho) {
        const double f = rho / rn;
        for (int r = tid; r < n_rows; r += NT) {
          const long long R = I.row0 + r;
          D.lamp[R] *= f;
          D.lamw[R] *= f;
        }
        for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.lam_e + q] *= f;
        lscale = (Real)f;
        rho = rn;
        gain_divisors<Real>(D, inst, rho);
        __syncthreads();
        if (warp == 0) riccati_factor_warp<Real>(D, inst, rho, ric_scr);
      }
    }

    // ---------------- row pass over state rows (bulk copies, double buffered) ----------------
    unsigned long long* const wc = tm.on ? &tm.acc[PH_WAIT] : nullptr;
    const bool rows_ok =
        first ? fa_row_pass<NX, NU, Real, true>(D, S, I, sm, bars, phase, s_flag, cm, gtc_arena, gto_arena, ar + L.Zp,
                                                block1, lscale, &arp, &ard, wc)
              : fa_row_pass<NX, NU, Real, false>(D, S, I, sm, bars, phase, s_flag, cm, gtc_arena, gto_arena, ar + L.Zp,
                                                 block1, lscale, &arp, &ard, wc);
    if (!rows_ok) {
      status = ST_TIMEOUT;
      goto done;
    }
    __syncthreads();
    tm.mark(PH_ROWS);
    double prp = (double)arp, prd = (double)ard;
    fa_control_rows<NX, NU, Real>(D, I, ar, L, gtc_arena, gto_arena, first, block1, lscale, prp, prd);
    double z2 = 0.0, z3 = 0.0;
    block_sum4(prp, prd, z2, z3, sm.red);
    tm.mark(PH_CTRL);

    // ---------------- convergence test of iteration b-1 ----------------
    if (!first) {
      r_p = sqrt(sc[SC_SCAL_RP] + prp);
      r_d = rho_prev * sqrt(sc[SC_SCAL_RD] + prd);
      rho_done = rho_prev;
      iters = b - 1;
      const bool bad = !(r_p == r_p) || !(r_d == r_d) || isinf(r_p) || isinf(r_d);
      if (bad) { status = ST_NUMERIC; break; }
      if (sp.check && r_p <= sp.eps_p && r_d <= sp.eps_d) { status = ST_CONVERGED; break; }
      if (sp.check && sp.stall_every > 0 && iters % sp.stall_every == 0) {
        if (iters >= 2 * sp.stall_every && r_p > sp.eps_p) {
          if (r_p > sp.stall_ratio * rp_mark) { status = ST_STALLED; break; }
          // budget stop: at the rate r_p fell over the last period it needs `need` more iterations
          if (sp.stall_budget > 0.0) {
            const double need = (double)sp.stall_every * log(sp.eps_p / r_p) / log(r_p / rp_mark);
            if ((double)iters + sp.stall_budget * need > (double)Lmax) { status = ST_STALLED; break; }
          }
        }
        rp_mark = r_p;
      }
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
    tm.mark(PH_SCAL1);
    // Riccati linear terms: q_t = 2Q_x(x̂_t - x_g) - ρ(e_t - λ_e,t) + (ρ/2) Σ_{rows at t} d_j a_j
    for (int q = tid; q < T * NX; q += NT) {
      const int t = q / NX + 1, c = q % NX;
      double v = 2.0 * ar[L.Qx + c] * (sa[SL.x_hat + (long long)t * NX + c] - ar[L.xg + c])
                 - rho * (ar[L.e + (long long)t * NX + c] - ar[L.lam_e + (long long)t * NX + c]);
      for (int s2 = 0; s2 < I.rows_per_t; ++s2) {
        const long long rr = (long long)(t - 1) * I.rows_per_t + s2;
        v += 0.5 * rho * D.dd[I.row0 + rr] * S.arow[I.arow0 + rr * NX + c];
      }
      b2.qs[(size_t)t * NX + c] = (Real)v;
    }
    //   r_k = 2R_u(û_k - u_ref) + (ρ/2) Σ_{control rows at (k,i)} σ_j d_j e_i
    for (int q = tid; q < T * NU; q += NT) {
      const int k = q / NU, iu = q % NU;
      double v = 2.0 * ar[L.Ru + iu] * (sa[SL.u_hat + q] - ar[L.uref + iu]);
      for (int g = k * gpk; g < (k + 1) * gpk; ++g) {
        const int2 gr = D.groups[I.grp0 + g];
        for (int qq = 0; qq < gr.y; ++qq) {
          const int4 ri = D.rinfo[gr.x + qq];
          if (ri.z == iu) v += 0.5 * rho * ((ri.y == ROW_UHI) ? 1.0 : -1.0) * D.dd[gr.x + qq];
        }
      }
      b2.rs[q] = (Real)v;
    }
    for (int q = tid; q < (T + 1) * NX; q += NT) ar[L.dx_prev + q] = ar[L.dx + q];
    __syncthreads();
    tm.mark(PH_QR);
    // ---------------- (c) gain update: K^b from Z'; Gtᵀ^b replaces the previous table ----------------
    // ---------------- (c) gain update and (b) Block 2, which are independent: the Riccati sweep runs
    // on warp 0 while the other warps solve for K^b (its Gtᵀ^b replaces the previous table) ----------------
    {
      const double gargs[2] = {I.sqrt_tau, rho * I.sqrt_tau};
      double* gt_new = ar + (gsel ? L.Gt0 : L.Gt1);
      const PcgArgs pcg{sp.kv_pcg_iters, sp.kv_pcg_tol, rho, I.tau, sa + SL.Gm, sm.red};
      if (!block2_sweep_and_gain<NX, NU, Real>(ar, L, T, b2, bars, phase, s_flag, sm.rowpart, gargs, ar + L.K1, gt_new,
                                               pcg, isr + IS_PCG)) {
        status = ST_TIMEOUT;
        goto done;
      }
      gsel ^= 1;
    }
    tm.mark(PH_RICCATI);
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
    tm.mark(PH_DUALS);
  }
done:
  // On a copy timeout the other buffer may still have a copy in flight: wait for it (bounded).
  if (status == ST_TIMEOUT && tid == 0) {
    for (int k = 0; k < 2; ++k) (void)mbar_wait_bounded(&bars[k], phase[k]);
  }
  if (tid == 0) {
    sc[SC_RP] = r_p; sc[SC_RD] = r_d;
    sc[SC_RPP] = sqrt(sc[SC_SCAL_RPP]); sc[SC_RDP] = rho_done * sqrt(sc[SC_SCAL_RDP]);
    sc[SC_RHO] = rho_done;
    sc[SC_RHOD] = rho;
    isr[IS_STATUS] = status; isr[IS_ITERS] = iters; isr[IS_CUMITERS] += iters;
    isr[IS_MOVED] = 0;
  }
  tm.flush(D.phase_cycles);
  __syncthreads();
}

template <int NX, int NU, typename Real>
__global__ void __launch_bounds__(FACfg<NX, NU, Real>::NT, FACfg<NX, NU, Real>::MINB) k_fulladmm(Dev<Real> D, SolveParams sp) {
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
    int* isr = D.is + inst * NIS;
    if (threadIdx.x == 0) isr[IS_FALLBACK] = 0;
    fulladmm_instance<NX, NU, Real>(D, sp, inst, sm, bars, ph, &s_flag, ric_scr);
    // learned warm start that stalled: rerun from the cold initialization with the full budget
    if (sp.warm && sp.fallback && isr[IS_STATUS] == ST_STALLED) {
      const int it1 = isr[IS_ITERS];
      SolveParams sp2 = sp;
      sp2.warm = 0;
      __syncthreads();
      if (threadIdx.x == 0) isr[IS_FALLBACK] = 1;
      {
        // residual balancing or a carried penalty may have refactored block 2 and the gain
        // divisors for another ρ
        if (sp.adapt_every > 0 || sp.warm != 0) {
          gain_divisors<Real>(D, inst, sp.rho);
          __syncthreads();
          if ((threadIdx.x >> 5) == 0) riccati_factor_warp<Real>(D, inst, sp.rho, ric_scr);
          __syncthreads();
        }
        fulladmm_instance<NX, NU, Real>(D, sp2, inst, sm, bars, ph, &s_flag, ric_scr);
        if (threadIdx.x == 0) isr[IS_ITERS] += it1;
      }
      __syncthreads();
    }
    if (isr[IS_STATUS] == ST_TIMEOUT) break;
  }
}

}  // namespace nrto
