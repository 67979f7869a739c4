// Device-side data layout and helpers of libnrto (NRTO inner loop on sm_103a).
//
// Storage model (one problem = a batch of independent instances):
//  * per-instance "arena" of doubles (parameters, per-step matrices, gains, solver vectors);
//  * two linearization "slots" (current nominal and candidate nominal of the outer loop), each
//    holding per-instance slot arenas (û, x̂, A_k, B_k, G_m) and the ragged row arrays;
//  * ragged row arrays in the compute precision `Real`: for a state constraint at time t the row
//    holds ζ-blocks 0..t ((t+1)·nx entries; a state constraint at t only sees the disturbances up
//    to t); a control bound holds one block (nx entries).
//      lam  : λ_ν (FullADMM) or η̃ (DR)          entries
//      bhat : b̂_j                                 entries (state rows)
//      bvec : b_{j,m}, nu values per block          (t+1)·nu per state row (block t is zero)
//  * per-row scalars in double (p, p̃, λ_p, lifted slack w, λ_w, projection scale s, ...).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#ifndef NRTO_HD
#define NRTO_HD __host__ __device__ __forceinline__
#endif

namespace nrto {

enum : int { KIND_UNICYCLE = 0, KIND_QUADCOPTER = 1, KIND_ARM = 2 };
// row codes (int4.y of the row table)
enum : int { ROW_SPHERE = 0, ROW_XHI = 1, ROW_XLO = 2, ROW_UHI = 3, ROW_ULO = 4 };
// instance status
enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXITER = 2, ST_NUMERIC = 3, ST_TIMEOUT = 4, ST_STALLED = 5 };

constexpr int MAX_DYN = 40;
// Arm parameters (dyn_params): DH rows (a, d, α) × 7, damping (7), inertia (7), clamping flag; the host
// completes a 21-value table (the double integrator) with zero damping, unit inertia and no clamping.
enum : int { ARM_DH = 0, ARM_DAMP = 21, ARM_INERT = 28, ARM_CLIP = 35, ARM_NPRM = 36 };

// Per-instance metadata (host builds it at create time).
struct Inst {
  int kind, nx, nu, T;
  int n_sr, n_cr, rows_per_t, n_groups;   // state rows, control rows, state rows per step, (k,i) groups
  int n_obs, obs_dim, n_link, n_dyn;
  int cb0, n_chunks;                      // chunk boundary table offset, number of chunks
  int pad0;
  long long row0;                         // first global row (state rows, then control rows)
  long long ent0;                         // first entry of the instance's rows
  long long n_ent;                        // entries of the instance (state + control rows)
  long long n_ent_state;                  // entries of the state rows
  long long bent0;                        // first bvec value
  long long grp0;                         // first control group
  long long arena0;                       // offset into the double arena
  long long slot0;                        // offset into each slot arena
  long long arow0;                        // offset into the a_j table (nx per state row)
  double dt, tau, sqrt_tau;
};

// One solver chunk: a run of whole state rows staged together in shared memory.  Entry and b
// ranges start 16-byte aligned (the host pads the row layout at every chunk start).
struct ChunkInfo {
  long long e0, b0;     // first entry / first b value of the chunk (global indices)
  int r0, r1;           // local state-row range [r0, r1) of the instance
  int ne, nb;           // entries / b values to copy, rounded up to 4 (16-byte multiples)
  int pad0, pad1;
};

// Per state row, offsets relative to its chunk (copied to shared memory with the chunk).
struct RowMeta {
  int off, boff, t, pad;
};

// Offsets (in doubles) inside one instance's arena.
struct Arena {
  long long x0, xg, uref, Qx, Ru, RK, ulo, uhi, xlo, xhi, dyn, obs, link, Sigma;
  long long Psi, SigU, SigL, Phi;
  long long K0, K1, Kt, Kacc, Gt0, Gt1, Zp;
  long long du, dx, du_prev, dx_prev, e, lam_e, qv, rv;
  long long Pf, Gam, Dv, RicL, RicAcl, RicN, RicM, Ws1, Ws2, Pc1, RicPk;
  long long total;
};

// Per-step record of the block-2 factors in the compute precision (N, M, L, A_cl, B), padded to a
// multiple of 4 values so that every record starts on a 16-byte boundary.
NRTO_HD constexpr int pk_stride(int nx, int nu) { return ((nu * nu + 3 * nu * nx + nx * nx) + 3) & ~3; }

NRTO_HD Arena arena_layout(int nx, int nu, int T, int n_obs, int n_link) {
  Arena a;
  long long o = 0;
  auto take = [&](long long n) { long long r = o; o += (n + 1) & ~1LL; return r; };
  a.x0 = take(nx); a.xg = take(nx); a.uref = take(nu); a.Qx = take(nx); a.Ru = take(nu); a.RK = take(nu);
  a.ulo = take(nu); a.uhi = take(nu); a.xlo = take(nx); a.xhi = take(nx); a.dyn = take(MAX_DYN);
  a.obs = take(4LL * (n_obs > 0 ? n_obs : 1)); a.link = take(5LL * (n_link > 0 ? n_link : 1));
  long long s1 = (long long)(T + 1);
  a.Sigma = take(s1 * nx * nx); a.Psi = take(s1 * nx * nx); a.SigU = take(s1 * nx * nx);
  a.SigL = take(s1 * nx); a.Phi = take(s1 * nx * nx);
  long long g = (long long)T * nu * nx;
  a.K0 = take(g); a.K1 = take(g); a.Kt = take(g); a.Kacc = take(g);
  a.Gt0 = take(s1 * nu * nx); a.Gt1 = take(s1 * nu * nx); a.Zp = take(g);
  a.du = take((long long)T * nu); a.dx = take(s1 * nx); a.du_prev = take((long long)T * nu);
  a.dx_prev = take(s1 * nx); a.e = take(s1 * nx); a.lam_e = take(s1 * nx); a.qv = take(s1 * nx);
  a.rv = take((long long)T * nu);
  a.Pf = take((long long)T * nu * nu); a.Gam = take((long long)T * nu); a.Dv = take(g);
  a.RicL = take(g); a.RicAcl = take((long long)T * nx * nx); a.RicN = take((long long)T * nu * nu);
  a.RicM = take(g); a.Ws1 = take(g); a.Ws2 = take(g); a.Pc1 = take(g);
  a.RicPk = take((long long)T * pk_stride(nx, nu));   // sized for double records
  a.total = o;
  return a;
}

// Offsets (in doubles) inside one instance's slot arena (one per linearization slot).
struct SlotL {
  long long u_hat, x_hat, A, B, Gm, total;
};

NRTO_HD SlotL slot_layout(int nx, int nu, int T) {
  SlotL s;
  long long o = 0;
  auto take = [&](long long n) { long long r = o; o += (n + 1) & ~1LL; return r; };
  s.u_hat = take((long long)T * nu);
  s.x_hat = take((long long)(T + 1) * nx);
  s.A = take((long long)T * nx * nx);
  s.B = take((long long)T * nx * nu);
  s.Gm = take((long long)T * nu * nu);
  s.total = o;
  return s;
}

// Per-instance scalar record (double) and integer record.
// SC_RHOD: the penalty the stored scaled duals are scaled for (the start penalty of a carried inner
// solve); SC_VIOL / SC_VIOLC: max_j g_j(x̄) + ‖Â_j k + b̂_j‖ of the accepted / candidate iterate.
enum : int { SC_RTRUST = 0, SC_RP, SC_RD, SC_RPP, SC_RDP, SC_SCAL_RP, SC_SCAL_RD, SC_SCAL_RPP, SC_SCAL_RDP,
             SC_PHI, SC_PHI_CAND, SC_COST, SC_RHO, SC_RDR, SC_RHOD, SC_VIOL, SC_VIOLC, SC_COST_ACC,
             SC_RHOW,   // penalty of a pending lifted warm start (0: the solver's)
             NSC = 20 };
// IS_ACCST: status of the inner solve whose candidate became the accepted iterate (0: none yet);
// IS_MOVED: the nominal moved to û + δû since the last inner solve (an accepted outer step).
// IS_PCG: PCG iterations of the k_v updates of the last inner solve (kv_pcg_iters > 0).
// IS_WLIFT: a lifted warm start (θ, λ_w, δû, λ_e, ρ) is pending for the next FullADMM inner solve.
enum : int { IS_STATUS = 0, IS_ITERS, IS_SLOT, IS_ACCEPT, IS_DRITERS, IS_CUMITERS, IS_NACC, IS_FALLBACK, IS_ACCST,
             IS_MOVED, IS_PCG, IS_WLIFT, NIS = 12 };

template <typename Real>
struct LinSlot {
  double* arena;     // slot arenas (per instance at Inst::slot0)
  double* g0;        // per row g_j(x̂) (control rows: ±û - bound)
  double* arow;      // ∇g_j (nx per state row)
  Real* bhat;        // per entry
  Real* bvec;        // per state-row block, nu values
};

template <typename Real>
struct Dev {
  int n_inst;
  const Inst* inst;
  double* arena;
  const int4* rinfo;            // per row: {t or k, code, a, b}
  const long long* rent;        // per row: first entry
  const long long* rbent;       // per state row: first bvec value (global row index)
  const ChunkInfo* chunks;      // n_chunks per instance at Inst::cb0
  const RowMeta* rmeta;         // per row (state rows only)
  const int2* groups;           // control groups: {first global row, count}, per instance at grp0
  LinSlot<Real> slot[2];
  Real* lam;                    // λ_ν or η̃ rows
  Real* sr;                     // per row: projection scale s_j in the compute precision (FullADMM row pass;
                                // state rows in their chunk storage order), 4 elements of tail padding
  double *p, *pt, *ptn, *lamp, *w, *lamw, *s, *ell, *dd, *rnorm;   // per row
  double* sc;                   // NSC per instance
  int* is;                      // NIS per instance
  int* queue;                   // work counters
  const int* order;             // instance order per launch
  unsigned long long* phase_cycles;   // NPHASE counters, or null when phase timing is off
};

// Inner-state carry: the next FullADMM inner solve of instance i starts from the previous one's final
// state when it is requested (warm mode 2) and the previous solve ended with a usable state.  The
// factor kernels launched before the solve and the solve itself take the same decision.
__device__ __forceinline__ bool carry_applies(const int* is, int i, int warm) {
  const int st = is[i * NIS + IS_STATUS];
  return warm == 2 && (st == ST_CONVERGED || st == ST_MAXITER || st == ST_STALLED);
}
// A pending lifted warm start with its own penalty (warm mode 1).
__device__ __forceinline__ bool lifted_warm_rho(const int* is, const double* sc, int i, int warm) {
  return warm == 1 && is[i * NIS + IS_WLIFT] != 0 && sc[(long long)i * NSC + SC_RHOW] > 0.0;
}
// Penalty the inner solve of instance i starts with: the carried one, a lifted warm start's, else rho0.
__device__ __forceinline__ double start_rho(const int* is, const double* sc, int i, int warm, double rho0) {
  if (carry_applies(is, i, warm)) return sc[(long long)i * NSC + SC_RHOD];
  if (lifted_warm_rho(is, sc, i, warm)) return sc[(long long)i * NSC + SC_RHOW];
  return rho0;
}

// Phases of one inner iteration timed by the persistent solvers (thread 0 of each CTA, SM cycles).
enum : int { PH_INIT = 0, PH_ROWS, PH_CTRL, PH_SCAL1, PH_QR, PH_GAIN, PH_RICCATI, PH_DUALS, PH_WAIT, NPHASE };

// ------------------------------------------------------------------------------------------
// warp helpers
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of up to 4 doubles; `red` is shared scratch of >= 4*(blockDim/32) doubles.
// All threads get the result.  Deterministic (fixed tree).
__device__ inline void block_sum4(double& a, double& b, double& c, double& d, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a); b = warp_sum(b); c = warp_sum(c); d = warp_sum(d);
  __syncthreads();
  if (lane == 0) { red[4 * wid] = a; red[4 * wid + 1] = b; red[4 * wid + 2] = c; red[4 * wid + 3] = d; }
  __syncthreads();
  a = b = c = d = 0.0;
  for (int i = 0; i < nw; ++i) { a += red[4 * i]; b += red[4 * i + 1]; c += red[4 * i + 2]; d += red[4 * i + 3]; }
  __syncthreads();
}

// Block-wide maximum of one double (same scratch as block_sum4); all threads get the result.
__device__ inline double block_max(double a, double* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  __syncthreads();
  if (lane == 0) red[wid] = a;
  __syncthreads();
  a = red[0];
  for (int i = 1; i < nw; ++i) a = fmax(a, red[i]);
  __syncthreads();
  return a;
}

// ------------------------------------------------------------------------------------------
// small dense linear algebra (row-major, sequential; used by single threads on tiny matrices)
// ------------------------------------------------------------------------------------------
// In-place Cholesky A = L Lᵀ (lower); returns false if not positive definite.
NRTO_HD bool chol_inplace(double* A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = v / d;
    }
    for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
  }
  return true;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n×n matrix (n <= 16).
// On return A is overwritten, lam holds eigenvalues, V (row-major) holds eigenvectors in columns.
NRTO_HD void jacobi_eig(double* A, int n, double* lam, double* V) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = A[i * n + j] * A[i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (apq == 0.0) continue;
        double app = A[p * n + p], aqq = A[q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // A ← Jᵀ A J  (rotate columns p,q then rows p,q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

}  // namespace nrto
