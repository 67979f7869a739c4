// Host side of libnrto: the C ABI declared in include/nrto.h.
//
// A problem owns every device buffer of its batch.  create() validates the descriptors, builds the
// row tables (constraint rows, ragged offsets, chunk boundaries for the persistent solver), uploads the
// parameters and runs the setup kernel; the outer loop and the inner solvers are kernel launches on
// the problem's stream.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <exception>
#include <mutex>
#include <thread>
#include <numeric>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nrto.h"
#include "fulladmm.cuh"
#include "montecarlo.cuh"
#include "solver_kernels.h"

using namespace nrto;

namespace {

thread_local std::string g_last_error;

struct NrtoError : std::runtime_error {
  nrto_status st;
  NrtoError(nrto_status s, const std::string& m) : std::runtime_error(m), st(s) {}
};

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      throw NrtoError(NRTO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

void fail(nrto_status s, const std::string& m) { throw NrtoError(s, m); }

// NVTX range over one call of the C ABI (a profiler's timeline shows the host side of each call;
// without a profiler attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int kind_nx(int k) { return k == KIND_UNICYCLE ? 3 : (k == KIND_QUADCOPTER ? 12 : 14); }
int kind_nu(int k) { return k == KIND_UNICYCLE ? 2 : (k == KIND_QUADCOPTER ? 4 : 7); }
int kind_tmax(int k) { return k == KIND_UNICYCLE ? 256 : (k == KIND_QUADCOPTER ? 160 : 128); }

// Dynamic shared memory per solver CTA: the SM's 228 KB (227 KB opt-in per block) are shared by the
// kind's resident CTAs, each of which also holds ~9.5 KB of static shared memory (mbarriers, flags,
// Riccati scratch) and 1 KB reserved.
template <typename Real>
int smem_budget(int kind) {
  int minb = 1;
  if (kind == KIND_UNICYCLE) minb = FACfg<3, 2, Real>::MINB;
  else if (kind == KIND_QUADCOPTER) minb = FACfg<12, 4, Real>::MINB;
  else minb = FACfg<14, 7, Real>::MINB;
  return minb > 1 ? (228 * 1024) / minb - 12 * 1024 : 227 * 1024 - 12 * 1024;
}

template <typename Real>
size_t smem_for(int kind, int chunk, int max_rows) {
  if (kind == KIND_UNICYCLE) return FASmem<3, 2, Real>::bytes(chunk, max_rows);
  if (kind == KIND_QUADCOPTER) return FASmem<12, 4, Real>::bytes(chunk, max_rows);
  return FASmem<14, 7, Real>::bytes(chunk, max_rows);
}

struct KindLaunch {
  int kind = 0, count = 0, order0 = 0, tmax = 0, chunk = 0, max_rows = 0;
  size_t smem = 0;
  long long entries = 0;   // row entries of the kind's instances (the launches start with the largest)
};

// ---- small kernels of the outer loop ----
__global__ void k_scatter(double* arena, const Inst* inst, const double* stage, const long long* stage_off,
                          const long long* stage_len, int n) {
  const int i = blockIdx.x;
  if (i >= n) return;
  double* dst = arena + inst[i].arena0;
  const double* src = stage + stage_off[i];
  for (long long q = threadIdx.x; q < stage_len[i]; q += blockDim.x) dst[q] = src[q];
}

__global__ void k_scatter_uhat(double* slot_arena, const Inst* inst, const double* src, const long long* off, int n) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const Inst I = inst[i];
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  double* dst = slot_arena + I.slot0 + SL.u_hat;
  for (int q = threadIdx.x; q < I.T * I.nu; q += blockDim.x) dst[q] = src[off[i] + q];
}

// Output gather: per instance (block), `cnt` values of a field at offset `off` inside its arena
// (which = 0) or inside its current solver slot (which = 1) into out + out_off[i], so that the host
// reads the batch's field with one copy.
enum : int { GF_DU = 0, GF_K1 = 1, GF_UHAT = 2, GF_KACC = 3 };
__global__ void k_gather_field(const Inst* inst, const int* is, const double* arena, const double* slot0,
                               const double* slot1, int field, const long long* out_off, double* out, int n) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const Inst I = inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const double* src = nullptr;
  long long cnt = 0;
  if (field == GF_UHAT) {
    const double* sa = is[i * NIS + IS_SLOT] == 0 ? slot0 : slot1;
    src = sa + I.slot0 + slot_layout(I.nx, I.nu, I.T).u_hat;
    cnt = (long long)I.T * I.nu;
  } else if (field == GF_DU) {
    src = arena + I.arena0 + L.du;
    cnt = (long long)I.T * I.nu;
  } else {
    src = arena + I.arena0 + (field == GF_K1 ? L.K1 : L.Kacc);
    cnt = (long long)I.T * I.nu * I.nx;
  }
  for (long long q = threadIdx.x; q < cnt; q += blockDim.x) out[out_off[i] + q] = src[q];
}

// Self-test of the bounded wait that guards every bulk copy of the solver kernels: one thread waits
// on an mbarrier that nothing arrives on.  The wait gives up after its cycle limit and the kernel
// records status 4 (the per-instance status of a copy that did not arrive) and the cycles waited.
__global__ void k_selftest_wait(long long* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    const long long t0 = clock64();
    const bool arrived = mbar_wait_bounded(&bar, 0);
    out[0] = arrived ? 1 : 4;
    out[1] = clock64() - t0;
  }
}

template <typename Real>
__global__ void k_candidate(Dev<Real> D) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const int cur = D.is[i * NIS + IS_SLOT];
  const double* src = D.slot[cur].arena + I.slot0 + SL.u_hat;
  double* dst = D.slot[1 - cur].arena + I.slot0 + SL.u_hat;
  const double* du = D.arena + I.arena0 + L.du;
  for (int q = threadIdx.x; q < I.T * I.nu; q += blockDim.x) dst[q] = src[q] + du[q];
}

template <typename Real>
__global__ void k_accept(Dev<Real> D, double r0, double r_min) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  double* sc = D.sc + (long long)i * NSC;
  __shared__ int acc;
  if (threadIdx.x == 0) {
    acc = sc[SC_PHI_CAND] < sc[SC_PHI] ? 1 : 0;
    D.is[i * NIS + IS_ACCEPT] = acc;
    D.is[i * NIS + IS_NACC] += acc;
    D.is[i * NIS + IS_MOVED] = acc;
    if (acc) {
      D.is[i * NIS + IS_SLOT] = 1 - D.is[i * NIS + IS_SLOT];
      D.is[i * NIS + IS_ACCST] = D.is[i * NIS + IS_STATUS];
      sc[SC_PHI] = sc[SC_PHI_CAND];
      sc[SC_VIOL] = sc[SC_VIOLC];
      sc[SC_COST_ACC] = sc[SC_COST];
      sc[SC_RTRUST] = fmin(1.5 * sc[SC_RTRUST], r0);
    } else {
      sc[SC_RTRUST] = fmax(0.8 * sc[SC_RTRUST], r_min);
    }
  }
  __syncthreads();
  if (acc)
    for (int q = threadIdx.x; q < I.T * I.nu * I.nx; q += blockDim.x) ar[L.Kacc + q] = ar[L.K1 + q];
}

template <typename Real>
__global__ void k_reset_outer(Dev<Real> D, double r0) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  if (threadIdx.x == 0) {
    D.is[i * NIS + IS_SLOT] = 0;
    D.is[i * NIS + IS_CUMITERS] = 0;
    D.is[i * NIS + IS_NACC] = 0;
    D.is[i * NIS + IS_ACCST] = 0;
    D.is[i * NIS + IS_MOVED] = 0;
    D.sc[(long long)i * NSC + SC_RTRUST] = r0;
  }
  for (int q = threadIdx.x; q < I.T * I.nu * I.nx; q += blockDim.x) ar[L.Kacc + q] = 0.0;
}

}  // namespace

struct nrto_problem;
template <typename Real>
void launch_dr(nrto_problem* P, const nrto_solver_opts& o, SolveParams sp);

// =============================================================================================
struct nrto_problem {
  int n = 0, prec = 0;
  cudaStream_t stream = nullptr;
  std::vector<Inst> h_inst;
  std::vector<int4> h_rinfo;
  std::vector<int> h_order;
  KindLaunch kl[3];
  long long n_rows = 0, n_ent = 0, n_bent = 0, arena_total = 0, slot_total = 0, arow_total = 0;
  long long n_groups_total = 0, n_cb_total = 0;
  std::vector<long long> stage_off, stage_len, uoff, koff;
  long long stage_total = 0, u_total = 0, k_total = 0;
  std::vector<void*> allocs;
  // When carve_base is set (nrto_solve_noalloc), device buffers are cut from that caller-owned area
  // instead of being allocated.
  char* carve_base = nullptr;
  size_t carve_cap = 0, carve_used = 0;
  // device
  Inst* d_inst = nullptr;
  double* d_arena = nullptr;
  int4* d_rinfo = nullptr;
  long long* d_rent = nullptr;
  long long* d_rbent = nullptr;
  ChunkInfo* d_chunks = nullptr;
  RowMeta* d_rmeta = nullptr;
  std::vector<long long> h_rent, h_rbent;
  int2* d_groups = nullptr;
  double* d_slot_arena[2] = {nullptr, nullptr};
  double* d_g0[2] = {nullptr, nullptr};
  double* d_arow[2] = {nullptr, nullptr};
  void* d_bhat[2] = {nullptr, nullptr};
  void* d_bvec[2] = {nullptr, nullptr};
  void* d_lam = nullptr;
  void* d_sr = nullptr;
  double *d_p = nullptr, *d_pt = nullptr, *d_ptn = nullptr, *d_lamp = nullptr, *d_w = nullptr, *d_lamw = nullptr,
         *d_s = nullptr, *d_ell = nullptr, *d_dd = nullptr, *d_rnorm = nullptr;
  double* d_sc = nullptr;
  int* d_is = nullptr;
  int* d_queue = nullptr;
  int* d_order = nullptr;
  int* d_wsmap = nullptr;          // row map of nrto_set_warm_start_from_network
  unsigned long long* d_phase = nullptr;
  double* d_stage = nullptr;
  long long* d_stage_off = nullptr;
  long long* d_stage_len = nullptr;
  long long* d_uoff = nullptr;
  long long* d_koff = nullptr;     // per-instance offsets of T·n_u·n_x fields in a gathered output
  double* d_gather = nullptr;      // output gather buffer (max(u_total, k_total) values)
  // Pinned host staging of the per-instance parameters and initial controls, kept across updates
  // (zero-filled once; every update rewrites the same positions).  Not used by nrto_solve_noalloc,
  // which allocates nothing and stages through temporary host vectors.
  double* h_stage = nullptr;
  double* h_ustage = nullptr;
  double* d_ustage = nullptr;
  // Second stream for running the persistent solver launches of different dynamics kinds at the
  // same time (the tail of one kind's launch overlaps the next kind's instances), with fork / join
  // events.  Not created for nrto_solve_noalloc, whose launches run one after another.
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // CUDA graph of nrto_solve's launch sequence: captured on a call, replayed by later calls with the
  // same options, outer-step count and warm-start state.  Off while profiling (per-launch events)
  // and for nrto_solve_noalloc (graph instantiation may allocate device memory).
  bool graph_enabled = true;
  int mapping = 1;   // launch mapping of the persistent solver launches (launch_solver_kinds)
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  long long graph_launches = 0, graph_captures = 0, graph_replays = 0;
  bool graph_carry_after = false;
  bool linearized = false;
  bool warm_pending = false;
  bool wlift_pending = false;    // nrto_set_warm_start_lifted since the warm start was set
  // A FullADMM inner solve ran since the last reset, so its final state can start the next one
  // (nrto_solver_opts.carry).
  bool carry_ok = false;
  long long launches = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;   // around each solver-kernel launch
  long long prof_launches = 0;

  template <typename T>
  T* dalloc(size_t count) {
    void* ptr = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (carve_base) {
      const size_t at = (carve_used + 255) & ~size_t(255);
      if (at + bytes > carve_cap)
        fail(NRTO_ERR_INVALID, "batch needs more than the " + std::to_string(carve_cap >> 20) +
                                   " MiB static device area of nrto_solve_noalloc; use nrto_problem_create");
      ptr = carve_base + at;
      carve_used = at + bytes;
    } else {
      CK(cudaMalloc(&ptr, bytes));
      allocs.push_back(ptr);
    }
    CK(cudaMemsetAsync(ptr, 0, bytes, stream));
    return static_cast<T*>(ptr);
  }
  ~nrto_problem() {
    for (auto& ev : prof_events) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (stream2) cudaStreamDestroy(stream2);
    for (void* a : allocs) cudaFree(a);
    if (h_stage) cudaFreeHost(h_stage);
    if (h_ustage) cudaFreeHost(h_ustage);
  }
  template <typename Real>
  Dev<Real> dev() const {
    Dev<Real> D;
    D.n_inst = n;
    D.inst = d_inst;
    D.arena = d_arena;
    D.rinfo = d_rinfo;
    D.rent = d_rent;
    D.rbent = d_rbent;
    D.chunks = d_chunks;
    D.rmeta = d_rmeta;
    D.groups = d_groups;
    for (int s = 0; s < 2; ++s) {
      D.slot[s].arena = d_slot_arena[s];
      D.slot[s].g0 = d_g0[s];
      D.slot[s].arow = d_arow[s];
      D.slot[s].bhat = static_cast<Real*>(d_bhat[s]);
      D.slot[s].bvec = static_cast<Real*>(d_bvec[s]);
    }
    D.lam = static_cast<Real*>(d_lam);
    D.sr = static_cast<Real*>(d_sr);
    D.p = d_p; D.pt = d_pt; D.ptn = d_ptn; D.lamp = d_lamp; D.w = d_w; D.lamw = d_lamw; D.s = d_s;
    D.ell = d_ell; D.dd = d_dd; D.rnorm = d_rnorm;
    D.sc = d_sc; D.is = d_is; D.queue = d_queue; D.order = d_order;
    D.phase_cycles = profiling ? d_phase : nullptr;
    return D;
  }
  void check_launch(const char* what) {
    ++launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(NRTO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
};

namespace {

bool finite_arr(const double* a, long long n) {
  if (n > 0 && a == nullptr) return false;
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

void validate(const nrto_problem_desc& d, int idx) {
  auto bad = [&](const std::string& m) { fail(NRTO_ERR_INVALID, "instance " + std::to_string(idx) + ": " + m); };
  auto num = [&](const std::string& m) { fail(NRTO_ERR_NUMERIC, "instance " + std::to_string(idx) + ": " + m); };
  if (d.dyn < 0 || d.dyn > 2) bad("unknown dyn kind");
  if (d.nx != kind_nx(d.dyn) || d.nu != kind_nu(d.dyn)) bad("nx/nu do not match the dynamics model");
  if (d.T < 1 || d.T > kind_tmax(d.dyn)) bad("T out of range");
  if (!(d.dt > 0) || !std::isfinite(d.dt)) bad("dt must be positive");
  if (!(d.tau >= 0) || !std::isfinite(d.tau)) bad("tau must be >= 0");
  const int need_dyn = d.dyn == KIND_QUADCOPTER ? 5 : (d.dyn == KIND_ARM ? 21 : 0);
  if (d.n_dyn_params < need_dyn || d.n_dyn_params > MAX_DYN) bad("wrong number of dyn_params");
  if (!finite_arr(d.dyn_params, d.n_dyn_params)) bad("dyn_params not finite");
  if (d.dyn == KIND_ARM) {
    // 21 values: DH table only (double integrator); 36: DH, damping, inertia, clamping flag
    if (d.n_dyn_params != 21 && d.n_dyn_params != ARM_NPRM) bad("arm dyn_params must hold 21 or 36 values");
    if (d.n_dyn_params == ARM_NPRM) {
      for (int i = 0; i < 7; ++i) {
        if (!(d.dyn_params[ARM_DAMP + i] >= 0)) bad("arm damping must be >= 0");
        if (!(d.dyn_params[ARM_INERT + i] > 0)) bad("arm inertia must be > 0");
      }
      const double cl = d.dyn_params[ARM_CLIP];
      if (cl != 0.0 && cl != 1.0) bad("arm clamping flag must be 0 or 1");
      if (cl == 1.0 && (!finite_arr(d.x_lo, 14) || !finite_arr(d.x_hi, 14)))
        bad("arm clamping needs finite state bounds (the joint position and velocity limits)");
    }
  }
  if (!finite_arr(d.x0, d.nx) || !finite_arr(d.x_goal, d.nx) || !finite_arr(d.u_ref, d.nu)) bad("x0/x_goal/u_ref");
  if (!finite_arr(d.u_init, (long long)d.T * d.nu)) num("u_init not finite");
  if (!finite_arr(d.Sigma, (long long)(d.T + 1) * d.nx * d.nx)) num("Sigma not finite");
  if (!finite_arr(d.Qx, d.nx) || !finite_arr(d.Ru, d.nu) || !finite_arr(d.RK, d.nu)) bad("weights");
  for (int i = 0; i < d.nu; ++i)
    if (!(d.Ru[i] > 0) || !(d.RK[i] > 0)) bad("Ru and RK must be positive");
  for (int i = 0; i < d.nx; ++i)
    if (d.Qx[i] < 0) bad("Qx must be >= 0");
  if (d.n_obs < 0) bad("n_obs < 0");
  if (d.n_obs > 0) {
    if (d.dyn == KIND_UNICYCLE ? d.obs_dim != 2 : d.obs_dim != 3) bad("obs_dim");
    if (!finite_arr(d.obs_center, (long long)d.n_obs * d.obs_dim) || !finite_arr(d.obs_radius, d.n_obs)) bad("obstacles");
  }
  if (d.dyn == KIND_ARM) {
    if (d.n_link < 0 || (d.n_link > 0 && !finite_arr(d.link_spheres, 5LL * d.n_link))) bad("link spheres");
    for (int l = 0; l < d.n_link; ++l) {
      int li = (int)d.link_spheres[5 * l];
      if (li < 1 || li > 7) bad("link index must be 1..7");
    }
  } else if (d.n_link != 0) {
    bad("n_link only for the arm");
  }
  if (!d.u_lo || !d.u_hi || !d.x_lo || !d.x_hi) bad("bounds arrays required (use ±inf)");
  for (int i = 0; i < d.nu; ++i) {
    if (std::isnan(d.u_lo[i]) || std::isnan(d.u_hi[i])) bad("NaN control bound");
    if (std::isfinite(d.u_lo[i]) && std::isfinite(d.u_hi[i]) && d.u_lo[i] > d.u_hi[i]) bad("u_lo > u_hi");
  }
  for (int i = 0; i < d.nx; ++i)
    if (std::isnan(d.x_lo[i]) || std::isnan(d.x_hi[i])) bad("NaN state bound");
  std::vector<double> C(d.nx * d.nx);
  for (int m = 0; m <= d.T; ++m) {
    for (int k = 0; k < d.nx * d.nx; ++k) C[k] = d.Sigma[(long long)m * d.nx * d.nx + k];
    for (int r = 0; r < d.nx; ++r)
      for (int c = 0; c < r; ++c)
        if (std::fabs(C[r * d.nx + c] - C[c * d.nx + r]) > 1e-12 * (std::fabs(C[r * d.nx + c]) + 1e-300)) bad("Sigma block not symmetric");
    if (!chol_inplace(C.data(), d.nx)) {
      // a singular block (a per-step disturbance map Γ_i of lower rank): positive semidefinite is enough
      std::vector<double> A(d.nx * d.nx), V(d.nx * d.nx), lam(d.nx);
      for (int k = 0; k < d.nx * d.nx; ++k) A[k] = d.Sigma[(long long)m * d.nx * d.nx + k];
      jacobi_eig(A.data(), d.nx, lam.data(), V.data());
      double lmax = 0.0, lmin = 0.0;
      for (int k = 0; k < d.nx; ++k) { lmax = std::max(lmax, std::fabs(lam[k])); lmin = std::min(lmin, lam[k]); }
      if (lmin < -1e-12 * std::max(lmax, 1e-300)) bad("Sigma block not positive semidefinite");
    }
  }
}

// rows of one instance in the shared row order
// Row counts of build_rows without building the rows.
void count_rows(const nrto_problem_desc& d, long long& n_sr, long long& n_cr) {
  long long per_t = (long long)d.n_obs * (d.dyn == KIND_ARM ? d.n_link : 1), per_k = 0;
  for (int i = 0; i < d.nx; ++i) per_t += (std::isfinite(d.x_hi[i]) ? 1 : 0) + (std::isfinite(d.x_lo[i]) ? 1 : 0);
  for (int i = 0; i < d.nu; ++i) per_k += (std::isfinite(d.u_hi[i]) ? 1 : 0) + (std::isfinite(d.u_lo[i]) ? 1 : 0);
  n_sr = per_t * d.T;
  n_cr = per_k * d.T;
}

void build_rows(const nrto_problem_desc& d, std::vector<int4>& srows, std::vector<int4>& crows, int& rows_per_t) {
  srows.clear();
  crows.clear();
  rows_per_t = 0;
  for (int t = 1; t <= d.T; ++t) {
    size_t before = srows.size();
    if (d.dyn == KIND_ARM) {
      for (int l = 0; l < d.n_link; ++l)
        for (int o = 0; o < d.n_obs; ++o) srows.push_back(make_int4(t, ROW_SPHERE, o, l));
    } else {
      for (int o = 0; o < d.n_obs; ++o) srows.push_back(make_int4(t, ROW_SPHERE, o, -1));
    }
    for (int i = 0; i < d.nx; ++i) {
      if (std::isfinite(d.x_hi[i])) srows.push_back(make_int4(t, ROW_XHI, i, -1));
      if (std::isfinite(d.x_lo[i])) srows.push_back(make_int4(t, ROW_XLO, i, -1));
    }
    rows_per_t = (int)(srows.size() - before);
  }
  for (int k = 0; k < d.T; ++k)
    for (int i = 0; i < d.nu; ++i) {
      if (std::isfinite(d.u_hi[i])) crows.push_back(make_int4(k, ROW_UHI, i, -1));
      if (std::isfinite(d.u_lo[i])) crows.push_back(make_int4(k, ROW_ULO, i, -1));
    }
}

void pack_params(const nrto_problem_desc& d, const Arena& L, double* dst) {
  auto put = [&](long long off, const double* src, long long n) { for (long long i = 0; i < n; ++i) dst[off + i] = src[i]; };
  put(L.x0, d.x0, d.nx); put(L.xg, d.x_goal, d.nx); put(L.uref, d.u_ref, d.nu);
  put(L.Qx, d.Qx, d.nx); put(L.Ru, d.Ru, d.nu); put(L.RK, d.RK, d.nu);
  put(L.ulo, d.u_lo, d.nu); put(L.uhi, d.u_hi, d.nu); put(L.xlo, d.x_lo, d.nx); put(L.xhi, d.x_hi, d.nx);
  if (d.n_dyn_params > 0) put(L.dyn, d.dyn_params, d.n_dyn_params);
  for (int i = d.n_dyn_params; i < MAX_DYN; ++i) dst[L.dyn + i] = 0.0;   // the staging is reused across updates
  if (d.dyn == KIND_ARM && d.n_dyn_params == 21)
    for (int i = 0; i < 7; ++i) dst[L.dyn + ARM_INERT + i] = 1.0;   // the double integrator: unit inertia
  for (int o = 0; o < d.n_obs; ++o) {
    for (int k = 0; k < 3; ++k) dst[L.obs + 4 * o + k] = (k < d.obs_dim) ? d.obs_center[o * d.obs_dim + k] : 0.0;
    dst[L.obs + 4 * o + 3] = d.obs_radius[o];
  }
  if (d.n_link > 0) put(L.link, d.link_spheres, 5LL * d.n_link);
  put(L.Sigma, d.Sigma, (long long)(d.T + 1) * d.nx * d.nx);
}

template <typename Real>
void launch_setup(nrto_problem* P) {
  k_setup<Real><<<P->n, 128, 0, P->stream>>>(P->dev<Real>());
  P->check_launch("k_setup");
}

// slot_sel: -1 = current slot of each instance, -2 = candidate slot (1 - current)
template <typename Real>
void launch_linearize(nrto_problem* P, int slot_sel) {
  Dev<Real> D = P->dev<Real>();
  k_rollout_jac<Real><<<P->n, 128, 0, P->stream>>>(D, slot_sel);
  P->check_launch("k_rollout_jac");
  k_rows<Real><<<P->n, 256, 0, P->stream>>>(D, slot_sel);
  P->check_launch("k_rows");
  k_adjoint<Real><<<P->n, 256, 0, P->stream>>>(D, slot_sel);
  P->check_launch("k_adjoint");
  k_gram<Real><<<P->n, 256, 0, P->stream>>>(D, slot_sel);
  P->check_launch("k_gram");
}

// One persistent launch of a solver kernel (FullADMM or NRTO-DR) for the instances of one kind:
// as many CTAs as fit on the GPU, at most one per instance; CTAs take instances from the queue.
template <int NX, int NU, typename Real>
void launch_solver_kind(nrto_problem* P, int solver, const KindLaunch& kl, SolveParams sp, cudaStream_t st,
                        int grid_cap) {
  using SK = SolverKernel<NX, NU, Real>;
  const char* name = solver == SOLVER_KERNEL_FULLADMM ? "k_fulladmm" : "k_dr";
  int dev = 0, nsm = 0, per_sm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(SK::configure(solver, kl.smem, &per_sm));
  if (per_sm < 1) fail(NRTO_ERR_CUDA, std::string(name) + " does not fit on an SM");
  int grid = std::min(kl.count, nsm * per_sm);
  if (grid_cap > 0) grid = std::min(grid, grid_cap);
  sp.chunk = kl.chunk; sp.max_rows = kl.max_rows; sp.tmax = kl.tmax; sp.n_order = kl.count;
  sp.order0 = kl.order0; sp.queue_idx = kl.kind;
  const cudaError_t le = SK::launch(solver, grid, kl.smem, st, P->dev<Real>(), sp);
  ++P->launches;
  if (le != cudaSuccess) fail(NRTO_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(le));
  if (P->profiling) P->prof_launches++;
}

// The persistent solver launches of every dynamics kind present: the first on the problem's stream,
// the others on the second stream between fork / join events, so that a kind's CTAs start on the SMs
// that the previous kind's launch frees at its end.  Profiling records one event pair around them.
template <typename Real>
void launch_solver_kinds(nrto_problem* P, int solver, const SolveParams& sp) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (P->profiling) {
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, P->stream));
  }
  int kinds[3] = {0, 1, 2};
  std::stable_sort(kinds, kinds + 3, [&](int a, int b) { return P->kl[a].entries > P->kl[b].entries; });
  // launch mapping (nrto_set_launch_mapping / nrto_autotune): 0 kinds one after another on the problem's
  // stream; 1 kinds at the same time, each with as many CTAs as fit; 2 and 3 at the same time with the
  // SMs split between the kinds in proportion to their row entries (2) or row entries × horizon (3)
  int caps[3] = {0, 0, 0};
  if (P->mapping >= 2) {
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    double wsum = 0.0, wk[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k)
      if (P->kl[k].count > 0) {
        wk[k] = (double)P->kl[k].entries * (P->mapping == 3 ? (double)P->kl[k].tmax : 1.0);
        wsum += wk[k];
      }
    for (int k = 0; k < 3; ++k)
      if (P->kl[k].count > 0) caps[k] = std::max(1, (int)(nsm * wk[k] / wsum));
  }
  int launched = 0;
  bool forked = false;
  for (int k : kinds) {
    const KindLaunch& kl = P->kl[k];
    if (kl.count == 0) continue;
    cudaStream_t st = P->stream;
    if (launched > 0 && P->stream2 && P->mapping != 0) {
      if (!forked) {
        CK(cudaEventRecord(P->ev_fork, P->stream));
        CK(cudaStreamWaitEvent(P->stream2, P->ev_fork, 0));
        forked = true;
      }
      st = P->stream2;
    }
    if (k == KIND_UNICYCLE) launch_solver_kind<3, 2, Real>(P, solver, kl, sp, st, caps[k]);
    else if (k == KIND_QUADCOPTER) launch_solver_kind<12, 4, Real>(P, solver, kl, sp, st, caps[k]);
    else launch_solver_kind<14, 7, Real>(P, solver, kl, sp, st, caps[k]);
    ++launched;
  }
  if (forked) {
    CK(cudaEventRecord(P->ev_join, P->stream2));
    CK(cudaStreamWaitEvent(P->stream, P->ev_join, 0));
  }
  if (P->profiling) {
    CK(cudaEventRecord(e1, P->stream));
    P->prof_events.push_back({e0, e1});
  }
}

template <typename Real>
void launch_solve(nrto_problem* P, const nrto_solver_opts& o) {
  Dev<Real> D = P->dev<Real>();
  SolveParams sp{};
  sp.rho = o.rho; sp.eps_p = o.eps_p; sp.eps_d = o.eps_d;
  sp.alpha = o.alpha; sp.r_chi = o.r_chi; sp.sigma = o.sigma; sp.eps_dr = o.eps_dr;
  sp.max_iter = o.max_inner; sp.check = o.check; sp.max_dr = o.max_dr;
  sp.warm = P->warm_pending ? 1 : ((o.carry && P->carry_ok && o.solver == NRTO_SOLVER_FULLADMM) ? 2 : 0);
  sp.adapt_every = o.adapt_every; sp.stall_every = o.stall_every;
  sp.adapt_mu = o.adapt_mu; sp.adapt_tau = o.adapt_tau; sp.rho_min = o.rho_min; sp.rho_max = o.rho_max;
  sp.stall_ratio = o.stall_ratio;
  sp.stall_budget = o.stall_budget;
  sp.fallback = o.warm_fallback;
  sp.kv_pcg_iters = o.solver == NRTO_SOLVER_FULLADMM ? o.kv_pcg_iters : 0;
  sp.kv_pcg_tol = o.kv_pcg_tol;
  if (P->wlift_pending && o.solver != NRTO_SOLVER_FULLADMM)
    fail(NRTO_ERR_STATE, "a lifted warm start applies to NRTO_SOLVER_FULLADMM only");
  P->warm_pending = false;
  P->wlift_pending = false;
  if (o.solver == NRTO_SOLVER_FULLADMM) {
    k_gain_factors<Real><<<P->n, 128, 0, P->stream>>>(D, o.rho, 0.0, sp.warm);
    P->check_launch("k_gain_factors");
    k_riccati_factor<Real><<<P->n, 32, 0, P->stream>>>(D, o.rho, sp.warm);
    P->check_launch("k_riccati_factor");
    CK(cudaMemsetAsync(P->d_queue, 0, 4 * sizeof(int), P->stream));
    launch_solver_kinds<Real>(P, SOLVER_KERNEL_FULLADMM, sp);
    P->carry_ok = true;
  } else if (o.solver == NRTO_SOLVER_FULLADMM_AW) {
    // block 2a factors its own Newton systems; only the gain-solve factors are needed
    k_gain_factors<Real><<<P->n, 128, 0, P->stream>>>(D, o.rho, 0.0, 0);
    P->check_launch("k_gain_factors");
    CK(cudaMemsetAsync(P->d_queue, 0, 4 * sizeof(int), P->stream));
    launch_solver_kinds<Real>(P, SOLVER_KERNEL_FULLADMM_AW, sp);
    P->carry_ok = false;
  } else {
    launch_dr<Real>(P, o, sp);
    P->carry_ok = false;
  }
}

// k_merit with the Gtᵀ table of the longest horizon of the batch in dynamic shared memory
template <typename Real>
void launch_merit(nrto_problem* P, int slot_sel, int kbuf, int gtbuf, double w_p, int out_idx) {
  size_t bytes = 0;
  for (int k = 0; k < 3; ++k)
    if (P->kl[k].count > 0)
      bytes = std::max(bytes, (size_t)(P->kl[k].tmax + 1) * kind_nu(k) * kind_nx(k) * sizeof(Real));
  CK(cudaFuncSetAttribute(k_merit<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  k_merit<Real><<<P->n, 256, bytes, P->stream>>>(P->dev<Real>(), slot_sel, kbuf, gtbuf, w_p, out_idx);
  P->check_launch("k_merit");
}

template <typename Real>
void launch_merit_current(nrto_problem* P, double w_p) {
  Dev<Real> D = P->dev<Real>();
  k_gain_to_gt<Real><<<P->n, 256, 0, P->stream>>>(D, 3, 0);
  P->check_launch("k_gain_to_gt");
  launch_merit<Real>(P, -1, 3, 0, w_p, SC_PHI);
}

template <typename Real>
void launch_outer_step(nrto_problem* P, const nrto_solver_opts& o) {
  Dev<Real> D = P->dev<Real>();
  launch_solve<Real>(P, o);
  k_candidate<Real><<<P->n, 128, 0, P->stream>>>(D);
  P->check_launch("k_candidate");
  launch_linearize<Real>(P, -2);
  k_gain_to_gt<Real><<<P->n, 256, 0, P->stream>>>(D, 1, 1);
  P->check_launch("k_gain_to_gt");
  launch_merit<Real>(P, -2, 1, 1, o.w_p, SC_PHI_CAND);
  k_accept<Real><<<P->n, 128, 0, P->stream>>>(D, o.r0, o.r_min);
  P->check_launch("k_accept");
}

// Threads of one row group of the solver kernels' row pass for the longest horizon of a launch; it
// must not exceed the CTA, or some columns of the rows would have no thread.
template <int NX, int NU, typename Real>
int row_group_threads(int tmax) {
  using C = FACfg<NX, NU, Real>;
  return ((tmax / 2 + 1) * C::NCG + 31) / 32 * 32;
}

template <typename Real>
void check_row_groups(const KindLaunch& kl) {
  int tpg = 0, nt = 0;
  if (kl.kind == KIND_UNICYCLE) { tpg = row_group_threads<3, 2, Real>(kl.tmax); nt = FACfg<3, 2, Real>::NT; }
  else if (kl.kind == KIND_QUADCOPTER) { tpg = row_group_threads<12, 4, Real>(kl.tmax); nt = FACfg<12, 4, Real>::NT; }
  else { tpg = row_group_threads<14, 7, Real>(kl.tmax); nt = FACfg<14, 7, Real>::NT; }
  if (tpg > nt) fail(NRTO_ERR_INVALID, "horizon too long for the solver kernel's thread block");
}

// Largest chunk of row entries staged per bulk-copy round (the budget of shared memory may cut it).
#ifndef NRTO_CHUNK_MAX
#define NRTO_CHUNK_MAX 12288
#endif

template <typename Real>
void choose_chunk(KindLaunch& kl) {
  check_row_groups<Real>(kl);
  const int nx = kind_nx(kl.kind);
  const int minc = ((kl.tmax + 1) * nx + 3) & ~3;
  int chunk = NRTO_CHUNK_MAX;
  while (chunk > minc && smem_for<Real>(kl.kind, chunk, chunk / (2 * nx) + 2) > (size_t)smem_budget<Real>(kl.kind)) chunk -= 256;
  if (chunk < minc) chunk = minc;
  kl.chunk = chunk;
  kl.max_rows = chunk / (2 * nx) + 2;
  kl.smem = smem_for<Real>(kl.kind, chunk, kl.max_rows);
  if (kl.smem > (size_t)smem_budget<Real>(kl.kind)) fail(NRTO_ERR_INVALID, "horizon too long for the shared-memory budget of this precision");
  // the block-2 sweep keeps q, r, l and a ring of >= 2 factor records in the chunk buffers
  const int nu = kind_nu(kl.kind);
  size_t bb = 0;
  if (kl.kind == KIND_UNICYCLE) bb = FASmem<3, 2, Real>::buf_bytes(chunk, kl.max_rows);
  else if (kl.kind == KIND_QUADCOPTER) bb = FASmem<12, 4, Real>::buf_bytes(chunk, kl.max_rows);
  else bb = FASmem<14, 7, Real>::buf_bytes(chunk, kl.max_rows);
  size_t fixed = 0;
  if (kl.kind == KIND_UNICYCLE) fixed = B2Smem<3, 2, Real>::fixed_bytes(kl.tmax);
  else if (kl.kind == KIND_QUADCOPTER) fixed = B2Smem<12, 4, Real>::fixed_bytes(kl.tmax);
  else fixed = B2Smem<14, 7, Real>::fixed_bytes(kl.tmax);
  const size_t need = fixed + 2 * (size_t)pk_stride(nx, nu) * sizeof(Real);
  if (need > 2 * bb) fail(NRTO_ERR_INVALID, "internal: chunk buffers too small for the block-2 sweep");
}

// Per-instance field of the batch (device → host): one gather launch into a contiguous device
// buffer, then one copy.
void copy_arena_field(nrto_problem* P, int field, double* dst) {
  const bool per_k = field == GF_K1 || field == GF_KACC;
  const long long total = per_k ? P->k_total : P->u_total;
  k_gather_field<<<P->n, 128, 0, P->stream>>>(P->d_inst, P->d_is, P->d_arena, P->d_slot_arena[0], P->d_slot_arena[1],
                                              field, per_k ? P->d_koff : P->d_uoff, P->d_gather, P->n);
  P->check_launch("k_gather_field");
  if (total > 0) CK(cudaMemcpyAsync(dst, P->d_gather, sizeof(double) * total, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
}


nrto_status handle(const std::exception& e) {
  if (auto ne = dynamic_cast<const NrtoError*>(&e)) {
    g_last_error = ne->what();
    return ne->st;
  }
  g_last_error = e.what();
  return NRTO_ERR_INVALID;
}

// Runs f(i) for i in [0, n) on up to hardware_concurrency host threads.  A failure of instance i is
// kept, and the failure of the lowest index is rethrown after all threads finish, so the reported
// error does not depend on scheduling.
template <typename F>
void parallel_instances(int n, F f) {
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), (n + 63) / 64));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::exception_ptr> err(nt);
  std::vector<int> err_at(nt, n);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < n; i += nt) {
        try {
          f(i);
        } catch (...) {
          err[t] = std::current_exception();
          err_at[t] = i;
          return;
        }
      }
    });
  for (auto& x : th) x.join();
  int first = -1;
  for (int t = 0; t < nt; ++t)
    if (err[t] && (first < 0 || err_at[t] < err_at[first])) first = t;
  if (first >= 0) std::rethrow_exception(err[first]);
}

void upload_params(nrto_problem* P, const nrto_problem_desc* descs) {
  std::vector<double> sv, uv;
  if (!P->carve_base && !P->h_stage) {
    CK(cudaHostAlloc(reinterpret_cast<void**>(&P->h_stage), sizeof(double) * std::max<long long>(P->stage_total, 1),
                     cudaHostAllocDefault));
    CK(cudaHostAlloc(reinterpret_cast<void**>(&P->h_ustage), sizeof(double) * std::max<long long>(P->u_total, 1),
                     cudaHostAllocDefault));
    std::memset(P->h_stage, 0, sizeof(double) * P->stage_total);
    std::memset(P->h_ustage, 0, sizeof(double) * P->u_total);
  }
  double* stage = P->h_stage;
  double* ust = P->h_ustage;
  if (!stage) {
    sv.assign(P->stage_total, 0.0);
    uv.assign(P->u_total, 0.0);
    stage = sv.data();
    ust = uv.data();
  }
  parallel_instances(P->n, [&](int i) {
    const Inst& I = P->h_inst[i];
    const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
    pack_params(descs[i], L, stage + P->stage_off[i]);
    std::memcpy(ust + P->uoff[i], descs[i].u_init, sizeof(double) * I.T * I.nu);
  });
  CK(cudaMemcpyAsync(P->d_stage, stage, sizeof(double) * P->stage_total, cudaMemcpyHostToDevice, P->stream));
  CK(cudaMemcpyAsync(P->d_ustage, ust, sizeof(double) * P->u_total, cudaMemcpyHostToDevice, P->stream));
  k_scatter<<<P->n, 256, 0, P->stream>>>(P->d_arena, P->d_inst, P->d_stage, P->d_stage_off, P->d_stage_len, P->n);
  P->check_launch("k_scatter");
  for (int s = 0; s < 2; ++s) {
    k_scatter_uhat<<<P->n, 128, 0, P->stream>>>(P->d_slot_arena[s], P->d_inst, P->d_ustage, P->d_uoff, P->n);
    P->check_launch("k_scatter_uhat");
  }
  CK(cudaStreamSynchronize(P->stream));   // the staging is reused (or goes out of scope) after this
}

void check_opts(const nrto_solver_opts* o) {
  if (!o) fail(NRTO_ERR_INVALID, "null options");
  if (o->solver != NRTO_SOLVER_DR && o->solver != NRTO_SOLVER_FULLADMM && o->solver != NRTO_SOLVER_FULLADMM_AW)
    fail(NRTO_ERR_INVALID, "unknown solver");
  if (!(o->rho > 0)) fail(NRTO_ERR_INVALID, "rho must be positive");
  if (o->max_inner < 0 || o->max_inner > 1000000) fail(NRTO_ERR_INVALID, "max_inner out of range");
  if (o->adapt_every < 0 || o->stall_every < 0) fail(NRTO_ERR_INVALID, "adapt_every and stall_every must be >= 0");
  if (o->adapt_every > 0 && !(o->adapt_mu > 1 && o->adapt_tau > 1 && o->rho_min > 0 && o->rho_max >= o->rho_min))
    fail(NRTO_ERR_INVALID, "residual balancing needs mu > 1, tau > 1, 0 < rho_min <= rho_max");
  if (o->stall_every > 0 && !(o->stall_ratio > 0 && o->stall_ratio < 1)) fail(NRTO_ERR_INVALID, "stall_ratio must be in (0,1)");
  if (!(o->stall_budget >= 0 && o->stall_budget < 1e300)) fail(NRTO_ERR_INVALID, "stall_budget must be finite and >= 0");
  if (o->carry != 0 && o->carry != 1) fail(NRTO_ERR_INVALID, "carry must be 0 or 1");
  if (o->max_inner_final < 0 || o->max_inner_final > 1000000) fail(NRTO_ERR_INVALID, "max_inner_final out of range");
  if (o->kv_pcg_iters < 0 || o->kv_pcg_iters > 1000000) fail(NRTO_ERR_INVALID, "kv_pcg_iters out of range");
  if (o->kv_pcg_iters > 0 && o->solver != NRTO_SOLVER_FULLADMM)
    fail(NRTO_ERR_INVALID, "kv_pcg_iters applies to NRTO_SOLVER_FULLADMM only");
  if (o->kv_pcg_iters > 0 && !(o->kv_pcg_tol >= 0 && o->kv_pcg_tol < 1)) fail(NRTO_ERR_INVALID, "kv_pcg_tol must be in [0,1)");
  if (o->solver == NRTO_SOLVER_DR) {
    if (!(o->alpha > 0 && o->alpha < 2)) fail(NRTO_ERR_INVALID, "alpha must be in (0,2)");
    if (!(o->r_chi > 0) || !(o->sigma > 0)) fail(NRTO_ERR_INVALID, "r_chi and sigma must be positive");
    if (o->max_dr < 1 || o->max_dr > 1000000) fail(NRTO_ERR_INVALID, "max_dr out of range");
  }
}

nrto_status finish_statuses(nrto_problem* p, const nrto_solver_opts* o, nrto_socp_out* out) {
  std::vector<int> is(p->n * NIS);
  std::vector<double> sc(p->n * NSC);
  CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(sc.data(), p->d_sc, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
  if (out->du) copy_arena_field(p, GF_DU, out->du);
  if (out->K) copy_arena_field(p, GF_K1, out->K);
  if (out->p) CK(cudaMemcpyAsync(out->p, p->d_p, sizeof(double) * p->n_rows, cudaMemcpyDeviceToHost, p->stream));
  if (out->ptilde) CK(cudaMemcpyAsync(out->ptilde, p->d_pt, sizeof(double) * p->n_rows, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  nrto_status st = NRTO_OK;
  for (int i = 0; i < p->n; ++i) {
    if (out->iters) out->iters[i] = is[i * NIS + IS_ITERS];
    if (out->status) out->status[i] = is[i * NIS + IS_STATUS];
    if (out->r_p) out->r_p[i] = sc[i * NSC + SC_RP];
    if (out->r_d) out->r_d[i] = sc[i * NSC + SC_RD];
    if (is[i * NIS + IS_STATUS] == ST_NUMERIC) st = NRTO_ERR_NUMERIC;
    else if (o->check && is[i * NIS + IS_STATUS] == ST_MAXITER && st == NRTO_OK) st = NRTO_ERR_NOT_CONVERGED;
  }
  if (st != NRTO_OK) g_last_error = st == NRTO_ERR_NUMERIC ? "non-finite residual in some instance" : "some instance hit its iteration cap";
  return st;
}

long long field_count(const Inst& I, int f) {
  switch (f) {
    case NRTO_F_XHAT: case NRTO_F_DX: return (long long)(I.T + 1) * I.nx;
    case NRTO_F_UHAT: case NRTO_F_DU: return (long long)I.T * I.nu;
    case NRTO_F_A: return (long long)I.T * I.nx * I.nx;
    case NRTO_F_B: return (long long)I.T * I.nx * I.nu;
    case NRTO_F_G0: case NRTO_F_P: case NRTO_F_PT: case NRTO_F_LAMP: return I.n_sr + I.n_cr;
    case NRTO_F_BHAT: return I.n_ent_state;
    case NRTO_F_BVEC: return (I.n_ent_state / I.nx) * I.nu;
    case NRTO_F_LAMNU: return I.n_ent_state + (long long)I.n_cr * I.nx;
    case NRTO_F_K: case NRTO_F_KACC: return (long long)I.T * I.nu * I.nx;
    case NRTO_F_GM: return (long long)I.T * I.nu * I.nu;
    case NRTO_F_SCAL: return 8;
    case NRTO_F_STATS: return 7;
    case NRTO_F_LAMW: case NRTO_F_S: return I.n_sr + I.n_cr;
    case NRTO_F_LAME: return (long long)(I.T + 1) * I.nx;
  }
  return -1;
}

nrto_status exchange(nrto_problem_t p, int field, int i, double* buf, long long count, bool to_host) {
  try {
    if (!p || !buf || i < 0 || i >= p->n) fail(NRTO_ERR_INVALID, "bad problem, instance or buffer");
    const Inst& I = p->h_inst[i];
    const long long need = field_count(I, field);
    if (need < 0) fail(NRTO_ERR_INVALID, "unknown field");
    if (count != need) fail(NRTO_ERR_INVALID, "count must be " + std::to_string(need));
    CK(cudaStreamSynchronize(p->stream));
    int is[NIS];
    CK(cudaMemcpy(is, p->d_is + i * NIS, sizeof(is), cudaMemcpyDeviceToHost));
    const int sl = is[IS_SLOT];
    const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
    const SlotL SL = slot_layout(I.nx, I.nu, I.T);
    const size_t rs = p->prec == NRTO_PREC_FP64 ? 8 : 4;
    double* dptr = nullptr;
    void* rptr = nullptr;   // arrays stored in the compute precision
    switch (field) {
      case NRTO_F_XHAT: dptr = p->d_slot_arena[sl] + I.slot0 + SL.x_hat; break;
      case NRTO_F_UHAT: dptr = p->d_slot_arena[sl] + I.slot0 + SL.u_hat; break;
      case NRTO_F_A: dptr = p->d_slot_arena[sl] + I.slot0 + SL.A; break;
      case NRTO_F_B: dptr = p->d_slot_arena[sl] + I.slot0 + SL.B; break;
      case NRTO_F_GM: dptr = p->d_slot_arena[sl] + I.slot0 + SL.Gm; break;
      case NRTO_F_G0: dptr = p->d_g0[sl] + I.row0; break;
      case NRTO_F_P: dptr = p->d_p + I.row0; break;
      case NRTO_F_PT: dptr = p->d_pt + I.row0; break;
      case NRTO_F_LAMP: dptr = p->d_lamp + I.row0; break;
      case NRTO_F_K: dptr = p->d_arena + I.arena0 + L.K1; break;
      case NRTO_F_KACC: dptr = p->d_arena + I.arena0 + L.Kacc; break;
      case NRTO_F_DU: dptr = p->d_arena + I.arena0 + L.du; break;
      case NRTO_F_DX: dptr = p->d_arena + I.arena0 + L.dx; break;
      case NRTO_F_LAMW: dptr = p->d_lamw + I.row0; break;
      case NRTO_F_S: dptr = p->d_s + I.row0; break;
      case NRTO_F_LAME: dptr = p->d_arena + I.arena0 + L.lam_e; break;
      case NRTO_F_BHAT: rptr = static_cast<char*>(p->d_bhat[sl]) + rs * I.ent0; break;
      case NRTO_F_BVEC: rptr = static_cast<char*>(p->d_bvec[sl]) + rs * I.bent0; break;
      case NRTO_F_LAMNU: rptr = static_cast<char*>(p->d_lam) + rs * I.ent0; break;
      case NRTO_F_STATS: {
        if (!to_host) fail(NRTO_ERR_INVALID, "stats are read-only");
        double scv[NSC];
        CK(cudaMemcpy(scv, p->d_sc + (long long)i * NSC, sizeof(scv), cudaMemcpyDeviceToHost));
        buf[0] = is[IS_CUMITERS]; buf[1] = is[IS_ITERS]; buf[2] = is[IS_STATUS]; buf[3] = is[IS_NACC];
        buf[4] = scv[SC_RHO]; buf[5] = is[IS_DRITERS]; buf[6] = is[IS_FALLBACK];
        return NRTO_OK;
      }
      case NRTO_F_SCAL: {
        double sc[NSC];
        CK(cudaMemcpy(sc, p->d_sc + (long long)i * NSC, sizeof(sc), cudaMemcpyDeviceToHost));
        const int idx[8] = {SC_RP, SC_RD, SC_RPP, SC_RDP, SC_PHI, SC_PHI_CAND, SC_COST, SC_RTRUST};
        if (to_host) {
          for (int k = 0; k < 8; ++k) buf[k] = sc[idx[k]];
        } else {
          for (int k = 0; k < 8; ++k) sc[idx[k]] = buf[k];
          CK(cudaMemcpy(p->d_sc + (long long)i * NSC, sc, sizeof(sc), cudaMemcpyHostToDevice));
        }
        return NRTO_OK;
      }
    }
    if (dptr) {
      CK(cudaMemcpy(to_host ? (void*)buf : (void*)dptr, to_host ? (void*)dptr : (void*)buf, sizeof(double) * count,
                    to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice));
      return NRTO_OK;
    }
    // Ragged fields: the device layout has padding at chunk starts; map compact <-> padded
    // element by element through the row tables.
    const bool is_b = field == NRTO_F_BVEC;
    const int nrow = field == NRTO_F_LAMNU ? I.n_sr + I.n_cr : I.n_sr;
    const long long base = is_b ? I.bent0 : I.ent0;
    long long span = 0;
    std::vector<std::pair<long long, long long>> seg;   // (padded offset rel. base, length)
    for (int r = 0; r < nrow; ++r) {
      const long long R = I.row0 + r;
      const int4 ri = p->h_rinfo[R];
      const long long len = r < I.n_sr ? (long long)(ri.x + 1) * (is_b ? I.nu : I.nx) : I.nx;
      const long long off = (is_b ? p->h_rbent[R] : p->h_rent[R]) - base;
      seg.push_back({off, len});
      span = std::max(span, off + len);
    }
    std::vector<double> full(span);
    if (!to_host) {
      // read-modify-write so that padding keeps its contents
      if (p->prec == NRTO_PREC_FP64) {
        CK(cudaMemcpy(full.data(), rptr, sizeof(double) * span, cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> tmp(span);
        CK(cudaMemcpy(tmp.data(), rptr, sizeof(float) * span, cudaMemcpyDeviceToHost));
        for (long long k = 0; k < span; ++k) full[k] = tmp[k];
      }
      long long o = 0;
      for (auto& sg : seg) { for (long long k = 0; k < sg.second; ++k) full[sg.first + k] = buf[o + k]; o += sg.second; }
    }
    if (p->prec == NRTO_PREC_FP64) {
      CK(cudaMemcpy(to_host ? (void*)full.data() : rptr, to_host ? rptr : (void*)full.data(), sizeof(double) * span,
                    to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice));
    } else {
      std::vector<float> tmp(span);
      if (to_host) {
        CK(cudaMemcpy(tmp.data(), rptr, sizeof(float) * span, cudaMemcpyDeviceToHost));
        for (long long k = 0; k < span; ++k) full[k] = tmp[k];
      } else {
        for (long long k = 0; k < span; ++k) tmp[k] = (float)full[k];
        CK(cudaMemcpy(rptr, tmp.data(), sizeof(float) * span, cudaMemcpyHostToDevice));
      }
    }
    if (to_host) {
      long long o = 0;
      for (auto& sg : seg) { for (long long k = 0; k < sg.second; ++k) buf[o + k] = full[sg.first + k]; o += sg.second; }
    }
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

}  // namespace

// Warm start from network outputs Y (device, n × out_dim): K from Y[i][k ..], p̃ and λ_p of instance
// row r from Y[i][pt + map[r]] and Y[i][lp + map[r]] (map < 0: zero).  Lifted parts, each absent
// (zero; the solver's ρ) when its offset is < 0: per row θ (clipped at 0, into D.dd) and λ_w, per
// instance δû (T·nu) and λ_e (steps 1..T, T·nx), and the penalty exp(Y[i][rho]).
struct WarmOffsets {
  int k, pt, lp, th, lw, du, le, rho;
  NRTO_HD bool lifted() const { return th >= 0 || lw >= 0 || du >= 0 || le >= 0 || rho >= 0; }
};
template <typename Real>
__global__ void k_scatter_warm(Dev<Real> D, const float* Y, int out_dim, const int* map, WarmOffsets o) {
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  double* ar = D.arena + I.arena0;
  const float* y = Y + (long long)i * out_dim;
  for (int q = threadIdx.x; q < I.T * I.nu * I.nx; q += blockDim.x) ar[L.K1 + q] = (double)y[o.k + q];
  for (int r = threadIdx.x; r < I.n_sr + I.n_cr; r += blockDim.x) {
    const long long R = I.row0 + r;
    const int m = map[R];
    D.pt[R] = m >= 0 ? (double)y[o.pt + m] : 0.0;
    D.lamp[R] = m >= 0 ? (double)y[o.lp + m] : 0.0;
    if (o.lifted()) {
      D.dd[R] = (m >= 0 && o.th >= 0) ? fmax((double)y[o.th + m], 0.0) : 0.0;
      D.lamw[R] = (m >= 0 && o.lw >= 0) ? (double)y[o.lw + m] : 0.0;
    }
  }
  if (!o.lifted() && threadIdx.x == 0) D.is[i * NIS + IS_WLIFT] = 0;
  if (o.lifted()) {
    for (int q = threadIdx.x; q < I.T * I.nu; q += blockDim.x) ar[L.du + q] = o.du >= 0 ? (double)y[o.du + q] : 0.0;
    for (int q = threadIdx.x; q < I.T * I.nx; q += blockDim.x)
      ar[L.lam_e + I.nx + q] = o.le >= 0 ? (double)y[o.le + q] : 0.0;
    if (threadIdx.x == 0) {
      D.is[i * NIS + IS_WLIFT] = 1;
      D.sc[(long long)i * NSC + SC_RHOW] = o.rho >= 0 ? exp((double)y[o.rho]) : 0.0;
    }
  }
}

const float* nrto_mlp_internal_forward_device(nrto_mlp_t m, const float* x, int batch, int* out_dim,
                                              cudaStream_t* stream);   // mlp.cu

// Message for nrto_last_error from the other translation units of the library.
void nrto_internal_set_error(const std::string& msg) { g_last_error = msg; }

// =============================================================================================
extern "C" {

const char* nrto_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Body of nrto_problem_create.  carve_base == nullptr: every device buffer comes from cudaMalloc;
// otherwise buffers are cut from [carve_base, carve_base + carve_cap).
nrto_status create_problem(const nrto_problem_desc* descs, int n, int precision, void* stream, char* carve_base,
                           size_t carve_cap, nrto_problem_t* out) {
  nrto_problem* P = nullptr;
  try {
    g_last_error.clear();
    if (!descs || n <= 0 || !out) fail(NRTO_ERR_INVALID, "descs, n > 0 and out are required");
    if (precision != NRTO_PREC_FP64 && precision != NRTO_PREC_MIXED) fail(NRTO_ERR_INVALID, "unknown precision");
    for (int i = 0; i < n; ++i) validate(descs[i], i);
    P = new nrto_problem();
    P->carve_base = carve_base;
    P->carve_cap = carve_cap;
    P->n = n;
    P->prec = precision;
    P->stream = static_cast<cudaStream_t>(stream);
    if (!carve_base) {
      CK(cudaStreamCreateWithFlags(&P->stream2, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
    }
    for (int k = 0; k < 3; ++k) P->kl[k].kind = k;
    for (int i = 0; i < n; ++i) {
      KindLaunch& kl = P->kl[descs[i].dyn];
      kl.count++;
      kl.tmax = std::max(kl.tmax, descs[i].T);
    }
    for (int k = 0; k < 3; ++k)
      if (P->kl[k].count > 0) {
        if (precision == NRTO_PREC_FP64) choose_chunk<double>(P->kl[k]);
        else choose_chunk<float>(P->kl[k]);
      }
    std::vector<long long>& rent = P->h_rent;
    std::vector<long long>& rbent = P->h_rbent;
    std::vector<ChunkInfo> chunks;
    std::vector<RowMeta> rmeta;
    std::vector<int2> groups;
    std::vector<int4> srows, crows;
    long long row = 0, ent = 0, bent = 0, arena = 0, slot = 0, arow = 0, grp = 0, stage = 0, uo = 0;
    int cb = 0;
    P->h_inst.resize(n);
    for (int i = 0; i < n; ++i) {
      const nrto_problem_desc& d = descs[i];
      int rpt = 0;
      build_rows(d, srows, crows, rpt);
      Inst I{};
      I.kind = d.dyn; I.nx = d.nx; I.nu = d.nu; I.T = d.T;
      I.n_sr = (int)srows.size(); I.n_cr = (int)crows.size(); I.rows_per_t = rpt;
      I.n_obs = d.n_obs; I.obs_dim = d.obs_dim; I.n_link = d.n_link; I.n_dyn = d.n_dyn_params;
      I.row0 = row; I.ent0 = ent; I.bent0 = bent; I.arena0 = arena; I.slot0 = slot; I.arow0 = arow;
      I.grp0 = grp; I.cb0 = cb;
      I.dt = d.dt; I.tau = d.tau; I.sqrt_tau = std::sqrt(d.tau);
      // State rows in chunks of whole rows for the persistent solver.  Their storage order folds the
      // time steps (t = 1, T, 2, T-1, ...) so that every chunk mixes short and long rows; the logical
      // row order (rinfo, per-row arrays, rent/rbent) stays time-major.  Every chunk starts on a
      // 4-element (16-byte) boundary of the entry and b arrays so that it can be bulk-copied.
      const int chunk = P->kl[d.dyn].chunk;
      const int nsr = (int)srows.size();
      std::vector<int> order;
      if (rpt > 0)
        for (int pidx = 0; pidx < d.T; ++pidx) {
          const int t = (pidx % 2 == 0) ? pidx / 2 + 1 : d.T - (pidx - 1) / 2;
          for (int q = 0; q < rpt; ++q) order.push_back((t - 1) * rpt + q);
        }
      if ((int)order.size() != nsr) fail(NRTO_ERR_INVALID, "internal: state rows not uniform over steps");
      rent.resize(row + nsr + crows.size());
      rbent.resize(row + nsr + crows.size());
      rmeta.resize(row + nsr + crows.size());
      for (int r = 0; r < nsr; ++r) P->h_rinfo.push_back(srows[r]);
      int nch = 0;
      long long accn = 0;
      long long n_ent_state = 0;
      for (int pos = 0; pos < nsr; ++pos) {
        const int r = order[pos];
        const int4& rr = srows[r];
        const long long len = (long long)(rr.x + 1) * d.nx;
        if (pos == 0 || accn + len > chunk) {
          if (pos > 0) {
            ChunkInfo& c = chunks.back();
            c.r1 = pos;
            c.ne = (int)(((ent - c.e0) + 3) & ~3LL);
            c.nb = (int)(((bent - c.b0) + 3) & ~3LL);
          }
          ent = (ent + 3) & ~3LL;
          bent = (bent + 3) & ~3LL;
          ChunkInfo c{};
          c.e0 = ent; c.b0 = bent; c.r0 = pos;
          chunks.push_back(c);
          ++nch;
          accn = 0;
        }
        accn += len;
        const ChunkInfo& c = chunks.back();
        RowMeta m{};
        m.off = (int)(ent - c.e0); m.boff = (int)(bent - c.b0); m.t = rr.x; m.pad = r;
        rmeta[row + pos] = m;
        rent[row + r] = ent;
        rbent[row + r] = bent;
        ent += len;
        bent += (long long)(rr.x + 1) * d.nu;
        n_ent_state += len;
      }
      if (nch > 0) {
        ChunkInfo& c = chunks.back();
        c.r1 = nsr;
        c.ne = (int)(((ent - c.e0) + 3) & ~3LL);
        c.nb = (int)(((bent - c.b0) + 3) & ~3LL);
        ent = (ent + 3) & ~3LL;
        bent = (bent + 3) & ~3LL;
      }
      I.n_chunks = nch;
      cb += nch;
      I.n_ent_state = n_ent_state;
      int ng = 0;
      for (size_t q = 0; q < crows.size(); ++q) {
        const long long R = row + I.n_sr + (long long)q;
        if (q == 0 || crows[q].x != crows[q - 1].x || crows[q].z != crows[q - 1].z) {
          groups.push_back(make_int2((int)R, 1));
          ++ng;
        } else {
          groups.back().y += 1;
        }
        P->h_rinfo.push_back(crows[q]);
        rmeta[R] = RowMeta{0, 0, -1, 0};
        rent[R] = ent;
        rbent[R] = -1;
        ent += d.nx;
      }
      I.n_groups = ng;
      if (ng > 0 && ng % d.T != 0) fail(NRTO_ERR_INVALID, "internal: control groups not uniform over steps");
      I.n_ent = ent - I.ent0;
      const Arena L = arena_layout(d.nx, d.nu, d.T, d.n_obs, d.n_link);
      const SlotL SL = slot_layout(d.nx, d.nu, d.T);
      P->stage_off.push_back(stage);
      P->stage_len.push_back(L.Psi);
      stage += L.Psi;
      P->uoff.push_back(uo);
      uo += (long long)d.T * d.nu;
      P->koff.push_back(P->k_total);
      P->k_total += (long long)d.T * d.nu * d.nx;
      arena += L.total; slot += SL.total; arow += (long long)I.n_sr * d.nx;
      row += I.n_sr + I.n_cr; grp += ng;
      P->h_inst[i] = I;
    }
    P->n_rows = row; P->n_ent = ent; P->n_bent = bent; P->arena_total = arena; P->slot_total = slot;
    P->arow_total = arow; P->n_groups_total = grp; P->n_cb_total = cb;
    P->stage_total = stage; P->u_total = uo;
    // instance order per kind: largest row count first (work-queue balance)
    for (int k = 0, o = 0; k < 3; ++k) {
      P->kl[k].order0 = o;
      std::vector<int> ids;
      for (int i = 0; i < n; ++i)
        if (P->h_inst[i].kind == k) ids.push_back(i);
      std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return P->h_inst[a].n_ent > P->h_inst[b].n_ent; });
      for (int id : ids) {
        P->h_order.push_back(id);
        P->kl[k].entries += P->h_inst[id].n_ent;
      }
      o += (int)ids.size();
    }
    const size_t rs = precision == NRTO_PREC_FP64 ? sizeof(double) : sizeof(float);
    P->d_inst = P->dalloc<Inst>(n);
    P->d_arena = P->dalloc<double>(arena);
    P->d_rinfo = P->dalloc<int4>(row);
    P->d_rent = P->dalloc<long long>(row);
    P->d_rbent = P->dalloc<long long>(row);
    P->d_chunks = P->dalloc<ChunkInfo>(cb);
    P->d_rmeta = P->dalloc<RowMeta>(row);
    P->d_groups = P->dalloc<int2>(grp);
    for (int s = 0; s < 2; ++s) {
      P->d_slot_arena[s] = P->dalloc<double>(slot);
      P->d_g0[s] = P->dalloc<double>(row);
      P->d_arow[s] = P->dalloc<double>(arow);
      P->d_bhat[s] = P->dalloc<char>(rs * (ent + 16));   // +16: bulk copies round sizes up
      P->d_bvec[s] = P->dalloc<char>(rs * (bent + 16));
    }
    P->d_lam = P->dalloc<char>(rs * (ent + 16));
    P->d_sr = P->dalloc<char>(rs * (row + 4));
    // per-row arrays that are bulk-copied are read from an even row index with an even count
    P->d_p = P->dalloc<double>(row + 4); P->d_pt = P->dalloc<double>(row); P->d_ptn = P->dalloc<double>(row);
    P->d_lamp = P->dalloc<double>(row + 4); P->d_w = P->dalloc<double>(row); P->d_lamw = P->dalloc<double>(row);
    P->d_s = P->dalloc<double>(row + 4); P->d_ell = P->dalloc<double>(row); P->d_dd = P->dalloc<double>(row);
    P->d_rnorm = P->dalloc<double>(row);
    P->d_sc = P->dalloc<double>((size_t)n * NSC);
    P->d_is = P->dalloc<int>((size_t)n * NIS);
    P->d_queue = P->dalloc<int>(8);
    P->d_phase = P->dalloc<unsigned long long>(NPHASE);
    P->d_order = P->dalloc<int>(n);
    P->d_stage = P->dalloc<double>(stage);
    P->d_stage_off = P->dalloc<long long>(n);
    P->d_stage_len = P->dalloc<long long>(n);
    P->d_uoff = P->dalloc<long long>(n);
    P->d_koff = P->dalloc<long long>(n);
    P->d_gather = P->dalloc<double>((size_t)std::max(P->u_total, P->k_total));
    P->d_ustage = P->dalloc<double>(uo);
    auto up = [&](void* dst, const void* src, size_t bytes) {
      if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, P->stream));
    };
    up(P->d_inst, P->h_inst.data(), sizeof(Inst) * n);
    up(P->d_rinfo, P->h_rinfo.data(), sizeof(int4) * row);
    up(P->d_rent, rent.data(), sizeof(long long) * row);
    up(P->d_rbent, rbent.data(), sizeof(long long) * row);
    up(P->d_chunks, chunks.data(), sizeof(ChunkInfo) * cb);
    up(P->d_rmeta, rmeta.data(), sizeof(RowMeta) * row);
    up(P->d_groups, groups.data(), sizeof(int2) * grp);
    up(P->d_order, P->h_order.data(), sizeof(int) * n);
    up(P->d_stage_off, P->stage_off.data(), sizeof(long long) * n);
    up(P->d_stage_len, P->stage_len.data(), sizeof(long long) * n);
    up(P->d_uoff, P->uoff.data(), sizeof(long long) * n);
    up(P->d_koff, P->koff.data(), sizeof(long long) * n);
    upload_params(P, descs);
    if (precision == NRTO_PREC_FP64) {
      launch_setup<double>(P);
      k_reset_outer<double><<<n, 128, 0, P->stream>>>(P->dev<double>(), 2.0);
    } else {
      launch_setup<float>(P);
      k_reset_outer<float><<<n, 128, 0, P->stream>>>(P->dev<float>(), 2.0);
    }
    P->check_launch("k_reset_outer");
    CK(cudaStreamSynchronize(P->stream));
    *out = P;
    return NRTO_OK;
  } catch (const std::exception& e) {
    delete P;
    return handle(e);
  }
}

}  // namespace

template <typename Real>
void launch_monte_carlo(nrto_problem* P, const double* dK, int n_int, int n_edge, unsigned long long seed, double tol,
                        double* d_worst, int* d_ok) {
  size_t smem = 0;
  for (const Inst& I : P->h_inst) smem = std::max(smem, sizeof(double) * (size_t)(I.T + 1) * I.nu * I.nx);
  CK(cudaFuncSetAttribute(k_monte_carlo<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_monte_carlo<Real><<<P->n, 128, smem, P->stream>>>(P->dev<Real>(), dK, P->d_koff, n_int, n_edge, seed, tol, d_worst,
                                                       d_ok);
  P->check_launch("k_monte_carlo");
}

extern "C" {

nrto_status nrto_problem_create(const nrto_problem_desc* descs, int n, int precision, void* stream,
                                nrto_problem_t* out) {
  NvtxRange nvtx_("nrto_problem_create");
  return create_problem(descs, n, precision, stream, nullptr, 0, out);
}

nrto_status nrto_problem_destroy(nrto_problem_t p) {
  if (!p) return NRTO_OK;
  cudaStreamSynchronize(p->stream);
  delete p;
  return NRTO_OK;
}

nrto_status nrto_problem_info(nrto_problem_t p, int i, nrto_instance_info* info) {
  try {
    if (!p || !info || i < 0 || i >= p->n) fail(NRTO_ERR_INVALID, "bad problem, instance or info");
    const Inst& I = p->h_inst[i];
    info->nx = I.nx; info->nu = I.nu; info->T = I.T;
    info->n_rows = I.n_sr + I.n_cr; info->n_state_rows = I.n_sr; info->n_control_rows = I.n_cr;
    info->n_entries = I.n_ent_state + (long long)I.n_cr * I.nx;   // compact (without layout padding)
    info->n_entries_state = I.n_ent_state;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_problem_update(nrto_problem_t p, const nrto_problem_desc* descs, int n) {
  try {
    if (!p || !descs || n != p->n) fail(NRTO_ERR_INVALID, "update needs the same number of instances");
    parallel_instances(n, [&](int i) {
      validate(descs[i], i);
      const Inst& I = p->h_inst[i];
      if (descs[i].dyn != I.kind || descs[i].T != I.T || descs[i].n_obs != I.n_obs || descs[i].n_link != I.n_link)
        fail(NRTO_ERR_INVALID, "instance " + std::to_string(i) + ": structure differs from create");
      long long nsr = 0, ncr = 0;
      count_rows(descs[i], nsr, ncr);
      if (nsr != I.n_sr || ncr != I.n_cr) fail(NRTO_ERR_INVALID, "row structure differs from create");
      if (descs[i].tau != I.tau || descs[i].dt != I.dt) fail(NRTO_ERR_INVALID, "dt/tau differ from create");
    });
    upload_params(p, descs);
    if (p->prec == NRTO_PREC_FP64) launch_setup<double>(p); else launch_setup<float>(p);
    p->linearized = false;
    p->carry_ok = false;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_linearize(nrto_problem_t p, const double* u_hat) {
  try {
    NvtxRange nvtx_("nrto_linearize");
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    if (u_hat) {
      if (!finite_arr(u_hat, p->u_total)) fail(NRTO_ERR_NUMERIC, "u_hat not finite");
      std::vector<int> is(p->n * NIS);
      CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
      CK(cudaStreamSynchronize(p->stream));
      for (int i = 0; i < p->n; ++i) {
        const Inst& I = p->h_inst[i];
        const SlotL SL = slot_layout(I.nx, I.nu, I.T);
        CK(cudaMemcpyAsync(p->d_slot_arena[is[i * NIS + IS_SLOT]] + I.slot0 + SL.u_hat, u_hat + p->uoff[i],
                           sizeof(double) * I.T * I.nu, cudaMemcpyHostToDevice, p->stream));
      }
      CK(cudaStreamSynchronize(p->stream));
      p->carry_ok = false;   // a new nominal from the caller: the next inner solve starts cold
    }
    if (p->prec == NRTO_PREC_FP64) launch_linearize<double>(p, -1); else launch_linearize<float>(p, -1);
    p->linearized = true;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_set_trust_radius(nrto_problem_t p, const double* r) {
  try {
    if (!p || !r) fail(NRTO_ERR_INVALID, "null argument");
    std::vector<double> sc(p->n * NSC);
    CK(cudaMemcpyAsync(sc.data(), p->d_sc, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < p->n; ++i) {
      if (!(r[i] > 0) || !std::isfinite(r[i])) fail(NRTO_ERR_INVALID, "trust radius must be positive");
      sc[i * NSC + SC_RTRUST] = r[i];
    }
    CK(cudaMemcpyAsync(p->d_sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_solve_socp(nrto_problem_t p, const nrto_solver_opts* o, nrto_socp_out* out) {
  try {
    NvtxRange nvtx_("nrto_solve_socp");
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    check_opts(o);
    if (!p->linearized) fail(NRTO_ERR_STATE, "nrto_linearize must be called before nrto_solve_socp");
    if (p->prec == NRTO_PREC_FP64) launch_solve<double>(p, *o); else launch_solve<float>(p, *o);
    if (out) return finish_statuses(p, o, out);
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_outer_step(nrto_problem_t p, const nrto_solver_opts* o, int* accepted) {
  try {
    NvtxRange nvtx_("nrto_outer_step");
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    check_opts(o);
    if (!p->linearized) fail(NRTO_ERR_STATE, "nrto_linearize must be called before nrto_outer_step");
    if (p->prec == NRTO_PREC_FP64) launch_outer_step<double>(p, *o); else launch_outer_step<float>(p, *o);
    if (accepted) {
      std::vector<int> is(p->n * NIS);
      CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
      CK(cudaStreamSynchronize(p->stream));
      for (int i = 0; i < p->n; ++i) accepted[i] = is[i * NIS + IS_ACCEPT];
    }
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_solve(nrto_problem_t p, const nrto_solver_opts* o, int n_outer, double* u_bar, double* K,
                       double* merit) {
  try {
    NvtxRange nvtx_("nrto_solve");
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    check_opts(o);
    if (n_outer < 0) fail(NRTO_ERR_INVALID, "n_outer < 0");
    const bool f64 = p->prec == NRTO_PREC_FP64;
    auto enqueue = [&]() {
      if (f64) k_reset_outer<double><<<p->n, 128, 0, p->stream>>>(p->dev<double>(), o->r0);
      else k_reset_outer<float><<<p->n, 128, 0, p->stream>>>(p->dev<float>(), o->r0);
      p->check_launch("k_reset_outer");
      p->carry_ok = false;
      k_scatter_uhat<<<p->n, 128, 0, p->stream>>>(p->d_slot_arena[0], p->d_inst, p->d_ustage, p->d_uoff, p->n);
      p->check_launch("k_scatter_uhat");
      if (f64) { launch_linearize<double>(p, -1); launch_merit_current<double>(p, o->w_p); }
      else { launch_linearize<float>(p, -1); launch_merit_current<float>(p, o->w_p); }
      nrto_solver_opts last = *o;
      if (o->max_inner_final > 0) last.max_inner = o->max_inner_final;
      for (int it = 0; it < n_outer; ++it) {
        const nrto_solver_opts& oi = (it == n_outer - 1) ? last : *o;
        if (f64) launch_outer_step<double>(p, oi); else launch_outer_step<float>(p, oi);
      }
    };
    // the legacy and per-thread default streams cannot be captured: those callers launch directly
    const bool capturable = p->stream != nullptr && p->stream != cudaStreamLegacy && p->stream != cudaStreamPerThread;
    if (p->graph_enabled && capturable && !p->profiling && !p->carve_base) {
      // key: the options, the outer-step count and whether a learned warm start is pending
      std::vector<unsigned char> key(sizeof(nrto_solver_opts) + sizeof(int) + 2);
      std::memcpy(key.data(), o, sizeof(nrto_solver_opts));
      std::memcpy(key.data() + sizeof(nrto_solver_opts), &n_outer, sizeof(int));
      key[key.size() - 2] = (unsigned char)p->mapping;
      key.back() = p->warm_pending ? 1 : 0;
      if (!p->graph_exec || key != p->graph_key) {
        if (p->graph_exec) { cudaGraphExecDestroy(p->graph_exec); p->graph_exec = nullptr; }
        const long long l0 = p->launches;
        const bool warm0 = p->warm_pending;
        CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeRelaxed));
        cudaGraph_t g = nullptr;
        try {
          enqueue();
        } catch (...) {
          cudaStreamEndCapture(p->stream, &g);
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          p->launches = l0;
          p->warm_pending = warm0;
          throw;
        }
        CK(cudaStreamEndCapture(p->stream, &g));
        const cudaError_t ie = cudaGraphInstantiate(&p->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) { p->graph_exec = nullptr; fail(NRTO_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie)); }
        p->graph_launches = p->launches - l0;
        p->launches = l0;
        p->graph_key = key;
        p->graph_carry_after = p->carry_ok;
        ++p->graph_captures;
      }
      CK(cudaGraphLaunch(p->graph_exec, p->stream));
      p->launches += p->graph_launches;
      ++p->graph_replays;
      p->carry_ok = p->graph_carry_after;
      p->warm_pending = false;
    } else {
      enqueue();
    }
    p->linearized = true;
    if (u_bar) copy_arena_field(p, GF_UHAT, u_bar);
    if (K) copy_arena_field(p, GF_KACC, K);
    if (merit) {
      std::vector<double> sc(p->n * NSC);
      CK(cudaMemcpyAsync(sc.data(), p->d_sc, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
      CK(cudaStreamSynchronize(p->stream));
      for (int i = 0; i < p->n; ++i) merit[i] = sc[i * NSC + SC_PHI];
    }
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_set_warm_start(nrto_problem_t p, const double* K, const double* ptilde, const double* lambda_p) {
  try {
    if (!p || !K || !ptilde || !lambda_p) fail(NRTO_ERR_INVALID, "null argument");
    long long o = 0;
    for (int i = 0; i < p->n; ++i) {
      const Inst& I = p->h_inst[i];
      const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
      const long long cnt = (long long)I.T * I.nu * I.nx;
      if (!finite_arr(K + o, cnt)) fail(NRTO_ERR_NUMERIC, "warm-start K not finite");
      CK(cudaMemcpyAsync(p->d_arena + I.arena0 + L.K1, K + o, sizeof(double) * cnt, cudaMemcpyHostToDevice, p->stream));
      o += cnt;
    }
    if (!finite_arr(ptilde, p->n_rows) || !finite_arr(lambda_p, p->n_rows)) fail(NRTO_ERR_NUMERIC, "warm start not finite");
    CK(cudaMemcpyAsync(p->d_pt, ptilde, sizeof(double) * p->n_rows, cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_lamp, lambda_p, sizeof(double) * p->n_rows, cudaMemcpyHostToDevice, p->stream));
    // a plain warm start replaces a lifted one that was not used
    std::vector<int> is(p->n * NIS);
    CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < p->n; ++i) is[i * NIS + IS_WLIFT] = 0;
    CK(cudaMemcpyAsync(p->d_is, is.data(), sizeof(int) * is.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->warm_pending = true;
    p->wlift_pending = false;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

static nrto_status warm_from_network(nrto_problem_t p, nrto_mlp_t m, const float* features, const int* row_map,
                                     WarmOffsets o) {
  try {
    if (!p || !m || !features || !row_map) fail(NRTO_ERR_INVALID, "null argument");
    for (long long r = 0; r < p->n_rows; ++r)
      if (row_map[r] < -1) fail(NRTO_ERR_INVALID, "row_map entries must be >= -1");
    int out_dim = 0;
    cudaStream_t ms = nullptr;
    const float* Y = nrto_mlp_internal_forward_device(m, features, p->n, &out_dim, &ms);
    if (!Y) return NRTO_ERR_INVALID;
    long long kmax = 0, umax = 0, xmax = 0;
    for (int i = 0; i < p->n; ++i) {
      const Inst& I = p->h_inst[i];
      kmax = std::max(kmax, (long long)I.T * I.nu * I.nx);
      umax = std::max(umax, (long long)I.T * I.nu);
      xmax = std::max(xmax, (long long)I.T * I.nx);
    }
    int mmax = -1;
    for (long long r = 0; r < p->n_rows; ++r) mmax = std::max(mmax, row_map[r]);
    auto fits = [&](int off, long long n) { return off >= 0 && off + n <= out_dim; };
    if (!fits(o.k, kmax) || !fits(o.pt, mmax + 1) || !fits(o.lp, mmax + 1))
      fail(NRTO_ERR_INVALID, "offsets and row map do not fit the network output");
    if ((o.th >= 0 && !fits(o.th, mmax + 1)) || (o.lw >= 0 && !fits(o.lw, mmax + 1)) || (o.du >= 0 && !fits(o.du, umax)) ||
        (o.le >= 0 && !fits(o.le, xmax)) || (o.rho >= 0 && !fits(o.rho, 1)))
      fail(NRTO_ERR_INVALID, "lifted offsets do not fit the network output");
    if (!p->d_wsmap) p->d_wsmap = p->dalloc<int>(p->n_rows);
    CK(cudaMemcpyAsync(p->d_wsmap, row_map, sizeof(int) * p->n_rows, cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(ms));   // network output ready
    if (p->prec == NRTO_PREC_FP64)
      k_scatter_warm<double><<<p->n, 256, 0, p->stream>>>(p->dev<double>(), Y, out_dim, p->d_wsmap, o);
    else
      k_scatter_warm<float><<<p->n, 256, 0, p->stream>>>(p->dev<float>(), Y, out_dim, p->d_wsmap, o);
    p->check_launch("k_scatter_warm");
    CK(cudaStreamSynchronize(p->stream));   // the network's output buffer may be reused after return
    p->warm_pending = true;
    p->wlift_pending = o.lifted();
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_set_warm_start_from_network(nrto_problem_t p, nrto_mlp_t m, const float* features,
                                            const int* row_map, int k_off, int pt_off, int lp_off) {
  return warm_from_network(p, m, features, row_map, WarmOffsets{k_off, pt_off, lp_off, -1, -1, -1, -1, -1});
}

nrto_status nrto_set_warm_start_from_network_lifted(nrto_problem_t p, nrto_mlp_t m, const float* features,
                                                    const int* row_map, const int* offsets) {
  if (!offsets) {
    g_last_error = "null offsets";
    return NRTO_ERR_INVALID;
  }
  return warm_from_network(p, m, features, row_map,
                           WarmOffsets{offsets[0], offsets[1], offsets[2], offsets[3], offsets[4], offsets[5], offsets[6],
                                       offsets[7]});
}

nrto_status nrto_set_warm_start_lifted(nrto_problem_t p, const double* theta, const double* lambda_w, const double* du,
                                       const double* lambda_e, const double* rho) {
  try {
    if (!p || !theta || !lambda_w || !du || !lambda_e) fail(NRTO_ERR_INVALID, "null argument");
    if (!p->warm_pending) fail(NRTO_ERR_STATE, "nrto_set_warm_start must come first");
    if (!finite_arr(theta, p->n_rows) || !finite_arr(lambda_w, p->n_rows) || !finite_arr(du, p->u_total))
      fail(NRTO_ERR_NUMERIC, "lifted warm start not finite");
    long long xtot = 0;
    for (const Inst& I : p->h_inst) xtot += (long long)I.T * I.nx;
    if (!finite_arr(lambda_e, xtot)) fail(NRTO_ERR_NUMERIC, "lifted warm start not finite");
    if (rho)
      for (int i = 0; i < p->n; ++i)
        if (!(rho[i] > 0) || !std::isfinite(rho[i])) fail(NRTO_ERR_INVALID, "warm-start penalties must be positive");
    std::vector<double> th(theta, theta + p->n_rows);
    for (double& v : th) v = std::max(v, 0.0);
    std::vector<int> is(p->n * NIS);
    std::vector<double> sc(p->n * NSC);
    CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(sc.data(), p->d_sc, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpyAsync(p->d_dd, th.data(), sizeof(double) * p->n_rows, cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_lamw, lambda_w, sizeof(double) * p->n_rows, cudaMemcpyHostToDevice, p->stream));
    long long xo = 0;
    for (int i = 0; i < p->n; ++i) {
      const Inst& I = p->h_inst[i];
      const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
      double* ar = p->d_arena + I.arena0;
      CK(cudaMemcpyAsync(ar + L.du, du + p->uoff[i], sizeof(double) * I.T * I.nu, cudaMemcpyHostToDevice, p->stream));
      CK(cudaMemcpyAsync(ar + L.lam_e + I.nx, lambda_e + xo, sizeof(double) * I.T * I.nx, cudaMemcpyHostToDevice,
                         p->stream));
      xo += (long long)I.T * I.nx;
      is[i * NIS + IS_WLIFT] = 1;
      sc[(size_t)i * NSC + SC_RHOW] = rho ? rho[i] : 0.0;
    }
    CK(cudaMemcpyAsync(p->d_is, is.data(), sizeof(int) * is.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(p->d_sc, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->wlift_pending = true;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_monte_carlo(nrto_problem_t p, const double* K, int n_interior, int n_edge, unsigned long long seed,
                             double tol, int* n_ok, double* worst) {
  NvtxRange nvtx_("nrto_monte_carlo");
  double* dK = nullptr;
  double* dw = nullptr;
  int* dok = nullptr;
  auto release = [&]() {
    if (dK) cudaFree(dK);
    if (dw) cudaFree(dw);
    if (dok) cudaFree(dok);
  };
  try {
    if (!p || !n_ok) fail(NRTO_ERR_INVALID, "null argument");
    if (n_interior < 0 || n_edge < 0 || (long long)n_interior + n_edge > (1 << 24))
      fail(NRTO_ERR_INVALID, "sample counts out of range");
    if (std::isnan(tol)) fail(NRTO_ERR_INVALID, "tol is NaN");
    if (!p->linearized) fail(NRTO_ERR_STATE, "nrto_linearize or nrto_solve must come before nrto_monte_carlo");
    if (K && !finite_arr(K, p->k_total)) fail(NRTO_ERR_NUMERIC, "K not finite");
    const long long ns = (long long)n_interior + n_edge;
    size_t smem = 0;
    for (const Inst& I : p->h_inst) smem = std::max(smem, sizeof(double) * (size_t)(I.T + 1) * I.nu * I.nx);
    if (smem > 227 * 1024) fail(NRTO_ERR_INVALID, "horizon too long for the Monte Carlo kernel's gain table");
    CK(cudaStreamSynchronize(p->stream));
    if (K) {
      CK(cudaMalloc(&dK, sizeof(double) * std::max<long long>(p->k_total, 1)));
      CK(cudaMemcpyAsync(dK, K, sizeof(double) * p->k_total, cudaMemcpyHostToDevice, p->stream));
    }
    if (worst && ns > 0) CK(cudaMalloc(&dw, sizeof(double) * (size_t)p->n * ns));
    CK(cudaMalloc(&dok, sizeof(int) * std::max(p->n, 1)));
    if (p->prec == NRTO_PREC_FP64) launch_monte_carlo<double>(p, dK, n_interior, n_edge, seed, tol, dw, dok);
    else launch_monte_carlo<float>(p, dK, n_interior, n_edge, seed, tol, dw, dok);
    CK(cudaMemcpyAsync(n_ok, dok, sizeof(int) * p->n, cudaMemcpyDeviceToHost, p->stream));
    if (dw) CK(cudaMemcpyAsync(worst, dw, sizeof(double) * (size_t)p->n * ns, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    release();
    return NRTO_OK;
  } catch (const std::exception& e) {
    if (p) cudaStreamSynchronize(p->stream);
    release();
    return handle(e);
  }
}

nrto_status nrto_get_stats(nrto_problem_t p, double* out, int width) {
  try {
    if (!p || !out) fail(NRTO_ERR_INVALID, "null argument");
    if (width < NRTO_NSTAT) fail(NRTO_ERR_INVALID, "width must be >= NRTO_NSTAT");
    std::vector<int> is(p->n * NIS);
    std::vector<double> sc(p->n * NSC);
    CK(cudaMemcpyAsync(is.data(), p->d_is, sizeof(int) * is.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaMemcpyAsync(sc.data(), p->d_sc, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    for (int i = 0; i < p->n; ++i) {
      const int* a = is.data() + (size_t)i * NIS;
      const double* c = sc.data() + (size_t)i * NSC;
      double* o = out + (size_t)i * width;
      o[0] = a[IS_CUMITERS]; o[1] = a[IS_ITERS]; o[2] = a[IS_STATUS]; o[3] = a[IS_NACC];
      o[4] = c[SC_RHO]; o[5] = a[IS_DRITERS]; o[6] = a[IS_FALLBACK]; o[7] = a[IS_ACCST];
      o[8] = c[SC_PHI]; o[9] = c[SC_COST_ACC]; o[10] = c[SC_VIOL]; o[11] = c[SC_RTRUST];
      o[12] = c[SC_RP]; o[13] = c[SC_RD]; o[14] = a[IS_PCG];
      for (int k = NRTO_NSTAT; k < width; ++k) o[k] = 0.0;
    }
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_export(nrto_problem_t p, int field, int i, double* dst, long long count) {
  return exchange(p, field, i, dst, count, true);
}

nrto_status nrto_import(nrto_problem_t p, int field, int i, const double* src, long long count) {
  return exchange(p, field, i, const_cast<double*>(src), count, false);
}

nrto_status nrto_set_graph(nrto_problem_t p, int enable) {
  try {
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    p->graph_enabled = enable != 0;
    if (!p->graph_enabled && p->graph_exec) {
      CK(cudaStreamSynchronize(p->stream));
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_set_launch_mapping(nrto_problem_t p, int mapping) {
  try {
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    if (mapping < 0 || mapping >= NRTO_NMAPPING) fail(NRTO_ERR_INVALID, "unknown launch mapping");
    p->mapping = mapping;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_autotune(nrto_problem_t p, const nrto_solver_opts* o, int n_outer, int reps, double* ms_out,
                          int* chosen) {
  try {
    NvtxRange nvtx_("nrto_autotune");
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    check_opts(o);
    if (n_outer < 1 || reps < 1) fail(NRTO_ERR_INVALID, "n_outer and reps must be >= 1");
    const bool prof = p->profiling;
    if (prof) fail(NRTO_ERR_STATE, "disable solver profiling before nrto_autotune");
    double best = 0.0;
    int best_m = p->mapping;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int m = 0; m < NRTO_NMAPPING; ++m) {
      p->mapping = m;
      nrto_status st = nrto_solve(p, o, n_outer, nullptr, nullptr, nullptr);   // warm-up (and capture)
      if (st != NRTO_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
      CK(cudaEventRecord(e0, p->stream));
      for (int r = 0; r < reps; ++r) {
        st = nrto_solve(p, o, n_outer, nullptr, nullptr, nullptr);
        if (st != NRTO_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
      }
      CK(cudaEventRecord(e1, p->stream));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      const double ms = t / reps;
      if (ms_out) ms_out[m] = ms;
      if (m == 0 || ms < best) { best = ms; best_m = m; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->mapping = best_m;
    if (chosen) *chosen = best_m;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_graph_info(nrto_problem_t p, long long* captures, long long* replays) {
  if (!p) { g_last_error = "null problem"; return NRTO_ERR_INVALID; }
  if (captures) *captures = p->graph_captures;
  if (replays) *replays = p->graph_replays;
  return NRTO_OK;
}

nrto_status nrto_profile(nrto_problem_t p, int enable, double* solver_ms, long long* solver_launches) {
  try {
    if (!p) fail(NRTO_ERR_INVALID, "null problem");
    double ms = 0.0;
    if (!p->prof_events.empty()) {
      CK(cudaStreamSynchronize(p->stream));
      for (auto& ev : p->prof_events) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ev.first, ev.second));
        ms += t;
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
      }
    }
    if (solver_ms) *solver_ms = ms;
    if (solver_launches) *solver_launches = p->prof_launches;
    p->prof_events.clear();
    p->prof_launches = 0;
    p->profiling = enable != 0;
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

nrto_status nrto_phase_cycles(nrto_problem_t p, long long* cycles, int n) {
  try {
    if (!p || !cycles || n < NPHASE) fail(NRTO_ERR_INVALID, "need a buffer of NRTO_NPHASE counters");
    unsigned long long h[NPHASE];
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpy(h, p->d_phase, sizeof(h), cudaMemcpyDeviceToHost));
    CK(cudaMemset(p->d_phase, 0, sizeof(h)));
    for (int k = 0; k < NPHASE; ++k) cycles[k] = (long long)h[k];
    return NRTO_OK;
  } catch (const std::exception& e) {
    return handle(e);
  }
}

long long nrto_kernel_launches(nrto_problem_t p) { return p ? p->launches : -1; }

nrto_status nrto_selftest_bounded_wait(void* stream, int* status_out, long long* cycles_out) {
  long long* d = nullptr;
  try {
    if (!status_out) fail(NRTO_ERR_INVALID, "status_out is required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMalloc(&d, 2 * sizeof(long long)));
    k_selftest_wait<<<1, 32, 0, s>>>(d);
    CK(cudaGetLastError());
    long long h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaFree(d));
    d = nullptr;
    *status_out = (int)h[0];
    if (cycles_out) *cycles_out = h[1];
    return NRTO_OK;
  } catch (const std::exception& e) {
    if (d) cudaFree(d);
    return handle(e);
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// nrto_solve_noalloc: the whole-batch solve of nrto_solve with every device buffer of the batch
// (row tables, linearization slots, solver arena with its gain-solve scratch, work queue) cut from
// one static device area instead of cudaMalloc.  For callers that must not allocate device memory
// after start-up: real-time control loops that cannot afford an allocation's latency or its
// implicit synchronization, and processes whose device memory is already reserved by another
// allocator (a framework's caching pool), where a cudaMalloc could fail mid-run.
namespace {

constexpr size_t NOALLOC_AREA_BYTES = size_t(32) << 20;   // 32 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_noalloc_area[NOALLOC_AREA_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;                                  // serializes the calls of this process
char* g_noalloc_dev_ptr[NOALLOC_MAX_DEVICES] = {};          // device address of the area, per device

}  // namespace

extern "C" nrto_status nrto_solve_noalloc(const nrto_problem_desc* descs, int n, int precision,
                                          const nrto_solver_opts* opts, int n_outer, void* stream,
                                          double* u_bar, double* K, double* merit) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  nrto_problem_t p = nullptr;
  try {
    g_last_error.clear();
    check_opts(opts);
    if (n_outer < 0) fail(NRTO_ERR_INVALID, "n_outer < 0");
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) fail(NRTO_ERR_INVALID, "device index out of range");
    if (!g_noalloc_dev_ptr[dev]) {
      // First call on this device: look up the device address of the static area (the host-side
      // symbol is only a stand-in and must never reach a kernel).
      void* ptr = nullptr;
      CK(cudaGetSymbolAddress(&ptr, g_noalloc_area));
      g_noalloc_dev_ptr[dev] = static_cast<char*>(ptr);
    }
    const nrto_status cs = create_problem(descs, n, precision, stream, g_noalloc_dev_ptr[dev],
                                          NOALLOC_AREA_BYTES, &p);
    if (cs != NRTO_OK) {
      // create may have queued clears of the area before it gave up; let them finish before the
      // next call reuses the area.
      cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
      return cs;
    }
    const nrto_status st = nrto_solve(p, opts, n_outer, u_bar, K, merit);
    const std::string msg = g_last_error;
    nrto_problem_destroy(p);   // synchronizes the stream: the area is free again when this returns
    g_last_error = msg;
    return st;
  } catch (const std::exception& e) {
    if (p) nrto_problem_destroy(p);
    return handle(e);
  }
}

// NRTO-DR: gain-solve factors for (Q_v + r_χ I + σ Σ Â_jᵀÂ_j), then one persistent launch per kind.
template <typename Real>
void launch_dr(nrto_problem* P, const nrto_solver_opts& o, SolveParams sp) {
  Dev<Real> D = P->dev<Real>();
  k_gain_factors<Real><<<P->n, 128, 0, P->stream>>>(D, o.sigma, o.r_chi, 0);
  P->check_launch("k_gain_factors");
  CK(cudaMemsetAsync(P->d_queue, 0, 4 * sizeof(int), P->stream));
  launch_solver_kinds<Real>(P, SOLVER_KERNEL_DR, sp);
}
