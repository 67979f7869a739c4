// Monte Carlo check of robust-constraint satisfaction (Sec. V, Methodology): per instance, rollouts
// of the nonlinear dynamics under disturbances drawn uniformly from the interior of the uncertainty
// set and on its boundary along convex combinations of the worst-case directions of the linearized
// robust constraints, each checked against every constraint of Problem 1.
//
// Sampling (whitened coordinates w ∈ R^{(T+1) n_x}, ‖w‖ ≤ 1, ζ_i = √τ Ψ_iᵀ w_i with Ψ_iᵀΨ_i = Σ_i):
//   interior sample: w = ρ g/‖g‖, g standard normal (Box–Muller over consecutive draw pairs),
//     ρ = U^{1/n}, n = (T+1) n_x, U the draw after the normals' draws;
//   edge sample e: n_c = 1 + (e mod 3) rows j_c = ⌊U_c · n_rows⌋ (state rows then control rows,
//     draws 0..n_c-1), weights a_c = 1 - U (draws n_c..2n_c-1), w = v/‖v‖ with
//     v = Σ_c a_c y_{j_c}/‖y_{j_c}‖ and y_j = Â_j k + b̂_j the row's SOC vector.
// Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the output function and increment
// of Vigna's splitmix64.c) used as a counter-based generator: the stream of (instance i, sample s)
// starts at key = mix(seed XOR mix(i·2³² + s)) and its n-th draw is mix(key + (n+1)·γ).
// Rollout: x_0 = x̄_0 + ζ_0, u_k = ū_k + K_k ζ_k, x_{k+1} = f(x_k, u_k) + ζ_{k+1}; the sample's worst
// value is the largest g_j(x_t) (state rows, t = 1..T) and control-bound value (k = 0..T-1).
// FP64 throughout.  One CTA per instance, threads over samples.
#pragma once
#include "dynamics.cuh"

namespace nrto {

__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr unsigned long long SM64_GAMMA = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ double sm64_uniform(unsigned long long key, long long n) {
  return (double)(sm64_mix(key + (unsigned long long)(n + 1) * SM64_GAMMA) >> 11) * 0x1.0p-53;
}

// Standard normals of one stream, read in increasing index order (each Box–Muller pair computed once).
struct NormalStream {
  unsigned long long key;
  long long pair = -1;
  double g0 = 0.0, g1 = 0.0;
  __device__ double get(long long k) {
    const long long p = k >> 1;
    if (p != pair) {
      pair = p;
      const double u0 = sm64_uniform(key, 2 * p), u1 = sm64_uniform(key, 2 * p + 1);
      const double r = sqrt(-2.0 * log(1.0 - u0));
      const double a = 2.0 * 3.141592653589793 * u1;
      g0 = r * cos(a);
      g1 = r * sin(a);
    }
    return (k & 1) ? g1 : g0;
  }
};

// Block m of y_j = Â_j k + b̂_j for logical row r of the instance (state rows first), from the
// gain table Gt_m[u][c] = √τ (K_m Ψ_mᵀ)[u][c] in shared memory.
template <typename Real>
__device__ inline void mc_row_block(const Dev<Real>& D, const Inst& I, const LinSlot<Real>& S, const double* gt, int r,
                                    int m, double* y) {
  const int nx = I.nx, nu = I.nu;
  for (int c = 0; c < nx; ++c) y[c] = 0.0;
  const long long R = I.row0 + r;
  const int4 ri = D.rinfo[R];
  if (r < I.n_sr) {
    if (m > ri.x) return;
    const long long e = D.rent[R] + (long long)m * nx;
    const long long be = D.rbent[R] + (long long)m * nu;
    for (int c = 0; c < nx; ++c) {
      double acc = (double)S.bhat[e + c];
      for (int u = 0; u < nu; ++u) acc += gt[(m * nu + u) * nx + c] * (double)S.bvec[be + u];
      y[c] = acc;
    }
  } else {
    if (m != ri.x) return;
    const double sg = ri.y == ROW_UHI ? 1.0 : -1.0;
    for (int c = 0; c < nx; ++c) y[c] = sg * gt[(m * nu + ri.z) * nx + c];
  }
}

constexpr int MC_MAX_NC = 3;

template <typename Real>
__global__ void k_monte_carlo(Dev<Real> D, const double* Kext, const long long* koff, int n_int, int n_edge,
                              unsigned long long seed, double tol, double* worst_out, int* ok_out) {
  extern __shared__ __align__(16) double mc_gt[];
  __shared__ int s_ok[32];
  const int i = blockIdx.x;
  const Inst I = D.inst[i];
  const Arena L = arena_layout(I.nx, I.nu, I.T, I.n_obs, I.n_link);
  const SlotL SL = slot_layout(I.nx, I.nu, I.T);
  const double* ar = D.arena + I.arena0;
  const int slot = D.is[i * NIS + IS_SLOT];
  const LinSlot<Real> S = D.slot[slot];
  const double* sa = S.arena + I.slot0;
  const int T = I.T, nx = I.nx, nu = I.nu;
  const double* K = Kext ? Kext + koff[i] : ar + L.Kacc;
  // Gt_m[u][c] = √τ Σ_q K_m[u][q] Ψ_m[c][q] (block T: no control)
  for (int q = threadIdx.x; q < (T + 1) * nu * nx; q += blockDim.x) {
    const int m = q / (nu * nx), u = (q / nx) % nu, c = q % nx;
    double acc = 0.0;
    if (m < T)
      for (int k = 0; k < nx; ++k) acc += K[(long long)m * nu * nx + u * nx + k] * ar[L.Psi + (long long)m * nx * nx + c * nx + k];
    mc_gt[q] = I.sqrt_tau * acc;
  }
  __syncthreads();
  const int ns = n_int + n_edge, n_rows = I.n_sr + I.n_cr;
  const long long n = (long long)(T + 1) * nx;
  int ok = 0;
  for (int s = threadIdx.x; s < ns; s += blockDim.x) {
    const unsigned long long key =
        sm64_mix(seed ^ sm64_mix(((unsigned long long)i << 32) + (unsigned long long)s));
    const bool interior = s < n_int;
    double scale = 0.0;
    int nc = 0, rows[MC_MAX_NC];
    double cf[MC_MAX_NC];
    double y[14], v[14];
    if (interior) {
      NormalStream g{key};
      double s2 = 0.0;
      for (long long k = 0; k < n; ++k) { const double z = g.get(k); s2 += z * z; }
      const double rad = pow(sm64_uniform(key, 2 * ((n + 1) / 2)), 1.0 / (double)n);
      scale = rad / sqrt(s2);
    } else {
      const int e = s - n_int;
      nc = n_rows > 0 ? 1 + e % 3 : 0;
      for (int c = 0; c < nc; ++c) {
        int j = (int)(sm64_uniform(key, c) * (double)n_rows);
        rows[c] = j < n_rows - 1 ? j : n_rows - 1;
      }
      for (int c = 0; c < nc; ++c) {
        double nr2 = 0.0;
        for (int m = 0; m <= T; ++m) {
          mc_row_block<Real>(D, I, S, mc_gt, rows[c], m, y);
          for (int q = 0; q < nx; ++q) nr2 += y[q] * y[q];
        }
        const double a = 1.0 - sm64_uniform(key, nc + c);
        cf[c] = nr2 > 0.0 ? a / sqrt(nr2) : 0.0;
      }
      double s2 = 0.0;
      for (int m = 0; m <= T; ++m) {
        for (int q = 0; q < nx; ++q) v[q] = 0.0;
        for (int c = 0; c < nc; ++c) {
          if (cf[c] == 0.0) continue;
          mc_row_block<Real>(D, I, S, mc_gt, rows[c], m, y);
          for (int q = 0; q < nx; ++q) v[q] += cf[c] * y[q];
        }
        for (int q = 0; q < nx; ++q) s2 += v[q] * v[q];
      }
      scale = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    }
    // ζ_m = √τ · scale · Ψ_mᵀ w̃_m, with w̃_m the block's normals or v
    NormalStream g{key};
    auto zeta = [&](int m, double* z) {
      double wt[14];
      if (interior) {
        for (int q = 0; q < nx; ++q) wt[q] = g.get((long long)m * nx + q);
      } else {
        for (int q = 0; q < nx; ++q) wt[q] = 0.0;
        for (int c = 0; c < nc; ++c) {
          if (cf[c] == 0.0) continue;
          mc_row_block<Real>(D, I, S, mc_gt, rows[c], m, y);
          for (int q = 0; q < nx; ++q) wt[q] += cf[c] * y[q];
        }
      }
      const double* Ps = ar + L.Psi + (long long)m * nx * nx;
      for (int b = 0; b < nx; ++b) {
        double acc = 0.0;
        for (int a = 0; a < nx; ++a) acc += Ps[a * nx + b] * wt[a];
        z[b] = I.sqrt_tau * scale * acc;
      }
    };
    double x[14], xn[14], zk[14], u[7], grad[14];
    zeta(0, zk);
    for (int c = 0; c < nx; ++c) x[c] = ar[L.x0 + c] + zk[c];
    double worst = -INFINITY;
    const double* ub = sa + SL.u_hat;
    for (int k = 0; k < T; ++k) {
      for (int a = 0; a < nu; ++a) {
        double acc = ub[(long long)k * nu + a];
        for (int c = 0; c < nx; ++c) acc += K[(long long)k * nu * nx + a * nx + c] * zk[c];
        u[a] = acc;
      }
      dyn_step(I.kind, ar + L.dyn, I.dt, x, u, xn, nullptr, nullptr, ar + L.xlo, ar + L.xhi);
      zeta(k + 1, zk);
      for (int c = 0; c < nx; ++c) x[c] = xn[c] + zk[c];
      // state rows of t = k + 1, then the control rows of step k (the rows of Problem 1)
      for (int q = 0; q < I.rows_per_t; ++q) {
        const int4 ri = D.rinfo[I.row0 + (long long)k * I.rows_per_t + q];
        worst = fmax(worst, row_g_grad(I, ar, L, ri, x, grad));
      }
      for (int a = 0; a < nu; ++a) {
        const double hi = ar[L.uhi + a], lo = ar[L.ulo + a];
        if (isfinite(hi)) worst = fmax(worst, u[a] - hi);
        if (isfinite(lo)) worst = fmax(worst, lo - u[a]);
      }
    }
    if (worst_out) worst_out[(long long)i * ns + s] = worst;
    ok += (worst <= tol) ? 1 : 0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  ok = warp_sum(ok);
  if (lane == 0) s_ok[wid] = ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_ok[w];
    ok_out[i] = t;
  }
}

}  // namespace nrto
