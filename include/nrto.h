/*
 * libnrto — the data-parallel inner loop of Nonlinear Robust Trajectory Optimization (NRTO) on
 * NVIDIA B300 (sm_103a): NRTO-FullADMM and NRTO-DR iterations for batches of robust trajectory
 * problems, with the successive-linearization outer step around them.
 *
 * Method: arXiv 2603.02642 ("cuNRTO").  Problem 1 (Sec. II-A) is the robust trajectory problem;
 * Problem 2 (Sec. II-B) its linearization with second-order-cone rows ‖Â_j k_v + b̂_j‖ ≤ p_j
 * (Supplementary Sec. I); the inner solvers are NRTO-DR (Sec. III, Supplementary Sec. II) and
 * NRTO-FullADMM (Sec. IV, Algorithm 1, Supplementary Sec. III).
 *
 * Conventions
 *  - All pointers passed to the functions below are HOST pointers unless stated otherwise.
 *    Input arrays are read during the call and not retained; the caller keeps ownership.
 *  - Arrays are row-major float64.  Per-instance arrays of a batch are concatenated in instance order.
 *  - Gains: K_k is nu×nx, stored row-major per step (k = 0..T-1); the paper's k_v is the
 *    column-wise vec of the K_k, stacked.
 *  - Row order of the robust constraints (index j): state rows for t = 1..T — for each t the sphere
 *    clearance rows (unicycle/quadcopter: obstacle o; arm: link sphere l major, static sphere o minor),
 *    then state-bound rows (state i ascending, upper before lower, finite bounds only); then control
 *    rows for k = 0..T-1 (input i ascending, upper before lower, finite bounds only).
 *  - Ragged row layout (λ_ν, b̂_j): a state row at time t has (t+1)·nx entries (ζ-blocks 0..t); a
 *    control row at step k has nx entries (ζ-block k).
 *  - Every call is asynchronous on the problem's stream unless it copies results to host memory, in
 *    which case it synchronizes that stream.  Functions return a status; C++ exceptions never cross
 *    the ABI; nrto_last_error() gives the message of the last failure on the calling thread.
 *  - Device loops are bounded (max_inner / max_dr); a solve never waits unboundedly.
 */
#ifndef NRTO_H
#define NRTO_H

#ifdef __cplusplus
extern "C" {
#endif

#define NRTO_ABI_VERSION 2

typedef enum {
  NRTO_OK = 0,
  NRTO_ERR_INVALID = 1,        /* bad argument or descriptor (nothing was changed)            */
  NRTO_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed                  */
  NRTO_ERR_NOT_CONVERGED = 3,  /* some instance stopped at its iteration cap                  */
  NRTO_ERR_NUMERIC = 4,        /* non-finite input, or a non-finite residual in some instance */
  NRTO_ERR_TIMEOUT = 5,        /* a bounded device wait gave up (nrto_mlp_train_step); solver
                                  instances that time out report per-instance status 4 instead */
  NRTO_ERR_STATE = 6           /* call order violated (e.g. solve before linearize)           */
} nrto_status;

typedef enum { NRTO_DYN_UNICYCLE = 0, NRTO_DYN_QUADCOPTER = 1, NRTO_DYN_ARM = 2 } nrto_dyn_kind;
/* NRTO_SOLVER_FULLADMM: Algorithm 1 with block 2a lifted (the linearized robust constraints and the
 * trust region as projected slack variables, so that block 2a is an LQ problem with a factorization
 * fixed per outer step).  NRTO_SOLVER_FULLADMM_AW: block 2a as the paper states it (Sec. IV), the
 * constrained (δû, p) QP solved exactly every iteration (NRTO-DR's subproblem 2 with v = p̃ - λ_p);
 * fixed ρ, no carry, no warm start.  Both have the Problem 2 solution as fixed point. */
typedef enum { NRTO_SOLVER_DR = 0, NRTO_SOLVER_FULLADMM = 1, NRTO_SOLVER_FULLADMM_AW = 2 } nrto_solver_kind;
typedef enum { NRTO_PREC_FP64 = 0, NRTO_PREC_MIXED = 1 } nrto_precision;

/* One instance of Problem 1 (Sec. II-A).  Dimensions must match the model:
 * unicycle (3,2), quadcopter (12,4), arm (14,7).  ±INFINITY marks an absent bound. */
typedef struct {
  int dyn;                       /* nrto_dyn_kind                                              */
  int nx, nu, T;                 /* state dim, input dim, horizon (1 <= T <= 256/160/128)     */
  double dt;                     /* forward-Euler step (> 0)                                   */
  const double* dyn_params;      /* quadcopter [m, g, Jx, Jy, Jz]; unicycle none; arm: standard-DH rows
                                    (a, d, α) × 7 — 21 values: the double integrator — optionally
                                    followed by damping d (7), inertia I (7) and a clamping flag (1):
                                    the Franka model q̈ = (τ - d q̇)/I with the joint position and
                                    velocity limits (the state bounds) clamped after each Euler step
                                    (Supplementary Sec. IV-A)                                       */
  int n_dyn_params;
  const double* x0;              /* nx    nominal initial state x̄_0                            */
  const double* x_goal;          /* nx    goal of the state-tracking cost                       */
  const double* u_init;          /* T*nu  initial nominal controls û                            */
  const double* u_ref;           /* nu    reference of the input cost                           */
  const double* Sigma;           /* (T+1)*nx*nx  blocks Σ_i = Γ_i S_i^{-1} Γ_iᵀ of the disturbance set
                                    {ζ = Γz, zᵀSz ≤ τ} with Γ and S block diagonal per step (Γ = I:
                                    Σ_i = S_i^{-1}); symmetric positive semidefinite (a Γ_i with fewer
                                    columns than rows gives a singular block)                       */
  double tau;                    /* ellipsoid radius τ >= 0                                     */
  const double* Qx;              /* nx    diagonal state-tracking weight                        */
  const double* Ru;              /* nu    diagonal input weight R_u (> 0)                       */
  const double* RK;              /* nu    diagonal gain weight R_K (> 0)                        */
  int n_obs, obs_dim;            /* spheres; obs_dim 2 (unicycle) or 3                          */
  const double* obs_center;      /* n_obs*obs_dim                                               */
  const double* obs_radius;      /* n_obs                                                       */
  int n_link;                    /* arm only: link spheres                                      */
  const double* link_spheres;    /* n_link*5: link index 1..7, offset x,y,z, radius             */
  const double* u_lo; const double* u_hi;   /* nu                                              */
  const double* x_lo; const double* x_hi;   /* nx                                              */
} nrto_problem_desc;

typedef struct {
  int solver;          /* nrto_solver_kind                                                      */
  double rho;          /* FullADMM penalty ρ (scaled duals); NRTO-DR: ADMM penalty of Problem 3  */
  double alpha;        /* DR relaxation α ∈ (0,1)                                                */
  double r_chi, sigma; /* DR proximal scalings R_χ = r_χ I, R_s = σ I                            */
  double eps_p, eps_d; /* inner stopping tolerances on the full primal / dual residuals         */
  double eps_dr;       /* DR stopping tolerance on ‖s̃^l - s̃^{l-1}‖                               */
  int max_inner;       /* FullADMM iterations / NRTO-DR ADMM iterations cap                      */
  int max_dr;          /* DR iterations cap per ADMM iteration                                   */
  int check;           /* 1: stop at tolerance; 0: run exactly max_inner iterations             */
  double r0, r_min, w_p;  /* outer loop: initial/max trust radius, minimum radius, merit weight   */
  /* FullADMM residual balancing (standard ADMM penalty adaptation; the paper keeps ρ fixed): every
   * adapt_every iterations ρ ← min(τρ, ρ_max) if r_p > μ r_d, ρ ← max(ρ/τ, ρ_min) if r_d > μ r_p,
   * using the residuals of the iteration before last; scaled duals are rescaled.  0 disables it. */
  int adapt_every;
  double adapt_mu, adapt_tau, rho_min, rho_max;
  /* Stall stop: every stall_every iterations, stop when r_p is above eps_p and fell by less than
   * the factor stall_ratio since the previous checkpoint (status 5; an infeasible linearization).
   * 0 disables it. */
  int stall_every;
  double stall_ratio;
  /* FullADMM with a warm start (nrto_set_warm_start): when the warm-started run stops on the stall
   * rule, rerun the instance from the cold initialization of Algorithm 1 with the full iteration
   * budget (reported iterations count both runs; NRTO_F_STATS flags it).  0 disables it. */
  int warm_fallback;
  /* FullADMM inner-state carry (the library's warm start across successive-linearization steps;
   * the paper re-initializes every inner solve, Algorithm 1): 1 starts each inner solve after the
   * first from the state the previous FullADMM inner solve of the problem ended in — K, p, p̃, the
   * scaled duals λ_p, λ_ν, λ_w, λ_e and the penalty they are scaled for; δû, δx and e as well
   * unless the nominal moved to û + δû since (an accepted outer step), in which case they restart
   * at zero, the previous solution's coordinates in the new linearization.  The first inner solve
   * after nrto_problem_create, nrto_problem_update, nrto_linearize with a new nominal or the reset
   * of nrto_solve starts cold, and so does one after a non-finite or timed-out solve.  A pending
   * learned warm start (nrto_set_warm_start*) takes precedence.  NRTO-DR ignores it.  0 disables. */
  int carry;
  /* nrto_solve only: iteration cap of the inner solve of its last outer step (0: max_inner), so that
   * the inner solves during the successive linearization can stay inexact (the paper runs 40 FullADMM
   * iterations per outer step, Supplementary Tables VI-VIII) while the subproblem of the returned step
   * is solved to the tolerances. */
  int max_inner_final;
  /* FullADMM (NRTO_SOLVER_FULLADMM) k_v update by matrix-free Jacobi-preconditioned conjugate
   * gradients (Sec. IV, GPU implementation: the k_v update by PCG) instead of the exact per-step
   * Kronecker solve: the system (Q_v + ρ Σ_j Â_jᵀÂ_j) k = r is applied step by step without being
   * formed, the preconditioner is its diagonal, each update starts from the previous gains and stops
   * when ‖r - H k‖ ≤ kv_pcg_tol ‖r‖ or after kv_pcg_iters iterations.  0 iterations: the exact solve.
   * Other solver kinds reject kv_pcg_iters > 0. */
  int kv_pcg_iters;
  double kv_pcg_tol;
  /* FullADMM budget stop, with stall_every > 0 (the library's scheduling rule; the paper runs a fixed
   * budget): at a stall checkpoint where r_p is above eps_p but fell by at least the factor
   * stall_ratio, stop (status 5) when stall_budget times the iterations that r_p would need to reach
   * eps_p, at the rate it fell over the last period, exceeds the iterations left under the cap, so that
   * a solve that cannot meet the tolerance within its cap ends early.  0 disables it; must be >= 0. */
  double stall_budget;
} nrto_solver_opts;

/* Per-instance sizes, for sizing output buffers. */
typedef struct {
  int nx, nu, T, n_rows, n_state_rows, n_control_rows;
  long long n_entries;           /* ragged row entries (state + control rows)                  */
  long long n_entries_state;
} nrto_instance_info;

/* Outputs of an inner solve; every pointer may be NULL (skipped).  Host buffers, concatenated
 * over instances with the sizes of nrto_instance_info. */
typedef struct {
  double* du;          /* Σ T*nu       δû                                                        */
  double* K;           /* Σ T*nu*nx    K_k                                                       */
  double* p;           /* Σ n_rows     p                                                         */
  double* ptilde;      /* Σ n_rows     p̃                                                         */
  int* iters;          /* n            iterations run                                            */
  double* r_p;         /* n            full primal residual                                      */
  double* r_d;         /* n            full dual residual                                        */
  int* status;         /* n            1 converged, 2 iteration cap, 3 non-finite, 4 copy timeout,
                                        5 stalled (primal residual stopped decreasing)            */
} nrto_socp_out;

typedef struct nrto_problem* nrto_problem_t;
typedef struct nrto_mlp* nrto_mlp_t;   /* the warm-start network (nrto_mlp_*) */

/* Create a batch of n_instances problems (descs[0..n-1]) in the given precision on `cuda_stream`
 * (a cudaStream_t, or NULL for the default stream).  Copies all inputs to the device, allocates all
 * device memory of the batch, validates every descriptor (dims, finiteness, Σ_i symmetric positive
 * semidefinite, τ >= 0).
 * The nominal of each instance is its u_init; the trust radius is 2.0 until set by nrto_solve or
 * nrto_set_trust_radius. */
nrto_status nrto_problem_create(const nrto_problem_desc* descs, int n_instances, int precision,
                                void* cuda_stream, nrto_problem_t* out);
nrto_status nrto_problem_destroy(nrto_problem_t p);
nrto_status nrto_problem_info(nrto_problem_t p, int instance, nrto_instance_info* info);

/* Replace the problem data of every instance (same dyn, nx, nu, T, obstacle and bound structure as
 * at create) and reset the nominal to the new u_init.  Host → device copies only. */
nrto_status nrto_problem_update(nrto_problem_t p, const nrto_problem_desc* descs, int n_instances);

/* Linearize Problem 1 around the current nominal (Problem 2 data, Supplementary Sec. I): rollout
 * x̂, Jacobians A_k, B_k, g_j(x̂), ∇g_j, the ragged rows b̂_j and b_j, and the Gram matrices of the
 * gain Hessian.  u_hat (Σ T*nu, host) replaces the nominal first; NULL keeps it. */
nrto_status nrto_linearize(nrto_problem_t p, const double* u_hat);

/* Set the trust radius r of Problem 2 per instance (host array of n values). */
nrto_status nrto_set_trust_radius(nrto_problem_t p, const double* r);

/* One inner solve of Problem 2 at the current linearization for every instance (FullADMM or
 * NRTO-DR per opts->solver).  Cold start (Algorithm 1 zero initialization) unless a warm start was
 * set.  out may be NULL (results stay on the device).  Returns NRTO_ERR_NOT_CONVERGED if some
 * instance hit its cap while opts->check == 1, NRTO_ERR_NUMERIC on non-finite residuals. */
nrto_status nrto_solve_socp(nrto_problem_t p, const nrto_solver_opts* opts, nrto_socp_out* out);

/* One successive-linearization step: inner solve, candidate ū = û + δû with gains K, linearization
 * at the candidate, merit test, accept/reject and trust-radius update.  accepted (n ints) may be NULL. */
nrto_status nrto_outer_step(nrto_problem_t p, const nrto_solver_opts* opts, int* accepted);

/* Full solve: reset to u_init and r = opts->r0, linearize, then n_outer outer steps.  Outputs
 * (host, may be NULL): u_bar Σ T*nu, K Σ T*nu*nx, merit n.
 * The launch sequence (one persistent solver launch per dynamics kind and outer step, and the
 * outer-loop kernels) is captured into a CUDA graph on a call and replayed by later calls with the same
 * options, n_outer and warm-start state, unless graphs are off (nrto_set_graph), solver profiling is
 * on (nrto_profile) or the problem runs on a default stream (NULL, legacy or per-thread; those cannot
 * be captured).  The first call with new options captures; make it outside any stream capture. */
nrto_status nrto_solve(nrto_problem_t p, const nrto_solver_opts* opts, int n_outer,
                       double* u_bar, double* K, double* merit);

/* Enable (default) or disable the CUDA graph of nrto_solve; disabling drops the captured graph. */
nrto_status nrto_set_graph(nrto_problem_t p, int enable);
/* Number of captures and of replays of nrto_solve's graph since create. */
nrto_status nrto_graph_info(nrto_problem_t p, long long* captures, long long* replays);

/* Launch mapping of the persistent inner-loop launches (one per dynamics kind of the batch; each CTA
 * takes whole instances from the kind's largest-first queue):
 *   0  the kinds one after another, each with as many CTAs as fit on the GPU;
 *   1  the kinds at the same time (largest kind first; the next kind's CTAs take the SMs the first
 *      frees), each with as many CTAs as fit — the default;
 *   2  the kinds at the same time with the SMs split in proportion to the kinds' row entries;
 *   3  as 2, in proportion to row entries × horizon.
 * Results do not depend on the mapping (instances are independent): only the time does. */
#define NRTO_NMAPPING 4
nrto_status nrto_set_launch_mapping(nrto_problem_t p, int mapping);
/* Autotuner of the launch mapping: for each mapping, one warm-up nrto_solve(opts, n_outer) and then
 * reps timed ones (CUDA events on the problem's stream); keeps the fastest for later launches.  ms_out
 * (may be NULL, NRTO_NMAPPING values) receives each mapping's milliseconds per solve, chosen the pick.
 * The solves replace the problem's solver state like nrto_solve does.  Profiling must be off. */
nrto_status nrto_autotune(nrto_problem_t p, const nrto_solver_opts* opts, int n_outer, int reps, double* ms_out,
                          int* chosen);

/* Warm start of the next inner solve from a network (the library's learned warm start; the paper
 * names it as future work): runs nrto_mlp_forward on features (host, n × network input) with the
 * output kept on the device, then for instance i sets K from output[i][k_off ..] (T*nu*nx values,
 * the K layout of nrto_export), and p̃ / λ_p of its row r from output[i][pt_off + row_map[R]] /
 * output[i][lp_off + row_map[R]] (R: row index over all instances in problem order; row_map < 0
 * gives 0).  λ_ν = 0.  The network's max_batch must be >= n.  Synchronizes both streams. */
nrto_status nrto_set_warm_start_from_network(nrto_problem_t p, nrto_mlp_t m, const float* features,
                                            const int* row_map, int k_off, int pt_off, int lp_off);

/* The lifted warm start (nrto_set_warm_start_lifted) from the network in one call: offsets (host,
 * 8 ints) into output[i]: K, p̃, λ_p as above, then per row θ (clipped at 0) and λ_w through row_map,
 * δû (T*nu), λ_e (T*nx, steps 1..T), and log ρ.  A lifted part whose offset is < 0 is absent (zero;
 * for ρ the solver's); with all five absent this is nrto_set_warm_start_from_network. */
nrto_status nrto_set_warm_start_from_network_lifted(nrto_problem_t p, nrto_mlp_t m, const float* features,
                                                    const int* row_map, const int* offsets);

/* Warm start for the next inner solve only: K (Σ T*nu*nx), p̃ and λ_p (Σ n_rows each); λ_ν = 0. */
nrto_status nrto_set_warm_start(nrto_problem_t p, const double* K, const double* ptilde,
                                const double* lambda_p);

/* Lifted warm start (NRTO_SOLVER_FULLADMM with the lifted block 2), on top of the pending
 * nrto_set_warm_start (NRTO_ERR_STATE without one): the rest of the iteration's state, so that a
 * solution's values restart at its fixed point.
 *   theta    host, Σ n_rows: per row θ_j ≥ 0 (negative values count as 0); the SOC dual becomes
 *            λ_ν,j = θ_j (Â_j k + b̂_j) with the warm-start gains k: at a fixed point
 *            ν_j = Π(Â_j k + b̂_j + λ_ν,j) = Â_j k + b̂_j, so λ_ν,j = (1/s_j - 1)(Â_j k + b̂_j) with the
 *            projection scale s_j (NRTO_F_S) of a row not projected to zero;
 *   lambda_w host, Σ n_rows: the orthant coupling's scaled dual (NRTO_F_LAMW);
 *   du       host, Σ T*nu: δû (then δx = F_u δû and b_jᵀδû are formed on the device);
 *   lambda_e host, Σ T*nx: the trust-region coupling's scaled dual at steps 1..T (NRTO_F_LAME);
 *   rho      host, n doubles, or null: the penalty the scaled duals belong to, at which the solve
 *            starts (and block 2 is factored); null: the solver's ρ.
 * The next inner solve must be FullADMM (another solver kind returns NRTO_ERR_STATE); a later
 * nrto_set_warm_start replaces the lifted start. */
nrto_status nrto_set_warm_start_lifted(nrto_problem_t p, const double* theta, const double* lambda_w,
                                       const double* du, const double* lambda_e, const double* rho);

/* Per-instance solve statistics of the whole batch in one call: out (host, n × width doubles,
 * width >= NRTO_NSTAT), row i = instance i:
 *  0 inner iterations since the last nrto_solve reset     1 iterations of the last inner solve
 *  2 status of the last inner solve (nrto_socp_out.status codes)
 *  3 accepted outer steps                                  4 final ρ of the last inner solve
 *  5 NRTO-DR iterations summed over its ADMM iterations    6 1 if the last solve fell back to cold
 *  7 status of the inner solve that produced the accepted iterate (0: no step accepted yet)
 *  8 merit φ of the accepted iterate                       9 cost J of the accepted iterate
 * 10 max_j g_j(x̄) + ‖Â_j k + b̂_j‖ of the accepted iterate: the largest robust-constraint value of
 *    Problem 2 at δû = 0, linearized at the accepted nominal x̄ (≤ 0: every robust constraint holds
 *    for all disturbances of the ellipsoid, to first order about x̄; -INFINITY without rows)
 * 11 trust radius                                         12, 13 full r_p, r_d of the last inner solve
 * 14 PCG iterations of the k_v updates of the last inner solve (kv_pcg_iters > 0; else 0)
 * Synchronizes the problem's stream. */
#define NRTO_NSTAT 15
nrto_status nrto_get_stats(nrto_problem_t p, double* out, int width);

/* Monte Carlo check of robust-constraint satisfaction (Sec. V, Methodology: disturbances drawn
 * uniformly from the interior of the uncertainty set and reproducible edge cases on its boundary
 * along convex combinations of the constraints' worst-case directions; the satisfaction
 * probability is the fraction of rollouts that violate no constraint).  Per instance, the policy
 * u_k = ū_k + K_k ζ_k at the nominal ū of the current linearization (after nrto_solve: the accepted
 * iterate) is rolled out through the nonlinear dynamics, x_0 = x̄_0 + ζ_0,
 * x_{k+1} = f(x_k, u_k) + ζ_{k+1}, under n_interior + n_edge disturbances ζ_i = √τ Ψ_iᵀ w_i
 * (Ψ_iᵀΨ_i = Σ_i, w ∈ R^{(T+1) n_x}):
 *  - samples 0 .. n_interior-1: w uniform in the unit ball (ζ uniform in the ellipsoid for Γ = I);
 *  - edge sample e: w = v/‖v‖, v = Σ_c a_c y_{j_c}/‖y_{j_c}‖ over n_c = 1 + (e mod 3) rows j_c drawn
 *    uniformly (state rows, then control rows), weights a_c in (0, 1], y_j = Â_j k + b̂_j the row's
 *    SOC vector of Problem 2 at the current linearization;
 * random numbers from SplitMix64 streams keyed by (seed, instance index, sample index), so that a
 * sample is reproducible on its own.  A rollout counts when every constraint of Problem 1 (state
 * rows at t = 1..T, control bounds at k = 0..T-1) is ≤ tol.  FP64 in both precisions (the SOC
 * vectors use the problem's stored b̂, b).
 * K: host, Σ T*nu*nx, the layout of nrto_socp_out.K, or null for the gains of the accepted iterate.
 * n_ok: host, n ints, the rollouts that satisfied every constraint.  worst: host,
 * n × (n_interior + n_edge) doubles (row i = instance i) or null: per sample the largest constraint
 * value.  Allocates and frees its own device scratch; synchronizes the problem's stream.
 * NRTO_ERR_STATE before the first linearization. */
nrto_status nrto_monte_carlo(nrto_problem_t p, const double* K, int n_interior, int n_edge, unsigned long long seed,
                             double tol, int* n_ok, double* worst);

/* Named internal arrays of one instance, converted to float64 (checkpointing and testing).
 * field: one of NRTO_F_*; count must equal the field's size for that instance. */
enum {
  NRTO_F_XHAT = 0,   /* (T+1)*nx   nominal states of the current linearization               */
  NRTO_F_UHAT = 1,   /* T*nu       nominal controls                                          */
  NRTO_F_A = 2,      /* T*nx*nx                                                              */
  NRTO_F_B = 3,      /* T*nx*nu                                                              */
  NRTO_F_G0 = 4,     /* n_rows     g_j at the nominal                                        */
  NRTO_F_BHAT = 5,   /* n_entries_state  b̂ rows (ragged)                                      */
  NRTO_F_BVEC = 6,   /* Σ_state rows (t+1)*nu  b_{j,m} rows (ragged, block t zero)            */
  NRTO_F_LAMNU = 7,  /* n_entries  λ_ν (FullADMM) or η̃ (DR) rows (ragged)                     */
  NRTO_F_K = 8,      /* T*nu*nx    gains of the last inner solve                             */
  NRTO_F_DU = 9,     /* T*nu       δû of the last inner solve                                */
  NRTO_F_P = 10,     /* n_rows                                                                */
  NRTO_F_PT = 11,    /* n_rows     p̃                                                          */
  NRTO_F_LAMP = 12,  /* n_rows     λ_p (FullADMM, scaled) or λ (NRTO-DR, unscaled)            */
  NRTO_F_GM = 13,    /* T*nu*nu    Σ_j b_{j,m} b_{j,m}ᵀ                                        */
  NRTO_F_KACC = 14,  /* T*nu*nx    gains of the accepted nominal (outer loop)                 */
  NRTO_F_DX = 15,    /* (T+1)*nx   δx of the last inner solve                                */
  NRTO_F_SCAL = 16,  /* 8: r_p, r_d, r_p(paper), r_d(paper), merit, candidate merit, cost, trust r */
  NRTO_F_STATS = 17, /* 7, read-only: inner iterations since the last nrto_solve reset, iterations of
                        the last inner solve, its status, accepted outer steps, its final ρ,
                        (NRTO-DR) the DR iterations summed over its ADMM iterations, and 1 if the
                        last solve fell back from a warm start to a cold start                    */
  NRTO_F_LAMW = 18,  /* n_rows     λ_w, the scaled dual of the lifted orthant coupling (FullADMM)     */
  NRTO_F_LAME = 19,  /* (T+1)*nx   λ_e, the scaled dual of the lifted trust-region coupling (step 0
                        unused)                                                                   */
  NRTO_F_S = 20      /* n_rows     projection scale s_j of the last row pass (ν_j = s_j η̂_j)           */
};
nrto_status nrto_export(nrto_problem_t p, int field, int instance, double* dst, long long count);
nrto_status nrto_import(nrto_problem_t p, int field, int instance, const double* src, long long count);

/* Solver-kernel timing with CUDA events recorded on the problem's stream around the persistent
 * inner-loop launches of each inner solve (one launch per dynamics kind in the batch; the kinds' launches
 * run at the same time on two streams).  Returns (and clears) the milliseconds of those intervals and
 * the number of kernel launches in them since the previous call, then enables (enable != 0) or
 * disables recording for later solves.  Synchronizes the stream when events are pending. */
nrto_status nrto_profile(nrto_problem_t p, int enable, double* solver_ms, long long* solver_launches);

/* Per-phase SM cycles of the inner-loop kernels, summed over CTAs (thread 0 of each CTA marks the
 * phase boundaries), recorded while nrto_profile recording is enabled; returned and cleared.
 * Phases: 0 initialization, 1 row pass (cone projections, λ_ν update, Z' accumulation), 2 control
 * rows and residual reduction, 3 orthant/ball slacks, 4 Riccati linear terms, 5 gain solve,
 * 6 Riccati sweep, 7 scalar duals, 8 time spent waiting for row-chunk copies (included in 1).
 * n must be >= NRTO_NPHASE. */
#define NRTO_NPHASE 9
nrto_status nrto_phase_cycles(nrto_problem_t p, long long* cycles, int n);

/* Number of kernel launches the library issued since create (all of its own kernels). */
long long nrto_kernel_launches(nrto_problem_t p);

/* Self-test of the device-side watchdog (the paper has no counterpart: it describes no failure
 * handling).  Every solver kernel waits for its bulk copies with a wait bounded by 2^32 SM cycles,
 * about two seconds, after which the instance ends with per-instance status 4 instead of hanging.
 * This call runs that wait on the current device against a barrier that nothing completes:
 * *status_out receives 4 when the wait gave up as designed (1 would mean the barrier completed),
 * *cycles_out (optional, may be NULL) the SM cycles waited.  It blocks for those two seconds,
 * allocates and frees 16 bytes of device memory, and leaves the device usable.  stream: a
 * cudaStream_t or NULL (legacy default stream).  NRTO_ERR_INVALID for a NULL status_out,
 * NRTO_ERR_CUDA for a CUDA failure. */
nrto_status nrto_selftest_bounded_wait(void* stream, int* status_out, long long* cycles_out);

/* ---- Learned warm start: a GELU multilayer perceptron (the paper names learning a warm start
 * for the inner solver as future work and fixes no network; this is the library's own).
 * z_l = h_{l-1} W_lᵀ + b_l, h_l = gelu(z_l) = z_l Φ(z_l) for hidden layers, y = z_L.  Trained on the
 * masked mean-squared error Σ mask (y - t)² / Σ mask with Adam (β₁ = 0.9, β₂ = 0.999, ε = 1e-8).
 * FP32 master parameters; bf16 weights and activations on fifth-generation tensor cores with FP32
 * accumulation.  Parameter layout (flat float array): for each layer l, W_l (out × in, row-major)
 * then b_l (out).  All array arguments are host pointers, row-major. ---- */

/* dims: n_dims widths (input, hidden..., output); every width after the input a multiple of 8.
 * max_batch: a multiple of 8.  Parameters start at zero (set them with nrto_mlp_set_params). */
nrto_status nrto_mlp_create(const int* dims, int n_dims, int max_batch, void* stream, nrto_mlp_t* out);
nrto_status nrto_mlp_destroy(nrto_mlp_t m);
long long nrto_mlp_num_params(nrto_mlp_t m);
/* Copy all parameters in (resets the Adam moments and step count) or out. */
nrto_status nrto_mlp_set_params(nrto_mlp_t m, const float* params);
nrto_status nrto_mlp_get_params(nrto_mlp_t m, float* params);
/* y (batch × out) = network(x) (batch × in), 1 <= batch <= max_batch. */
nrto_status nrto_mlp_forward(nrto_mlp_t m, const float* x, int batch, float* y);
/* One training step on (x, target, mask): forward, backward, then Adam with learning rate lr
 * (lr = 0: gradients only).  loss (may be NULL) receives the masked MSE before the update; grads
 * (may be NULL) the gradient in the parameter layout.  batch: a multiple of 8 <= max_batch.
 * NRTO_ERR_TIMEOUT if a tensor-core pipeline wait gave up (the result is then invalid). */
nrto_status nrto_mlp_train_step(nrto_mlp_t m, const float* x, const float* target, const float* mask,
                                int batch, float lr, double* loss, float* grads);
/* Number of kernel launches issued for this network since create. */
long long nrto_mlp_kernel_launches(nrto_mlp_t m);
/* Tensor-core GEMM timing: CUDA events on the network's stream around every GEMM launch while
 * enabled.  Returns (and clears) the milliseconds, the algorithmic FLOPs (2·M·N·K) and the launch
 * count since the previous call, then enables (enable != 0) or disables recording. */
nrto_status nrto_mlp_profile(nrto_mlp_t m, int enable, double* gemm_ms, double* gemm_flops,
                             long long* gemm_launches);

/* nrto_solve without device allocation.  The paper has no counterpart: this is a library service.
 * Some callers cannot call cudaMalloc: real-time control loops that must not pay an allocation's
 * latency and implicit synchronization, and processes whose device memory is held by another
 * allocator (a framework's caching pool), where an allocation may fail mid-run.  This call does what
 * nrto_problem_create + nrto_solve + nrto_problem_destroy do, with the same kernels and results, but
 * every device buffer of the batch is cut from one static 32 MiB device area that the library holds
 * on every GPU that loads it, until the process exits.  It calls no cudaMalloc or cudaFree.
 *   descs, n, precision: as nrto_problem_create; opts, n_outer, u_bar, K, merit: as nrto_solve
 *     (host arrays, may be NULL); stream: CUDA stream (NULL: default stream).
 *   Errors: NRTO_ERR_INVALID when the batch does not fit in the area (the message says so; use
 *     nrto_problem_create then), otherwise as nrto_problem_create and nrto_solve.
 * The first call on a device looks up the device address of the area (cudaGetSymbolAddress); make
 * that first call before any stream capture on that device.  All calls share the area, which keeps
 * the previous call's contents: each call clears every buffer it uses before use.  Two calls that
 * ran on the GPU at the same time would overwrite each other's data, so calls in one process are
 * serialized by a lock and each returns only after its GPU work has finished. */
nrto_status nrto_solve_noalloc(const nrto_problem_desc* descs, int n, int precision,
                               const nrto_solver_opts* opts, int n_outer, void* stream,
                               double* u_bar, double* K, double* merit);

/* Message of the last failure on the calling thread ("" if none). */
const char* nrto_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NRTO_H */
