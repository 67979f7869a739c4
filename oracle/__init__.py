"""CPU oracle for the NRTO inner loop: plain, slow, FP64 NumPy.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference leg of `bench.py` may import anything from this
package.  The CUDA library never calls it and shares no code with it: the two
meet only at the seeded inputs of `paper_2603_02642_b300.workloads`.

Modules (each function cites the passage of the paper it follows):
  models     dynamics f(x,u) of Supplementary Sec. IV-A and the constraint functions g, h;
             Jacobians by complex-step differentiation
  problem    constraint rows, linearization, F_u, F_ζ, b_j, Â_j, b̂_j (Supplementary Sec. I)
  soc        closed-form second-order-cone projection (Supplementary Sec. II-C)
  fulladmm   NRTO-FullADMM inner loop (Sec. IV, Algorithm 1, Supplementary Sec. III),
             lifted reading of the Block-2 QP
  dr         NRTO-DR: relaxed Douglas–Rachford on subproblem (7) inside the NRTO ADMM
             (Sec. II-B, Sec. III, Supplementary Sec. II)
  outer      successive-linearization outer loop (Fig. 1, Problem 2)
  mlp        FP64 reference MLP forward/backward for the learned warm start
  montecarlo robust-constraint satisfaction under sampled interior and edge disturbances
             (Sec. V, Methodology), SplitMix64 counter-based random numbers

Parity status: every function here is pinned by `tests/test_oracle_*.py` against
closed forms, invariants, brute force or an independent solver.  The outer loop
(`outer.solve`) is pinned on a convex case, where its end point is fixed by the
mathematics; the constants of its accept/reject rule and radius schedule come from
prior work that the paper does not restate, so they remain a reading.
"""
