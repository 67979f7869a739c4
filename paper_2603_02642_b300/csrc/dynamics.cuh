// Analytic dynamics, Jacobians and constraint gradients (device side of libnrto).
//
// Models (Supplementary Sec. IV-A, forward Euler): unicycle (3,2), quadcopter (12,4) with
// R = Rz(ψ)Ry(θ)Rx(φ) and Euler-rate map T(φ,θ), and the 7-joint Franka joint-space model (damping,
// inertia, clamped limits; the double integrator when those are off) whose link spheres move through
// a Denavit–Hartenberg chain.
#pragma once
#include "nrto_dev.cuh"

namespace nrto {

// x_{k+1} = f(x_k, u_k); A = ∂f/∂x, B = ∂f/∂u (row-major nx×nx, nx×nu). A, B may be null.
// xlo, xhi: the state bounds (the arm's clamping limits).
__device__ inline void dyn_step(int kind, const double* prm, double dt, const double* x, const double* u,
                                double* xn, double* A, double* B, const double* xlo, const double* xhi) {
  if (kind == KIND_UNICYCLE) {
    double c = cos(x[2]), s = sin(x[2]);
    xn[0] = x[0] + u[0] * c * dt;
    xn[1] = x[1] + u[0] * s * dt;
    xn[2] = x[2] + u[1] * dt;
    if (A) {
      A[0] = 1; A[1] = 0; A[2] = -u[0] * s * dt;
      A[3] = 0; A[4] = 1; A[5] = u[0] * c * dt;
      A[6] = 0; A[7] = 0; A[8] = 1;
    }
    if (B) {
      B[0] = c * dt; B[1] = 0;
      B[2] = s * dt; B[3] = 0;
      B[4] = 0; B[5] = dt;
    }
    return;
  }
  if (kind == KIND_QUADCOPTER) {
    const double m = prm[0], g = prm[1], Jx = prm[2], Jy = prm[3], Jz = prm[4];
    const double ph = x[6], th = x[7], ps = x[8], wp = x[9], wq = x[10], wr = x[11];
    const double f = u[0];
    const double cph = cos(ph), sph = sin(ph), cth = cos(th), sth = sin(th), cps = cos(ps), sps = sin(ps);
    const double tth = sth / cth;
    const double r0 = cps * sth * cph + sps * sph;   // R e3
    const double r1 = sps * sth * cph - cps * sph;
    const double r2 = cth * cph;
    double xd[12];
    xd[0] = x[3]; xd[1] = x[4]; xd[2] = x[5];
    xd[3] = f / m * r0; xd[4] = f / m * r1; xd[5] = f / m * r2 - g;
    xd[6] = wp + wq * sph * tth + wr * cph * tth;
    xd[7] = wq * cph - wr * sph;
    xd[8] = (wq * sph + wr * cph) / cth;
    xd[9] = (u[1] - (Jz - Jy) * wq * wr) / Jx;
    xd[10] = (u[2] - (Jx - Jz) * wr * wp) / Jy;
    xd[11] = (u[3] - (Jy - Jx) * wp * wq) / Jz;
    for (int i = 0; i < 12; ++i) xn[i] = x[i] + dt * xd[i];
    if (A) {
      double J[144];
      for (int i = 0; i < 144; ++i) J[i] = 0.0;
      J[0 * 12 + 3] = 1; J[1 * 12 + 4] = 1; J[2 * 12 + 5] = 1;
      const double fm = f / m;
      J[3 * 12 + 6] = fm * (-cps * sth * sph + sps * cph);
      J[3 * 12 + 7] = fm * (cps * cth * cph);
      J[3 * 12 + 8] = fm * (-sps * sth * cph + cps * sph);
      J[4 * 12 + 6] = fm * (-sps * sth * sph - cps * cph);
      J[4 * 12 + 7] = fm * (sps * cth * cph);
      J[4 * 12 + 8] = fm * (cps * sth * cph + sps * sph);
      J[5 * 12 + 6] = fm * (-cth * sph);
      J[5 * 12 + 7] = fm * (-sth * cph);
      J[6 * 12 + 6] = wq * cph * tth - wr * sph * tth;
      J[6 * 12 + 7] = (wq * sph + wr * cph) / (cth * cth);
      J[6 * 12 + 9] = 1; J[6 * 12 + 10] = sph * tth; J[6 * 12 + 11] = cph * tth;
      J[7 * 12 + 6] = -wq * sph - wr * cph;
      J[7 * 12 + 10] = cph; J[7 * 12 + 11] = -sph;
      J[8 * 12 + 6] = (wq * cph - wr * sph) / cth;
      J[8 * 12 + 7] = (wq * sph + wr * cph) * sth / (cth * cth);
      J[8 * 12 + 10] = sph / cth; J[8 * 12 + 11] = cph / cth;
      J[9 * 12 + 10] = -(Jz - Jy) * wr / Jx; J[9 * 12 + 11] = -(Jz - Jy) * wq / Jx;
      J[10 * 12 + 9] = -(Jx - Jz) * wr / Jy; J[10 * 12 + 11] = -(Jx - Jz) * wp / Jy;
      J[11 * 12 + 9] = -(Jy - Jx) * wq / Jz; J[11 * 12 + 10] = -(Jy - Jx) * wp / Jz;
      for (int i = 0; i < 144; ++i) A[i] = dt * J[i];
      for (int i = 0; i < 12; ++i) A[i * 12 + i] += 1.0;
    }
    if (B) {
      for (int i = 0; i < 48; ++i) B[i] = 0.0;
      B[3 * 4 + 0] = dt * r0 / m; B[4 * 4 + 0] = dt * r1 / m; B[5 * 4 + 0] = dt * r2 / m;
      B[9 * 4 + 1] = dt / Jx; B[10 * 4 + 2] = dt / Jy; B[11 * 4 + 3] = dt / Jz;
    }
    return;
  }
  // arm (Franka joint-space model): q̈ = (τ - d q̇)/I; q̇' = clip(q̇ + q̈ dt), q' = clip(q + q̇' dt) when
  // clamping is on (limits: the state bounds).  A clamped component has zero derivatives.
  const double* dmp = prm + ARM_DAMP;
  const double* inr = prm + ARM_INERT;
  const bool clamp = prm[ARM_CLIP] != 0.0;
  if (A) for (int i = 0; i < 196; ++i) A[i] = 0.0;
  if (B) for (int i = 0; i < 98; ++i) B[i] = 0.0;
  for (int i = 0; i < 7; ++i) {
    double v = x[7 + i] + (u[i] - dmp[i] * x[7 + i]) / inr[i] * dt;
    double sv = 1.0;
    if (clamp) {
      if (v < xlo[7 + i]) { v = xlo[7 + i]; sv = 0.0; }
      else if (v > xhi[7 + i]) { v = xhi[7 + i]; sv = 0.0; }
    }
    double qn = x[i] + v * dt;
    double sq = 1.0;
    if (clamp) {
      if (qn < xlo[i]) { qn = xlo[i]; sq = 0.0; }
      else if (qn > xhi[i]) { qn = xhi[i]; sq = 0.0; }
    }
    xn[7 + i] = v;
    xn[i] = qn;
    const double dv_dv = sv * (1.0 - dt * dmp[i] / inr[i]), dv_du = sv * dt / inr[i];
    if (A) {
      A[(7 + i) * 14 + 7 + i] = dv_dv;
      A[i * 14 + i] = sq;
      A[i * 14 + 7 + i] = sq * dt * dv_dv;
    }
    if (B) {
      B[(7 + i) * 7 + i] = dv_du;
      B[i * 7 + i] = sq * dt * dv_du;
    }
  }
}

// Arm: world position of one link sphere and its Jacobian w.r.t. q (3×7 row-major).
// DH link transform Rot_z(q_i) Trans_z(d_i) Trans_x(a_i) Rot_x(α_i); joint i rotates about the
// z axis of frame i-1, so ∂p/∂q_i = z_{i-1} × (p - o_{i-1}) for i <= link.
__device__ inline void arm_sphere(const double* dh, const double* sph, const double* q, double* p, double* Jp) {
  int link = (int)sph[0];
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double o[3] = {0, 0, 0};
  double zs[7][3], os[7][3];
  for (int i = 0; i < link; ++i) {
    zs[i][0] = R[2]; zs[i][1] = R[5]; zs[i][2] = R[8];
    os[i][0] = o[0]; os[i][1] = o[1]; os[i][2] = o[2];
    const double a = dh[3 * i], d = dh[3 * i + 1], al = dh[3 * i + 2];
    const double ct = cos(q[i]), st = sin(q[i]), ca = cos(al), sa = sin(al);
    const double M[9] = {ct, -st * ca, st * sa, st, ct * ca, -ct * sa, 0, sa, ca};
    const double tr[3] = {a * ct, a * st, d};
    for (int r = 0; r < 3; ++r) o[r] += R[r * 3] * tr[0] + R[r * 3 + 1] * tr[1] + R[r * 3 + 2] * tr[2];
    double Rn[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Rn[r * 3 + c] = R[r * 3] * M[c] + R[r * 3 + 1] * M[3 + c] + R[r * 3 + 2] * M[6 + c];
    for (int k = 0; k < 9; ++k) R[k] = Rn[k];
  }
  for (int r = 0; r < 3; ++r) p[r] = o[r] + R[r * 3] * sph[1] + R[r * 3 + 1] * sph[2] + R[r * 3 + 2] * sph[3];
  for (int i = 0; i < 7; ++i) {
    if (i < link) {
      double dx = p[0] - os[i][0], dy = p[1] - os[i][1], dz = p[2] - os[i][2];
      Jp[0 * 7 + i] = zs[i][1] * dz - zs[i][2] * dy;
      Jp[1 * 7 + i] = zs[i][2] * dx - zs[i][0] * dz;
      Jp[2 * 7 + i] = zs[i][0] * dy - zs[i][1] * dx;
    } else {
      Jp[i] = Jp[7 + i] = Jp[14 + i] = 0.0;
    }
  }
}

// State constraint g_j(x_t) and its gradient for one row (Problem 1 robust constraint): concave
// sphere clearance g = r - ‖P x - c‖ (planar/3-D position, or arm link sphere vs static sphere), or a
// linear state bound.  `ar` is the instance arena, `L` its layout.  At zero distance the gradient
// direction is taken along the first position axis.
__device__ inline double row_g_grad(const Inst& I, const double* ar, const Arena& L, int4 ri,
                                    const double* x, double* grad) {
  const int nx = I.nx;
  for (int c = 0; c < nx; ++c) grad[c] = 0.0;
  const int code = ri.y, a = ri.z, b = ri.w;
  if (code == ROW_XHI) { grad[a] = 1.0; return x[a] - ar[L.xhi + a]; }
  if (code == ROW_XLO) { grad[a] = -1.0; return ar[L.xlo + a] - x[a]; }
  const double* ob = ar + L.obs + 4 * a;   // cx, cy, cz, r
  if (I.kind == KIND_ARM) {
    const double* sp = ar + L.link + 5 * b;
    double p[3], Jp[21];
    arm_sphere(ar + L.dyn, sp, x, p, Jp);
    double d[3] = {p[0] - ob[0], p[1] - ob[1], p[2] - ob[2]};
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (n > 0.0) { d[0] /= n; d[1] /= n; d[2] /= n; } else { d[0] = 1.0; d[1] = d[2] = 0.0; }
    for (int i = 0; i < 7; ++i) grad[i] = -(d[0] * Jp[i] + d[1] * Jp[7 + i] + d[2] * Jp[14 + i]);
    return sp[4] + ob[3] - n;
  }
  const int dim = I.obs_dim;
  double n2 = 0.0;
  for (int k = 0; k < dim; ++k) { double d = x[k] - ob[k]; n2 += d * d; }
  double n = sqrt(n2);
  if (n > 0.0) {
    for (int k = 0; k < dim; ++k) grad[k] = -(x[k] - ob[k]) / n;
  } else {
    grad[0] = -1.0;
  }
  return ob[3] - n;
}

}  // namespace nrto
