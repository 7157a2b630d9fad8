// Quadrotor dynamics, its hand-derived vector-Jacobian product, and one RK4
// step with its adjoint, templated on the scalar type (float, double or the
// forward-mode Dual of either).
//
// Model (Sec. VI quadrotor NMPC; constants are the design readings): state
// (p, v, eta = ZYX Euler angles (phi, theta, psi), omega = body rates), input
// four rotor thrusts.  p' = v; v' = R(eta) e3 T / m - g e3; eta' = W(eta) omega;
// omega' = J^{-1} (tau - omega x J omega) with "+" layout torques.
#pragma once

#include "scalar.cuh"

namespace bipm {

// f(x, u) for one quadrotor.
template <class S>
__host__ __device__ __forceinline__ void quad_f(const S x[12], const S u[4], S out[12]) {
  typedef typename Base<S>::type T;
  S sph, cph, sth, cth, sps, cps;
  sincos_s(x[6], &sph, &cph);
  sincos_s(x[7], &sth, &cth);
  sincos_s(x[8], &sps, &cps);
  S thrust = u[0] + u[1] + u[2] + u[3];
  S tm = thrust * (T)(1.0 / kMass);
  out[0] = x[3];
  out[1] = x[4];
  out[2] = x[5];
  S spsph = sps * sph, cpsph = cps * sph;
  S sthcph = sth * cph;
  out[3] = (cps * sthcph + spsph) * tm;
  out[4] = (sps * sthcph - cpsph) * tm;
  out[5] = cth * cph * tm + (T)(-kGrav);
  S icth = cst<S>((T)1) / cth;
  S tth = sth * icth;
  S a = sph * x[10] + cph * x[11];
  out[6] = x[9] + tth * a;
  out[7] = cph * x[10] - sph * x[11];
  out[8] = a * icth;
  out[9] = ((T)kArm * (u[1] - u[3]) - (T)(kJz - kJy) * (x[10] * x[11])) * (T)(1.0 / kJx);
  out[10] = ((T)kArm * (u[2] - u[0]) - (T)(kJx - kJz) * (x[11] * x[9])) * (T)(1.0 / kJy);
  out[11] = ((T)kYaw * (u[0] - u[1] + u[2] - u[3]) - (T)(kJy - kJx) * (x[9] * x[10])) *
            (T)(1.0 / kJz);
}

// (df/dz)^T w for z = (x, u) of one quadrotor.  `eo` holds (eta, omega) of the
// evaluation point (f's Jacobian depends on nothing else besides the thrust
// sum).  gx[0..11] and gu[0..3] are overwritten.
template <class S>
__host__ __device__ __forceinline__ void quad_vjp(const S eo[6], S thrust, const S w[12], S gx[12],
                                         S gu[4]) {
  typedef typename Base<S>::type T;
  S sph, cph, sth, cth, sps, cps;
  sincos_s(eo[0], &sph, &cph);
  sincos_s(eo[1], &sth, &cth);
  sincos_s(eo[2], &sps, &cps);
  const S& w1 = eo[3];
  const S& w2 = eo[4];
  const S& w3 = eo[5];
  S tm = thrust * (T)(1.0 / kMass);
  // translational part: a = tm * R3(eta) - g e3
  S r0 = cps * sth * cph + sps * sph;
  S r1 = sps * sth * cph - cps * sph;
  S r2 = cth * cph;
  S dphi0 = sps * cph - cps * sth * sph, dphi1 = -(sps * sth * sph) - cps * cph, dphi2 = -(cth * sph);
  S dth0 = cps * cth * cph, dth1 = sps * cth * cph, dth2 = -(sth * cph);
  S dps0 = cps * sph - sps * sth * cph, dps1 = r0;
  S g_phi = tm * (w[3] * dphi0 + w[4] * dphi1 + w[5] * dphi2);
  S g_th = tm * (w[3] * dth0 + w[4] * dth1 + w[5] * dth2);
  S g_ps = tm * (w[3] * dps0 + w[4] * dps1);
  S g_t = (w[3] * r0 + w[4] * r1 + w[5] * r2) * (T)(1.0 / kMass);
  // Euler-rate part
  S icth = cst<S>((T)1) / cth;
  S tth = sth * icth;
  S a = sph * w2 + cph * w3;
  S ad = cph * w2 - sph * w3;  // d a / d phi
  g_phi = g_phi + w[6] * (tth * ad) - w[7] * a + w[8] * (ad * icth);
  S ic2 = icth * icth;
  g_th = g_th + w[6] * (a * ic2) + w[8] * (a * sth * ic2);
  S g_w1 = w[6];
  S g_w2 = w[6] * (sph * tth) + w[7] * cph + w[8] * (sph * icth);
  S g_w3 = w[6] * (cph * tth) - w[7] * sph + w[8] * (cph * icth);
  // rotational part
  const T cx = (T)((kJz - kJy) / kJx), cy = (T)((kJx - kJz) / kJy), cz = (T)((kJy - kJx) / kJz);
  g_w1 = g_w1 - w[10] * (cy * w3) - w[11] * (cz * w2);
  g_w2 = g_w2 - w[9] * (cx * w3) - w[11] * (cz * w1);
  g_w3 = g_w3 - w[9] * (cx * w2) - w[10] * (cy * w1);
  const T lx = (T)(kArm / kJx), ly = (T)(kArm / kJy), yz = (T)(kYaw / kJz);
  gu[0] = g_t - w[10] * ly + w[11] * yz;
  gu[1] = g_t + w[9] * lx - w[11] * yz;
  gu[2] = g_t + w[10] * ly + w[11] * yz;
  gu[3] = g_t - w[9] * lx - w[11] * yz;
  gx[0] = cst<S>((T)0);
  gx[1] = cst<S>((T)0);
  gx[2] = cst<S>((T)0);
  gx[3] = w[0];
  gx[4] = w[1];
  gx[5] = w[2];
  gx[6] = g_phi;
  gx[7] = g_th;
  gx[8] = g_ps;
  gx[9] = g_w1;
  gx[10] = g_w2;
  gx[11] = g_w3;
}

// F = x + dt/6 (k1 + 2 k2 + 2 k3 + k4): one classical RK4 step, value only.
template <class S>
__host__ __device__ __forceinline__ void rk4_value(const S x[12], const S u[4], typename Base<S>::type dt,
                                          S F[12]) {
  typedef typename Base<S>::type T;
  const T cf[4] = {(T)(dt / 6), (T)(dt / 3), (T)(dt / 3), (T)(dt / 6)};
  const T ca[4] = {(T)0, (T)(dt / 2), (T)(dt / 2), dt};
  S z[12], k[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) F[i] = x[i];
  quad_f(x, u, k);
#pragma unroll
  for (int st = 1; st < 4; ++st) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      F[i] = F[i] + cf[st - 1] * k[i];
      z[i] = x[i] + ca[st] * k[i];
    }
    quad_f(z, u, k);
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) F[i] = F[i] + cf[3] * k[i];
}

// One RK4 step and the gradient of lam^T F with respect to (x, u), by a
// reverse sweep over the four stage evaluations.  With Dual scalars seeded
// in one direction this also yields the Jacobian column (F.d) and the
// Hessian-vector product of lam^T F (gx.d, gu.d).
template <class S>
__host__ __device__ __forceinline__ void rk4_fwd_rev(const S x[12], const S u[4],
                                            typename Base<S>::type dt,
                                            const typename Base<S>::type lam[12], S F[12],
                                            S gx[12], S gu[4]) {
  typedef typename Base<S>::type T;
  S eo[4][6];
  S z[12], k[12];
  S thrust = u[0] + u[1] + u[2] + u[3];
#pragma unroll
  for (int i = 0; i < 12; ++i) F[i] = x[i];
#pragma unroll
  for (int i = 0; i < 6; ++i) eo[0][i] = x[6 + i];
  quad_f(x, u, k);
  const T cf[4] = {(T)(dt / 6), (T)(dt / 3), (T)(dt / 3), (T)(dt / 6)};
  const T ca[4] = {(T)0, (T)(dt / 2), (T)(dt / 2), dt};
#pragma unroll
  for (int st = 1; st < 4; ++st) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      F[i] = F[i] + cf[st - 1] * k[i];
      z[i] = x[i] + ca[st] * k[i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) eo[st][i] = z[6 + i];
    quad_f(z, u, k);
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) F[i] = F[i] + cf[3] * k[i];

  // reverse sweep: w = adjoint of k_st
  S w[12], gzx[12], gzu[4];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    gx[i] = cst<S>(lam[i]);
    w[i] = cst<S>(cf[3] * lam[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) gu[i] = cst<S>((T)0);
#pragma unroll
  for (int st = 3; st >= 0; --st) {
    quad_vjp(eo[st], thrust, w, gzx, gzu);
#pragma unroll
    for (int i = 0; i < 12; ++i) gx[i] = gx[i] + gzx[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] = gu[i] + gzu[i];
    if (st > 0) {
#pragma unroll
      for (int i = 0; i < 12; ++i) w[i] = ca[st] * gzx[i] + cf[st - 1] * lam[i];
    }
  }
}

}  // namespace bipm
