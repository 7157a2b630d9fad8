// The 13-state quaternion quadrotor of Sec. VI: dynamics, its hand-derived
// vector-Jacobian product, and one RK4 step with its adjoint, templated on the
// scalar type (float, double or the forward-mode Dual of either), in the form
// of the 12-state routines of quad_model.cuh.  Not yet used by the iteration
// kernels (they solve the 12-state model); host builds of these templates are
// checked against the oracle.
//
// Model (constants are the design readings): state (p, q, v, omega) with q =
// (q_w, q_x, q_y, q_z) the attitude quaternion (body to world), v the body-frame
// velocity, omega the body rates; input four rotor speeds Omega (rad/s), rotor
// thrust K_F Omega^2, "+" layout.  p' = R(q) v; q' = q (x) (0, omega) / 2;
// v' = (T / m) e3 - omega x v - g R(q)^T e3; omega' = J^{-1} (tau - omega x J omega),
// with R(q) = I + 2 q_w [q_v]x + 2 [q_v]x^2 (the unit-quaternion rotation matrix).
#pragma once

#include "scalar.cuh"

namespace bipm {

constexpr double kOmegaHover = 400.0;                                 // rotor speed at hover (rad/s)
constexpr double kThrustCoef = kHover / (kOmegaHover * kOmegaHover);  // K_F: thrust = K_F Omega^2
constexpr double kOmegaMax = 1.4142135623730951 * kOmegaHover;        // thrust range [0, 2 m g / 4]

template <class S>
__host__ __device__ __forceinline__ void cross3(const S a[3], const S b[3], S out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

template <class S>
__host__ __device__ __forceinline__ S dot3(const S a[3], const S b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// R(q) b (sgn = 1) or R(q)^T b (sgn = -1): b + 2 sgn q_w (q_v x b) + 2 q_v x (q_v x b)
template <class S>
__host__ __device__ __forceinline__ void quat_rotate(const S q[4], const S b[3], int sgn, S out[3]) {
  typedef typename Base<S>::type T;
  const S* qv = q + 1;
  S c1[3], c2[3];
  cross3(qv, b, c1);
  cross3(qv, c1, c2);
  const S w2 = (T)(2 * sgn) * q[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = b[i] + w2 * c1[i] + (T)2 * c2[i];
}

// gq += scale * d(a^T R(q) b)/dq, with a^T R b = a.b + 2 q_w q_v.(b x a)
// + 2 ((a.q_v)(q_v.b) - |q_v|^2 a.b)
template <class S>
__host__ __device__ __forceinline__ void quat_rot_grad(const S q[4], const S a[3], const S b[3], S scale,
                                                       S gq[4]) {
  typedef typename Base<S>::type T;
  const S* qv = q + 1;
  S bxa[3];
  cross3(b, a, bxa);
  const S s2 = (T)2 * scale;
  const S qb = dot3(qv, b), aq = dot3(a, qv), ab = dot3(a, b);
  gq[0] = gq[0] + s2 * dot3(qv, bxa);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    gq[1 + i] = gq[1 + i] + s2 * (q[0] * bxa[i] + qb * a[i] + aq * b[i] - (T)2 * ab * qv[i]);
}

// f(x, u) for one quadrotor of the 13-state model.
template <class S>
__host__ __device__ __forceinline__ void quat_f(const S x[13], const S u[4], S out[13]) {
  typedef typename Base<S>::type T;
  const S* q = x + 3;
  const S* v = x + 7;
  const S* w = x + 10;
  S f[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) f[i] = (T)kThrustCoef * (u[i] * u[i]);
  const S thrust = f[0] + f[1] + f[2] + f[3];
  quat_rotate(q, v, 1, out);
  // q' = (-q_v.w, q_w w + q_v x w) / 2
  S qxw[3];
  cross3(q + 1, w, qxw);
  out[3] = (T)(-0.5) * dot3(q + 1, w);
#pragma unroll
  for (int i = 0; i < 3; ++i) out[4 + i] = (T)0.5 * (q[0] * w[i] + qxw[i]);
  // v' = (T / m) e3 - w x v - g R^T e3
  const S e3[3] = {cst<S>((T)0), cst<S>((T)0), cst<S>((T)1)};
  S gb[3], wxv[3];
  quat_rotate(q, e3, -1, gb);
  cross3(w, v, wxv);
  out[7] = -wxv[0] - (T)kGrav * gb[0];
  out[8] = -wxv[1] - (T)kGrav * gb[1];
  out[9] = thrust * (T)(1.0 / kMass) - wxv[2] - (T)kGrav * gb[2];
  // Euler's rotation equations with the "+" layout torques
  out[10] = ((T)kArm * (f[1] - f[3]) - (T)(kJz - kJy) * (w[1] * w[2])) * (T)(1.0 / kJx);
  out[11] = ((T)kArm * (f[2] - f[0]) - (T)(kJx - kJz) * (w[2] * w[0])) * (T)(1.0 / kJy);
  out[12] = ((T)kYaw * (f[0] - f[1] + f[2] - f[3]) - (T)(kJy - kJx) * (w[0] * w[1])) * (T)(1.0 / kJz);
}

// (df/dz)^T lam for z = (x, u) of one quadrotor.  s = (q, v, omega) of the
// evaluation point (f does not depend on p), u its rotor speeds; gx[0..12] and
// gu[0..3] are overwritten.
template <class S>
__host__ __device__ __forceinline__ void quat_vjp(const S s[10], const S u[4], const S lam[13], S gx[13],
                                                  S gu[4]) {
  typedef typename Base<S>::type T;
  const S* q = s;
  const S* v = s + 4;
  const S* w = s + 7;
  const S* lp = lam;
  const S lqw = lam[3];
  const S* lqv = lam + 4;
  const S* lv = lam + 7;
  const S* lw = lam + 10;
  S gq[4] = {cst<S>((T)0), cst<S>((T)0), cst<S>((T)0), cst<S>((T)0)};
  S gv[3], gw[3], t3[3];
  // p' = R(q) v
  quat_rotate(q, lp, -1, gv);
  quat_rot_grad(q, lp, v, cst<S>((T)1), gq);
  // q' = (-q_v.w, q_w w + q_v x w) / 2
  gq[0] = gq[0] + (T)0.5 * dot3(lqv, w);
  cross3(w, lqv, t3);
#pragma unroll
  for (int i = 0; i < 3; ++i) gq[1 + i] = gq[1 + i] + (T)0.5 * (t3[i] - lqw * w[i]);
  cross3(lqv, q + 1, t3);
#pragma unroll
  for (int i = 0; i < 3; ++i) gw[i] = (T)0.5 * (q[0] * lqv[i] + t3[i] - lqw * q[1 + i]);
  // v' = (T / m) e3 - w x v - g R^T e3
  cross3(w, lv, t3);
#pragma unroll
  for (int i = 0; i < 3; ++i) gv[i] = gv[i] + t3[i];
  cross3(lv, v, t3);
#pragma unroll
  for (int i = 0; i < 3; ++i) gw[i] = gw[i] + t3[i];
  const S e3[3] = {cst<S>((T)0), cst<S>((T)0), cst<S>((T)1)};
  quat_rot_grad(q, e3, lv, cst<S>((T)(-kGrav)), gq);
  const S g_thrust = lv[2] * (T)(1.0 / kMass);
  // Euler's rotation equations
  const T cx = (T)((kJz - kJy) / kJx), cy = (T)((kJx - kJz) / kJy), cz = (T)((kJy - kJx) / kJz);
  gw[0] = gw[0] - lw[1] * (cy * w[2]) - lw[2] * (cz * w[1]);
  gw[1] = gw[1] - lw[0] * (cx * w[2]) - lw[2] * (cz * w[0]);
  gw[2] = gw[2] - lw[0] * (cx * w[1]) - lw[1] * (cy * w[0]);
  const T lx = (T)(kArm / kJx), ly = (T)(kArm / kJy), yz = (T)(kYaw / kJz);
  S gf[4];
  gf[0] = g_thrust - lw[1] * ly + lw[2] * yz;
  gf[1] = g_thrust + lw[0] * lx - lw[2] * yz;
  gf[2] = g_thrust + lw[1] * ly + lw[2] * yz;
  gf[3] = g_thrust - lw[0] * lx - lw[2] * yz;
#pragma unroll
  for (int i = 0; i < 4; ++i) gu[i] = gf[i] * ((T)(2 * kThrustCoef) * u[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) gx[i] = cst<S>((T)0);
#pragma unroll
  for (int i = 0; i < 4; ++i) gx[3 + i] = gq[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    gx[7 + i] = gv[i];
    gx[10 + i] = gw[i];
  }
}

// F = x + dt/6 (k1 + 2 k2 + 2 k3 + k4): one classical RK4 step, value only.
template <class S>
__host__ __device__ __forceinline__ void quat_rk4_value(const S x[13], const S u[4], typename Base<S>::type dt,
                                                        S F[13]) {
  typedef typename Base<S>::type T;
  const T cf[4] = {(T)(dt / 6), (T)(dt / 3), (T)(dt / 3), (T)(dt / 6)};
  const T ca[4] = {(T)0, (T)(dt / 2), (T)(dt / 2), dt};
  S z[13], k[13];
#pragma unroll
  for (int i = 0; i < 13; ++i) F[i] = x[i];
  quat_f(x, u, k);
#pragma unroll
  for (int st = 1; st < 4; ++st) {
#pragma unroll
    for (int i = 0; i < 13; ++i) {
      F[i] = F[i] + cf[st - 1] * k[i];
      z[i] = x[i] + ca[st] * k[i];
    }
    quat_f(z, u, k);
  }
#pragma unroll
  for (int i = 0; i < 13; ++i) F[i] = F[i] + cf[3] * k[i];
}

// One RK4 step and the gradient of lam^T F with respect to (x, u), by a reverse
// sweep over the four stage evaluations.  With Dual scalars seeded in one
// direction this also yields the Jacobian column (F.d) and the Hessian-vector
// product of lam^T F (gx.d, gu.d).
template <class S>
__host__ __device__ __forceinline__ void quat_rk4_fwd_rev(const S x[13], const S u[4],
                                                          typename Base<S>::type dt,
                                                          const typename Base<S>::type lam[13], S F[13],
                                                          S gx[13], S gu[4]) {
  typedef typename Base<S>::type T;
  S st_s[4][10];
  S z[13], k[13];
  const T cf[4] = {(T)(dt / 6), (T)(dt / 3), (T)(dt / 3), (T)(dt / 6)};
  const T ca[4] = {(T)0, (T)(dt / 2), (T)(dt / 2), dt};
#pragma unroll
  for (int i = 0; i < 13; ++i) F[i] = x[i];
#pragma unroll
  for (int i = 0; i < 10; ++i) st_s[0][i] = x[3 + i];
  quat_f(x, u, k);
#pragma unroll
  for (int st = 1; st < 4; ++st) {
#pragma unroll
    for (int i = 0; i < 13; ++i) {
      F[i] = F[i] + cf[st - 1] * k[i];
      z[i] = x[i] + ca[st] * k[i];
    }
#pragma unroll
    for (int i = 0; i < 10; ++i) st_s[st][i] = z[3 + i];
    quat_f(z, u, k);
  }
#pragma unroll
  for (int i = 0; i < 13; ++i) F[i] = F[i] + cf[3] * k[i];

  // reverse sweep: w = adjoint of k_st
  S w[13], gzx[13], gzu[4];
#pragma unroll
  for (int i = 0; i < 13; ++i) {
    gx[i] = cst<S>(lam[i]);
    w[i] = cst<S>(cf[3] * lam[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) gu[i] = cst<S>((T)0);
#pragma unroll
  for (int st = 3; st >= 0; --st) {
    quat_vjp(st_s[st], u, w, gzx, gzu);
#pragma unroll
    for (int i = 0; i < 13; ++i) gx[i] = gx[i] + gzx[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] = gu[i] + gzu[i];
    if (st > 0) {
#pragma unroll
      for (int i = 0; i < 13; ++i) w[i] = ca[st] * gzx[i] + cf[st - 1] * lam[i];
    }
  }
}

}  // namespace bipm
