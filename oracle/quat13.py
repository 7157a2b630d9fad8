"""The 13-state quaternion quadrotor of Sec. VI as plain NLPs of the form of Eq. 1
(oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. VI fixes the model's shape, not its constants: each quadrotor's state stacks
position, attitude quaternion, and body linear and angular velocities (13
numbers), its inputs are the four rotor angular velocities, the dynamics are the
standard rigid-body kinematics, and the NMPC runs at dt = 0.1 s over a horizon of
30.  The readings taken here, beside those of the 12-state model
(`oracle/quadrotor.py`, whose mass, inertia, arm length, torque ratio, cost
structure, inequality rows and variable order carry over):

* x = (p, q, v, w) per quadrotor: p the world position, q = (q_w, q_x, q_y, q_z)
  the attitude quaternion (body to world, Hamilton product), v the body-frame
  linear velocity, w the body rates; u = (Omega_1..Omega_4) rotor speeds in
  rad/s, "+" layout as in the 12-state model;
* rotor i gives thrust f_i = K_F Omega_i^2 along the body z axis and the
  reaction torque about that axis of the 12-state model, KAPPA (f_1 - f_2 + f_3
  - f_4); K_F = m g / (4 Omega_h^2) with the hover speed Omega_h = 400 rad/s; the
  speeds are bounded to [0, sqrt(2) Omega_h], the 12-state thrust range
  [0, 2 m g / 4];
* p' = R(q) v,  q' = q (x) (0, w) / 2,  v' = (T / m) e3 - w x v - g R(q)^T e3,
  w' = J^-1 (tau - w x J w), with T = sum f_i, R(q) the rotation matrix of the
  unit-quaternion formula (q is not renormalised: RK4 keeps |q| = 1 to its own
  order);
* one classical RK4 step per interval;
* cost sum_{k<N} |x_k - r_k|_Q^2 + |u_k - Omega_h|_R^2 + |x_N - r_N|_{Q_N}^2 with
  Q = diag(10 I3, I4, I3, 0.1 I3), r_k = (p_ref(t_k), (1, 0, 0, 0), v_ref(t_k), 0)
  (the reference velocity read in the body frame, which is the world frame at
  level attitude and zero yaw), R = 0.1 (2 K_F Omega_h)^2 I4 (the 12-state input
  weight carried through dT/dOmega at hover), Q_N = 10 Q.

parity unpinned: nothing on the CUDA path computes this model yet; the pins of
tests/test_oracle_quat13.py fix it against closed forms and against the 12-state
model.
"""

from __future__ import annotations

import math

import torch

from .quadrotor import ARM, F64, GRAV, HOVER, INERTIA, KAPPA, MASS, QuadNLP

OMEGA_H = 400.0
K_F = HOVER / OMEGA_H ** 2
OMEGA_MAX = math.sqrt(2.0) * OMEGA_H
Q13_DIAG = (10.0,) * 3 + (1.0,) * 4 + (1.0,) * 3 + (0.1,) * 3
R13 = 0.1 * (2.0 * K_F * OMEGA_H) ** 2


def rot(q):
    """Rotation matrix (..., 3, 3) of the quaternions q = (w, x, y, z) (..., 4)."""
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    r = [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
         [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
         [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]
    return torch.stack([torch.stack(row, dim=-1) for row in r], dim=-2)


def quat_mul(a, b):
    """Hamilton product a (x) b of quaternions (..., 4)."""
    aw, av = a[..., 0:1], a[..., 1:4]
    bw, bv = b[..., 0:1], b[..., 1:4]
    w = aw * bw - (av * bv).sum(-1, keepdim=True)
    v = aw * bv + bw * av + torch.cross(av, bv, dim=-1)
    return torch.cat([w, v], dim=-1)


def quat13_rhs(x, u):
    """Continuous-time dynamics of the 13-state model, batched over leading dims."""
    q = x[..., 3:7]
    v = x[..., 7:10]
    w = x[..., 10:13]
    f = K_F * u ** 2
    thrust = f.sum(-1)
    R = rot(q)
    pd = (R @ v.unsqueeze(-1)).squeeze(-1)
    qd = 0.5 * quat_mul(q, torch.cat([torch.zeros_like(w[..., 0:1]), w], dim=-1))
    e3 = torch.tensor([0.0, 0.0, 1.0], dtype=x.dtype)
    g_body = R[..., 2, :]  # R(q)^T e3: the world vertical in the body frame
    vd = (thrust / MASS).unsqueeze(-1) * e3 - torch.cross(w, v, dim=-1) - GRAV * g_body
    J = torch.tensor(INERTIA, dtype=x.dtype)
    tau = torch.stack([ARM * (f[..., 1] - f[..., 3]),
                       ARM * (f[..., 2] - f[..., 0]),
                       KAPPA * (f[..., 0] - f[..., 1] + f[..., 2] - f[..., 3])], dim=-1)
    wd = (tau - torch.cross(w, J * w, dim=-1)) / J
    return torch.cat([pd, qd, vd, wd], dim=-1)


class QuatNLP(QuadNLP):
    """One NMPC instance of the 13-state model as a plain NLP; structure, cost form,
    inequalities and orders as QuadNLP (desc: a workloads.QuatProblemDesc)."""

    NXQ = 13
    U_LO, U_HI = 0.0, OMEGA_MAX

    @staticmethod
    def rhs(x, u):
        return quat13_rhs(x, u)

    def reference(self):
        p, v = self.reference_circles()
        r = torch.zeros(self.N + 1, self.nq, 13, dtype=F64)
        r[..., 0:3] = p
        r[..., 3] = 1.0
        r[..., 7:10] = v
        return r

    def weights(self):
        return (torch.tensor(Q13_DIAG, dtype=F64).repeat(self.nq),
                torch.full((self.nu,), R13, dtype=F64),
                torch.full((self.nu,), OMEGA_H, dtype=F64))
