"""Quadrotor NMPC problems as plain NLPs of the form of Eq. 1 (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's problem class (Sec. III, Eq. 1) is min f(x) s.t. c(x) = 0,
x_L <= x <= x_U, with inequalities written through slack variables.  Its
experiments use quadrotor NMPC (Sec. VI).  The model and weights the paper
leaves open are fixed by these readings:

* state per quadrotor (p, v, eta = ZYX Euler angles (phi, theta, psi), omega
  body rates), input = four rotor thrusts in N; "+" rotor layout;
  m = 0.5 kg, g = 9.81, J = diag(2.32e-3, 2.32e-3, 4.00e-3), arm L = 0.175 m,
  drag-torque coefficient kappa = 0.01 m; thrust bounds [0, 2 * m g / 4];
* one classical RK4 step per interval (multiple shooting), N intervals;
* cost sum_{k<N} |x_k - r_k|_Q^2 + |u_k - u_hover|_R^2 + |x_N - r_N|_{Q_N}^2 with
  Q = diag(10 I3, I3, I3, 0.1 I3), R = 0.1 I4, Q_N = 10 Q (no factor 1/2);
* inequalities at stages 1..N, squared-distance form g(x) - s = 0, s >= 0:
  spheres |p_i - c|^2 - r^2, cylinders (p_ix - cx)^2 + (p_iy - cy)^2 - r^2,
  moving spheres |p_i - (c + v k dt)|^2 - r^2 at stage k (time-varying
  obstacles with known trajectories, Sec. VI), pairs |p_i - p_j|^2 - d^2;
  order: spheres, cylinders, moving spheres (each quad-major), then pairs
  (i < j, lexicographic);
* variable order: for k = 0..N: x_k, then u_k (k < N), then s_k (k >= 1);
  equality order: x_0 - xbar, then for k = 0..N-1 the dynamics rows
  x_{k+1} - F(x_k, u_k) followed by the stage-(k+1) inequality rows.
"""

from __future__ import annotations

import numpy as np
import torch

from workloads import ProblemDesc, theta_layout

F64 = torch.float64

MASS = 0.5
GRAV = 9.81
INERTIA = (2.32e-3, 2.32e-3, 4.00e-3)
ARM = 0.175
KAPPA = 0.01
HOVER = MASS * GRAV / 4.0
U_MAX = 2.0 * HOVER
Q_DIAG = (10.0,) * 3 + (1.0,) * 3 + (1.0,) * 3 + (0.1,) * 3
R_DIAG = (0.1,) * 4
QN_SCALE = 10.0


def quad_rhs(x, u):
    """Continuous-time rigid-body quadrotor dynamics, batched over leading dims."""
    v = x[..., 3:6]
    phi, th, psi = x[..., 6], x[..., 7], x[..., 8]
    w1, w2, w3 = x[..., 9], x[..., 10], x[..., 11]
    thrust = u.sum(-1)
    cph, sph = torch.cos(phi), torch.sin(phi)
    cth, sth = torch.cos(th), torch.sin(th)
    cps, sps = torch.cos(psi), torch.sin(psi)
    # acceleration = R(eta) e3 * T / m - g e3, R = Rz(psi) Ry(theta) Rx(phi)
    ax = (cps * sth * cph + sps * sph) * thrust / MASS
    ay = (sps * sth * cph - cps * sph) * thrust / MASS
    az = cth * cph * thrust / MASS - GRAV
    # Euler-angle rates from body rates
    phid = w1 + sph * torch.tan(th) * w2 + cph * torch.tan(th) * w3
    thd = cph * w2 - sph * w3
    psid = (sph * w2 + cph * w3) / cth
    # body torques of the "+" layout and Euler's rotation equations
    jx, jy, jz = INERTIA
    tx = ARM * (u[..., 1] - u[..., 3])
    ty = ARM * (u[..., 2] - u[..., 0])
    tz = KAPPA * (u[..., 0] - u[..., 1] + u[..., 2] - u[..., 3])
    w1d = (tx - (w2 * (jz * w3) - w3 * (jy * w2))) / jx
    w2d = (ty - (w3 * (jx * w1) - w1 * (jz * w3))) / jy
    w3d = (tz - (w1 * (jy * w2) - w2 * (jx * w1))) / jz
    return torch.stack([v[..., 0], v[..., 1], v[..., 2], ax, ay, az,
                        phid, thd, psid, w1d, w2d, w3d], dim=-1)


def rk4(x, u, dt, rhs=quad_rhs):
    """One classical fourth-order Runge-Kutta step of x' = rhs(x, u)."""
    k1 = rhs(x, u)
    k2 = rhs(x + 0.5 * dt * k1, u)
    k3 = rhs(x + 0.5 * dt * k2, u)
    k4 = rhs(x + dt * k3, u)
    return x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


class QuadNLP:
    """One quadrotor NMPC instance as a plain NLP (n variables, m equalities)."""

    # per-quadrotor state size, continuous dynamics and input bounds of the model
    NXQ = 12
    U_LO, U_HI = 0.0, U_MAX

    @staticmethod
    def rhs(x, u):
        return quad_rhs(x, u)

    def __init__(self, desc: ProblemDesc, theta: np.ndarray):
        self.desc = desc
        d = desc
        self.nq, self.N, self.dt = d.nq, d.horizon, d.dt
        self.nx, self.nu, self.ni = d.nx, d.nu, d.ni
        self.n, self.m = d.n, d.m
        self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float64))
        lay = theta_layout(d)
        th = self.theta
        self.xbar = th[lay["xbar"]:lay["xbar"] + self.nx]
        self.ref = th[lay["ref"]:lay["ref"] + 6 * self.nq].reshape(self.nq, 6)
        self.sph = th[lay["sph"]:lay["sph"] + 4 * d.n_sph].reshape(d.n_sph, 4)
        self.cyl = th[lay["cyl"]:lay["cyl"] + 3 * d.n_cyl].reshape(d.n_cyl, 3)
        self.mov = th[lay["mov"]:lay["mov"] + 7 * d.n_mov].reshape(d.n_mov, 7)
        self.pairs = [(i, j) for i in range(self.nq) for j in range(i + 1, self.nq)] \
            if d.pair_dist > 0 else []

        # index maps into the decision vector
        xi, ui, si = [], [], []
        pos = 0
        for k in range(self.N + 1):
            xi.append(np.arange(pos, pos + self.nx)); pos += self.nx
            if k < self.N:
                ui.append(np.arange(pos, pos + self.nu)); pos += self.nu
            if k >= 1:
                si.append(np.arange(pos, pos + self.ni)); pos += self.ni
        assert pos == self.n
        self.xi = torch.as_tensor(np.stack(xi))
        self.ui = torch.as_tensor(np.stack(ui))
        self.si = torch.as_tensor(np.stack(si)) if self.ni > 0 else torch.zeros((self.N, 0), dtype=torch.long)

        self.xl = np.full(self.n, -np.inf)
        self.xu = np.full(self.n, np.inf)
        self.xl[self.ui.numpy().ravel()] = self.U_LO
        self.xu[self.ui.numpy().ravel()] = self.U_HI
        if self.ni > 0:
            self.xl[self.si.numpy().ravel()] = 0.0

        self.xref = self.reference().reshape(self.N + 1, self.nx)
        self.qw, self.rw, self.uh = self.weights()

    def reference_circles(self):
        """Position and velocity (N + 1, nq, 3) of every quadrotor's reference circle
        at the stage times."""
        t = torch.arange(self.N + 1, dtype=torch.float64) * self.dt
        p = torch.zeros(self.N + 1, self.nq, 3, dtype=F64)
        v = torch.zeros(self.N + 1, self.nq, 3, dtype=F64)
        for i in range(self.nq):
            cx, cy, cz, rad, rate, ph = self.ref[i]
            a = rate * t + ph
            p[:, i, 0] = cx + rad * torch.cos(a)
            p[:, i, 1] = cy + rad * torch.sin(a)
            p[:, i, 2] = cz
            v[:, i, 0] = -rad * rate * torch.sin(a)
            v[:, i, 1] = rad * rate * torch.cos(a)
        return p, v

    def reference(self):
        """Reference states (N + 1, nq, 12): the circle's position and velocity, zero
        attitude and rates."""
        p, v = self.reference_circles()
        r = torch.zeros(self.N + 1, self.nq, 12, dtype=F64)
        r[..., 0:3] = p
        r[..., 3:6] = v
        return r

    def weights(self):
        """State weights (nx), input weights (nu) and the input reference (nu)."""
        return (torch.tensor(Q_DIAG, dtype=F64).repeat(self.nq),
                torch.tensor(R_DIAG, dtype=F64).repeat(self.nq),
                torch.full((self.nu,), HOVER, dtype=F64))

    # ------------------------------------------------------------ functions
    def split(self, w):
        return w[self.xi], w[self.ui], w[self.si]

    def ineq(self, xs, ks=None):
        """Inequality values g(x_k) for the given stacked states (K, nx) -> (K, ni);
        ks are the stage indices of the rows (default 1..K: the states x_1..x_N),
        which place the moving spheres at time k dt."""
        p = xs.reshape(xs.shape[0], self.nq, self.NXQ)[..., 0:3]
        if ks is None:
            ks = torch.arange(1, xs.shape[0] + 1, dtype=F64)
        t = torch.as_tensor(ks, dtype=F64).reshape(-1) * self.dt
        out = []
        for i in range(self.nq):
            for j in range(self.sph.shape[0]):
                c, rad = self.sph[j, 0:3], self.sph[j, 3]
                out.append(((p[:, i] - c) ** 2).sum(-1) - rad ** 2)
        for i in range(self.nq):
            for j in range(self.cyl.shape[0]):
                cx, cy, rad = self.cyl[j]
                out.append((p[:, i, 0] - cx) ** 2 + (p[:, i, 1] - cy) ** 2 - rad ** 2)
        for i in range(self.nq):
            for j in range(self.mov.shape[0]):
                c0, rad, v = self.mov[j, 0:3], self.mov[j, 3], self.mov[j, 4:7]
                cen = c0 + t.reshape(-1, 1) * v          # centre at each row's stage time
                out.append(((p[:, i] - cen) ** 2).sum(-1) - rad ** 2)
        dd = self.desc.pair_dist
        for (i, j) in self.pairs:
            out.append(((p[:, i] - p[:, j]) ** 2).sum(-1) - dd ** 2)
        if not out:
            return torch.zeros(xs.shape[0], 0, dtype=F64)
        return torch.stack(out, dim=-1)

    def f_t(self, w):
        x, u, _ = self.split(w)
        ex = x - self.xref
        eu = u - self.uh
        stage = (self.qw * ex[:-1] ** 2).sum() + (self.rw * eu ** 2).sum()
        term = QN_SCALE * (self.qw * ex[-1] ** 2).sum()
        return stage + term

    def step_t(self, x, u):
        """Discrete dynamics F(x_k, u_k) for stacked (K, nx), (K, nu)."""
        xq = x.reshape(x.shape[0], self.nq, self.NXQ)
        uq = u.reshape(u.shape[0], self.nq, 4)
        return rk4(xq, uq, self.dt, self.rhs).reshape(x.shape[0], self.nx)

    def c_t(self, w):
        x, u, s = self.split(w)
        rows = [x[0] - self.xbar]
        fx = self.step_t(x[:-1], u)
        g = self.ineq(x[1:])
        for k in range(self.N):
            rows.append(x[k + 1] - fx[k])
            rows.append(g[k] - s[k])
        return torch.cat(rows)

    # ------------------------------------------------ NLP interface (numpy)
    def f(self, w):
        return float(self.f_t(torch.as_tensor(w)))

    def c(self, w):
        return self.c_t(torch.as_tensor(w)).numpy()

    def grad_f(self, w):
        return torch.func.grad(self.f_t)(torch.as_tensor(w)).numpy()

    # Derivatives.  c and the Lagrangian are sums of per-stage terms: the dynamics
    # row block of interval k depends only on (x_k, u_k, x_{k+1}), an inequality
    # block only on (x_k, s_k), the objective is a sum of stage costs.  The
    # Jacobian and the Lagrangian Hessian (Eq. 4) are therefore assembled from
    # autograd derivatives of these stage functions (vectorised over stages);
    # jac_c_whole / hess_lag_whole differentiate the whole decision vector at
    # once and serve as the check of the assembly.
    def _dyn(self, z):
        """F(x_k, u_k) of one interval from z = (x_k, u_k)."""
        x = z[:self.nx].reshape(self.nq, self.NXQ)
        u = z[self.nx:].reshape(self.nq, 4)
        return rk4(x, u, self.dt, self.rhs).reshape(self.nx)

    def _ineq1(self, xk, k):
        return self.ineq(xk.reshape(1, -1), k.reshape(1))[0]

    def _stage_cost(self, z, r):
        """Cost of interval k < N from z = (x_k, u_k) and the reference r = x^ref_k."""
        ex = z[:self.nx] - r
        eu = z[self.nx:] - self.uh
        return (self.qw * ex ** 2).sum() + (self.rw * eu ** 2).sum()

    def _term_cost(self, x, r):
        return QN_SCALE * (self.qw * (x - r) ** 2).sum()

    def jac_c(self, w):
        """Constraint Jacobian, assembled from the stage Jacobians."""
        wt = torch.as_tensor(w)
        x, u, _ = self.split(wt)
        nx, ni, N = self.nx, self.ni, self.N
        xi, ui, si = self.xi.numpy(), self.ui.numpy(), self.si.numpy()
        J = np.zeros((self.m, self.n))
        J[np.arange(nx), xi[0]] = 1.0
        Z = torch.cat([x[:-1], u], dim=1)
        Jd = torch.func.vmap(torch.func.jacfwd(self._dyn))(Z).numpy()
        ks = torch.arange(1, N + 1, dtype=F64)
        Jg = torch.func.vmap(torch.func.jacfwd(self._ineq1))(x[1:], ks).numpy() if ni else None
        row = nx
        for k in range(N):
            J[row:row + nx][:, np.concatenate([xi[k], ui[k]])] = -Jd[k]
            J[np.arange(row, row + nx), xi[k + 1]] = 1.0
            row += nx
            if ni:
                J[row:row + ni][:, xi[k + 1]] = Jg[k]
                J[np.arange(row, row + ni), si[k]] = -1.0
                row += ni
        return J

    def hess_lag(self, w, y, obj_factor=1.0):
        """obj_factor * Hess f + sum_i y_i Hess c_i (Hessian of the Lagrangian, Eq. 4),
        assembled from the stage Hessians."""
        wt = torch.as_tensor(w)
        yt = torch.as_tensor(np.asarray(y, dtype=np.float64))
        x, u, _ = self.split(wt)
        nx, ni, N = self.nx, self.ni, self.N
        xi, ui = self.xi.numpy(), self.ui.numpy()
        blk = nx + ni
        # multipliers of the dynamics rows x_{k+1} - F(z_k) and of the rows g(x_{k+1}) - s
        ydyn = torch.stack([yt[nx + k * blk: nx + k * blk + nx] for k in range(N)])
        Z = torch.cat([x[:-1], u], dim=1)
        Hd = torch.func.vmap(torch.func.hessian(lambda z, lam: -(lam * self._dyn(z)).sum()))(Z, ydyn).numpy()
        if obj_factor != 0.0:
            Hc = torch.func.vmap(torch.func.hessian(self._stage_cost))(Z, self.xref[:-1]).numpy()
            Ht = torch.func.hessian(self._term_cost)(x[-1], self.xref[-1]).numpy()
        H = np.zeros((self.n, self.n))
        for k in range(N):
            idx = np.concatenate([xi[k], ui[k]])
            blkH = Hd[k] + (obj_factor * Hc[k] if obj_factor != 0.0 else 0.0)
            H[np.ix_(idx, idx)] += blkH
        if obj_factor != 0.0:
            H[np.ix_(xi[N], xi[N])] += obj_factor * Ht
        if ni:
            yin = torch.stack([yt[nx + k * blk + nx: nx + (k + 1) * blk] for k in range(N)])
            ks = torch.arange(1, N + 1, dtype=F64)
            Hg = torch.func.vmap(torch.func.hessian(lambda xk, lam, k: (lam * self._ineq1(xk, k)).sum()))(
                x[1:], yin, ks).numpy()
            for k in range(N):
                H[np.ix_(xi[k + 1], xi[k + 1])] += Hg[k]
        return H

    def jac_c_whole(self, w):
        return torch.func.jacfwd(self.c_t)(torch.as_tensor(w)).numpy()

    def hess_lag_whole(self, w, y, obj_factor=1.0):
        yt = torch.as_tensor(y)

        def lag(wt):
            return obj_factor * self.f_t(wt) + (yt * self.c_t(wt)).sum()

        return torch.func.hessian(lag)(torch.as_tensor(w)).numpy()

    def default_start(self):
        """Default primal guess: every state at xbar, inputs at their reference (hover),
        slacks at g(xbar)."""
        w = torch.zeros(self.n, dtype=F64)
        w[self.xi] = self.xbar
        w[self.ui] = self.uh
        if self.ni > 0:
            # g(xbar) at every stage (moving spheres sit at each stage's time)
            w[self.si] = self.ineq(self.xbar.reshape(1, -1).repeat(self.N, 1))
        return w.numpy()
