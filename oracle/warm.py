"""Warm-start encodings on the CPU: network input features, training targets,
and the primal starting point decoded from a network output.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The learned warm start proposes a primal starting point for the interior-point
iteration of Sec. IV from a problem's parameters.  It is defined for the
cluttered-environment family: one quadrotor, vertical cylinders, a fixed goal.

Features (12 + 3 K values, K = number of nearest cylinders kept):
    (p0 - g) / 10, v0 / 2, eta0, omega0 / 2             initial state vs goal g
    then for the K cylinders nearest to p0 in the horizontal plane, in order of
    increasing centre distance (ties: lower index first):
        (cx - p0x) / 10, (cy - p0y) / 10, r
    a cylinder whose centre is more than 30 m away, or a rank beyond the
    problem's cylinder count, contributes (0, 0, 0).

Targets / network output (12 (N + 1) + 4 N values), for a trajectory x:
    (x_k - xbar) / S  for k = 0..N, S = (2, 2, 2, 2, 2, 2, .5, .5, .5, 2, 2, 2)
    (u_k - u_hover) / u_hover  for k = 0..N-1

Decoding inverts the target map for k >= 1 (x_0 is xbar: its equality row),
and sets every slack to its inequality value g(x_k) at the decoded state.

Warm starting point: the decoded x pushed inside the bounds with bound push
and bound fraction 1e-3, mu_0 = 1e-2, and bound multipliers centred on the
barrier, z = mu_0 / (distance to the bound); y from least squares as for a
cold start.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from workloads import theta_layout

from . import ipm
from .quadrotor import HOVER

POS_SCALE = 10.0
VEL_SCALE = 2.0
RATE_SCALE = 2.0
CUTOFF = 30.0
STATE_SCALE = np.array([2.0] * 6 + [0.5] * 3 + [2.0] * 3)


def _check_family(desc):
    if desc.nq != 1 or desc.n_sph != 0 or desc.pair_dist > 0:
        raise ValueError("the warm start is defined for one quadrotor among cylinders")


def feature_dim(k_near):
    return 12 + 3 * k_near


def output_dim(desc):
    return 12 * (desc.horizon + 1) + 4 * desc.horizon


def features(desc, theta, k_near=50):
    """Network input of one problem (length 12 + 3 k_near)."""
    _check_family(desc)
    lay = theta_layout(desc)
    th = np.asarray(theta, dtype=np.float64)
    x0 = th[lay["xbar"]:lay["xbar"] + 12]
    goal = th[lay["ref"]:lay["ref"] + 3]
    f = np.zeros(feature_dim(k_near))
    f[0:3] = (x0[0:3] - goal) / POS_SCALE
    f[3:6] = x0[3:6] / VEL_SCALE
    f[6:9] = x0[6:9]
    f[9:12] = x0[9:12] / RATE_SCALE
    cyl = th[lay["cyl"]:lay["cyl"] + 3 * desc.n_cyl].reshape(desc.n_cyl, 3)
    d2 = [((c[0] - x0[0]) ** 2 + (c[1] - x0[1]) ** 2, j) for j, c in enumerate(cyl)]
    for rank, (dist2, j) in enumerate(sorted(d2)[:k_near]):
        if np.sqrt(dist2) <= CUTOFF:
            cx, cy, r = cyl[j]
            f[12 + 3 * rank:15 + 3 * rank] = ((cx - x0[0]) / POS_SCALE, (cy - x0[1]) / POS_SCALE, r)
    return f


def _split(desc, x):
    N, nx, nu, ni = desc.horizon, desc.nx, desc.nu, desc.ni
    xs, us, ss, pos = [], [], [], 0
    for k in range(N + 1):
        xs.append(slice(pos, pos + nx)); pos += nx
        if k < N:
            us.append(slice(pos, pos + nu)); pos += nu
        if k >= 1:
            ss.append(slice(pos, pos + ni)); pos += ni
    return xs, us, ss


def encode(desc, theta, x):
    """Training target of one solved trajectory x (length n)."""
    _check_family(desc)
    lay = theta_layout(desc)
    xbar = np.asarray(theta, dtype=np.float64)[lay["xbar"]:lay["xbar"] + 12]
    xs, us, _ = _split(desc, np.asarray(x))
    N = desc.horizon
    o = np.zeros(output_dim(desc))
    for k in range(N + 1):
        o[12 * k:12 * k + 12] = (x[xs[k]] - xbar) / STATE_SCALE
    base = 12 * (N + 1)
    for k in range(N):
        o[base + 4 * k:base + 4 * k + 4] = (x[us[k]] - HOVER) / HOVER
    return o


def decode(desc, theta, out, ineq):
    """Primal starting point (length n) from a network output.

    `ineq(states)` evaluates the inequality functions g of the problem at the
    stacked states (K, 12) -> (K, ni); the slacks start at those values."""
    _check_family(desc)
    lay = theta_layout(desc)
    xbar = np.asarray(theta, dtype=np.float64)[lay["xbar"]:lay["xbar"] + 12]
    out = np.asarray(out, dtype=np.float64)
    N = desc.horizon
    x = np.zeros(desc.n)
    xs, us, ss = _split(desc, x)
    states = np.zeros((N + 1, 12))
    for k in range(N + 1):
        states[k] = xbar if k == 0 else xbar + STATE_SCALE * out[12 * k:12 * k + 12]
        x[xs[k]] = states[k]
    base = 12 * (N + 1)
    for k in range(N):
        x[us[k]] = HOVER * (1.0 + out[base + 4 * k:base + 4 * k + 4])
    if desc.ni:
        g = np.asarray(ineq(states[1:]))
        for k in range(1, N + 1):
            x[ss[k - 1]] = g[k - 1]
    return x


def warm_options(**kw):
    """Solver options of a warm start (mu_0 1e-2, bound push 1e-3, centred z)."""
    base = dict(mu_init=1e-2, bound_push=1e-3, bound_frac=1e-3, z_centred=True)
    base.update(kw)
    return dataclasses.replace(ipm.Options(), **base)
