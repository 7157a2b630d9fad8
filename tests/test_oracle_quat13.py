"""Pins of the oracle's 13-state quaternion quadrotor (oracle/quat13.py, Sec. VI).

The model is fixed against things outside itself: the 12-state Euler-angle model
(pinned in test_oracle_model.py) describes the same rigid body, so at one
physical state the two must give the same world velocity, world acceleration,
body angular acceleration and attitude rate; free fall and a torque-free spin
about a principal axis have closed forms; hover is an equilibrium; the
quaternion derivative is orthogonal to the quaternion.  The NLP built on it is
checked against finite differences and against whole-vector autograd, and on a
problem whose optimum is known (hover at the goal).
"""

import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import ipm
from oracle.quadrotor import GRAV, U_MAX, quad_rhs, rk4
from oracle.quat13 import K_F, OMEGA_H, OMEGA_MAX, QuatNLP, quat13_rhs, rot
from workloads import QuatProblemDesc, make_batch, theta_layout

F64 = torch.float64


def euler_to_quat(eta):
    """Quaternion of the ZYX Euler angles (phi, theta, psi): q_z(psi) q_y(theta) q_x(phi),
    written out from the half-angle products."""
    phi, th, psi = eta[..., 0] / 2, eta[..., 1] / 2, eta[..., 2] / 2
    cf, sf, ct, st, cp, sp = torch.cos(phi), torch.sin(phi), torch.cos(th), torch.sin(th), torch.cos(psi), torch.sin(psi)
    return torch.stack([cp * ct * cf + sp * st * sf,
                        cp * ct * sf - sp * st * cf,
                        cp * st * cf + sp * ct * sf,
                        sp * ct * cf - cp * st * sf], dim=-1)


def euler_rot(eta):
    """R = Rz(psi) Ry(theta) Rx(phi) from the elementary rotations."""
    phi, th, psi = eta
    rx = torch.tensor([[1, 0, 0], [0, math.cos(phi), -math.sin(phi)], [0, math.sin(phi), math.cos(phi)]], dtype=F64)
    ry = torch.tensor([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]], dtype=F64)
    rz = torch.tensor([[math.cos(psi), -math.sin(psi), 0], [math.sin(psi), math.cos(psi), 0], [0, 0, 1]], dtype=F64)
    return rz @ ry @ rx


def random_physical_state(rng):
    eta = torch.tensor([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(-3, 3)], dtype=F64)
    p = torch.tensor(rng.uniform(-2, 2, 3), dtype=F64)
    v_world = torch.tensor(rng.uniform(-2, 2, 3), dtype=F64)
    w = torch.tensor(rng.uniform(-1.5, 1.5, 3), dtype=F64)
    f = torch.tensor(rng.uniform(0.0, U_MAX, 4), dtype=F64)
    return eta, p, v_world, w, f


def test_rotation_of_the_euler_quaternion_is_the_euler_rotation():
    rng = np.random.default_rng(3)
    for _ in range(20):
        eta = random_physical_state(rng)[0]
        q = euler_to_quat(eta)
        assert abs(float(q.norm()) - 1.0) < 1e-15
        assert torch.allclose(rot(q), euler_rot(eta.tolist()), atol=1e-15, rtol=0)


def test_hover_is_an_equilibrium_at_every_yaw():
    for psi in (0.0, 0.7, -2.5):
        q = torch.tensor([math.cos(psi / 2), 0, 0, math.sin(psi / 2)], dtype=F64)
        x = torch.cat([torch.tensor([1.0, -2.0, 3.0], dtype=F64), q, torch.zeros(6, dtype=F64)])
        xd = quat13_rhs(x, torch.full((4,), OMEGA_H, dtype=F64))
        assert float(xd.abs().max()) < 1e-14


def test_matches_the_12_state_model_at_the_same_physical_state():
    """World velocity R v_b, world acceleration R (v_b' + w x v_b), body angular
    acceleration and the attitude rate dq/deta * eta' of the 12-state model agree."""
    rng = np.random.default_rng(7)
    for _ in range(25):
        eta, p, v_world, w, f = random_physical_state(rng)
        x12 = torch.cat([p, v_world, eta, w])
        d12 = quad_rhs(x12, f)
        q = euler_to_quat(eta)
        R = rot(q)
        v_b = R.T @ v_world
        omega = torch.sqrt(f / K_F)
        d13 = quat13_rhs(torch.cat([p, q, v_b, w]), omega)
        assert torch.allclose(d13[0:3], v_world, atol=1e-13, rtol=0)
        acc_world = R @ (d13[7:10] + torch.cross(w, v_b, dim=0))
        assert torch.allclose(acc_world, d12[3:6], atol=1e-12, rtol=0)
        assert torch.allclose(d13[10:13], d12[9:12], atol=1e-10, rtol=1e-13)
        _, qdot = torch.func.jvp(euler_to_quat, (eta,), (d12[6:9],))
        assert torch.allclose(d13[3:7], qdot, atol=1e-13, rtol=0)


def test_quaternion_rate_is_orthogonal_to_the_quaternion():
    rng = np.random.default_rng(11)
    for _ in range(20):
        x = torch.tensor(rng.uniform(-1, 1, 13), dtype=F64)  # q not normalised on purpose
        u = torch.tensor(rng.uniform(0, OMEGA_MAX, 4), dtype=F64)
        d = quat13_rhs(x, u)
        assert abs(float(x[3:7] @ d[3:7])) < 1e-15


def test_free_fall_step_is_the_closed_form():
    """No thrust, no rotation: p(t) = p0 + R v0 t - g t^2 e3 / 2 in the world frame,
    v(t) = v0 - g t R^T e3 in the body frame; RK4 integrates this quadratic motion
    exactly."""
    rng = np.random.default_rng(5)
    dt = 0.1
    for _ in range(10):
        eta, p, v_world, _, _ = random_physical_state(rng)
        q = euler_to_quat(eta)
        R = rot(q)
        v0 = R.T @ v_world
        x0 = torch.cat([p, q, v0, torch.zeros(3, dtype=F64)])
        x1 = rk4(x0, torch.zeros(4, dtype=F64), dt, quat13_rhs)
        e3 = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
        assert torch.allclose(x1[0:3], p + R @ v0 * dt - 0.5 * GRAV * dt * dt * e3, atol=1e-14, rtol=0)
        assert torch.allclose(x1[3:7], q, atol=1e-16, rtol=0)
        assert torch.allclose(x1[7:10], v0 - GRAV * dt * (R.T @ e3), atol=1e-14, rtol=0)


@pytest.mark.parametrize("axis", [0, 2])
def test_torque_free_spin_about_a_principal_axis(axis):
    """A constant body rate w about principal axis a (no torque: rotors at rest, and
    w x J w = 0) turns q into q0 (x) (cos(|w| t / 2), sin(|w| t / 2) e_a); RK4's
    local error is fifth order, so halving the step cuts it about 32-fold."""
    q0 = euler_to_quat(torch.tensor([0.3, -0.2, 1.1], dtype=F64))
    rate = 2.0
    w = torch.zeros(3, dtype=F64)
    w[axis] = rate

    def err(dt):
        x0 = torch.cat([torch.zeros(3, dtype=F64), q0, torch.zeros(3, dtype=F64), w])
        x1 = rk4(x0, torch.zeros(4, dtype=F64), dt, quat13_rhs)
        ang = rate * dt / 2
        e = torch.zeros(4, dtype=F64)
        e[0] = math.cos(ang)
        e[1 + axis] = math.sin(ang)
        a, b = q0, e
        exact = torch.cat([a[0:1] * b[0:1] - (a[1:] * b[1:]).sum(0, keepdim=True),
                           a[0] * b[1:] + b[0] * a[1:] + torch.cross(a[1:], b[1:], dim=0)])
        assert torch.allclose(x1[10:13], w, atol=1e-15, rtol=0)
        return float((x1[3:7] - exact).abs().max())

    e1, e2 = err(0.1), err(0.05)
    assert e1 < 1e-6
    assert 20.0 < e1 / e2 < 45.0


def _small(horizon, **kw):
    desc = dataclasses.replace(make_batch("track_quat", 1)[0], horizon=horizon, **kw)
    _, th = make_batch("track_quat", 2, desc=desc)
    return desc, th


def test_stage_assembly_matches_whole_vector_derivatives():
    desc, th = _small(5)
    nlp = QuatNLP(desc, th[1])
    w = nlp.default_start() + 0.01 * np.random.default_rng(0).standard_normal(nlp.n)
    y = np.random.default_rng(1).standard_normal(nlp.m)
    assert np.abs(nlp.jac_c(w) - nlp.jac_c_whole(w)).max() < 1e-12
    assert np.abs(nlp.hess_lag(w, y) - nlp.hess_lag_whole(w, y)).max() < 1e-9


def test_constraint_jacobian_matches_finite_differences():
    desc, th = _small(3)
    nlp = QuatNLP(desc, th[0])
    rng = np.random.default_rng(2)
    w = nlp.default_start() + 0.05 * rng.standard_normal(nlp.n)
    J = nlp.jac_c(w)
    h = 1e-6
    for j in rng.choice(nlp.n, 25, replace=False):
        e = np.zeros(nlp.n)
        e[j] = h
        fd = (nlp.c(w + e) - nlp.c(w - e)) / (2 * h)
        assert np.abs(fd - J[:, j]).max() <= 1e-6 * max(1.0, np.abs(J[:, j]).max())


def test_hover_at_the_goal_is_the_optimum():
    """Start in hover at a fixed goal (reference radius 0) with no obstacle: staying
    there at the hover speed costs nothing and satisfies every constraint."""
    desc = QuatProblemDesc(nq=1, horizon=6, dt=0.1)
    lay = theta_layout(desc)
    th = np.zeros(lay["end"])
    goal = np.array([1.0, -0.5, 2.0])
    th[lay["xbar"]:lay["xbar"] + 3] = goal
    th[lay["xbar"] + 3] = 1.0
    th[lay["ref"]:lay["ref"] + 3] = goal
    nlp = QuatNLP(desc, th)
    st, _ = ipm.solve(nlp)
    assert st.status == ipm.CONVERGED
    x = st.normal.x
    assert nlp.f(x) < 1e-10
    assert np.abs(x[nlp.ui.numpy().ravel()] - OMEGA_H).max() < 1e-5
    assert np.abs(x[nlp.xi.numpy()][:, 0:3] - goal).max() < 1e-7


def test_tracking_problem_converges():
    desc, th = _small(10)
    nlp = QuatNLP(desc, th[0])
    st, _ = ipm.solve(nlp)
    m = ipm.final_metrics(nlp, st)
    assert st.status == ipm.CONVERGED
    assert m["kkt"] <= 1e-6 and m["inf"] <= 1e-6


def test_workload_start_is_the_tracking_start_in_the_quaternion_layout():
    desc_q, th_q = make_batch("track_quat", 3)
    d12 = dataclasses.replace(make_batch("track", 1)[0], horizon=desc_q.horizon, dt=desc_q.dt)
    from workloads.quadrotor import _track, problem_stream

    lq, l12 = theta_layout(desc_q), theta_layout(d12)
    for j in range(3):
        t12 = _track(problem_stream(1009, j), d12)
        x = th_q[j, lq["xbar"]:lq["xbar"] + 13]
        assert np.array_equal(x[0:3], t12[0:3]) and np.array_equal(x[7:10], t12[3:6])
        assert np.array_equal(x[3:7], [1.0, 0.0, 0.0, 0.0]) and np.array_equal(x[10:13], [0.0, 0.0, 0.0])
        assert np.array_equal(th_q[j, lq["ref"]:], t12[l12["ref"]:])


def test_the_library_rejects_the_quaternion_model():
    from paper_2606_26341_gb300.bipm import desc_c

    with pytest.raises(ValueError, match="12-state"):
        desc_c(make_batch("track_quat", 1)[0])


def test_stored_quaternion_outcomes_are_reproduced():
    """tests/golden/track_quat_oracle.json (written by make_track_quat.py, the
    oracle only): the oracle reproduces the stored status and iteration count of
    the first two problems, and their solutions to 1e-9."""
    import json
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "track_quat_oracle.json")
    with open(path) as fh:
        golden = json.load(fh)
    desc, theta = make_batch("track_quat", 2)
    for j in range(2):
        nlp = QuatNLP(desc, theta[j])
        st, _ = ipm.solve(nlp)
        assert st.status == golden["status"][j] and st.iter == golden["iters"][j]
        x = np.asarray(golden["x"][j])
        assert np.abs(st.normal.x - x).max() <= 1e-9 * max(1.0, np.abs(x).max())


def _lqr_rollout(A, B, Q, R, QN, x0, N):
    """Finite-horizon discrete LQR (textbook backward Riccati recursion) and its rollout."""
    P = QN
    Ks = []
    for _ in range(N):
        K = -np.linalg.solve(R + B.T @ P @ B, B.T @ P @ A)
        P = Q + A.T @ P @ A + A.T @ P @ B @ K
        Ks.append(K)
    Ks = Ks[::-1]
    xs, us = [x0], []
    for k in range(N):
        us.append(Ks[k] @ xs[-1])
        xs.append(A @ xs[-1] + B @ us[-1])
    return np.array(xs), np.array(us)


def test_small_offsets_from_hover_follow_the_lqr_of_the_linearisation():
    """Starting delta away from hover at the goal (no obstacles), the NMPC solution
    approaches the textbook LQR rollout of the RK4 step linearised at hover (its
    Jacobians by central differences) to second order in delta."""
    N, dt = 6, 0.1
    desc = QuatProblemDesc(nq=1, horizon=N, dt=dt)
    lay = theta_layout(desc)
    xh = np.zeros(13)
    xh[3] = 1.0
    uh = np.full(4, OMEGA_H)

    def step(x, u):
        return rk4(torch.as_tensor(x), torch.as_tensor(u), dt, quat13_rhs).numpy()

    h = 1e-6
    A = np.stack([(step(xh + h * e, uh) - step(xh - h * e, uh)) / (2 * h) for e in np.eye(13)], axis=1)
    B = np.stack([(step(xh, uh + h * e) - step(xh, uh - h * e)) / (2 * h) for e in np.eye(4)], axis=1)
    # the weights of the reading, restated: Q = diag(10 I3 (p), I4 (q), I3 (v), 0.1 I3 (w)),
    # R = 0.1 (dT/dOmega at hover)^2 with thrust m g / 4 = K_F Omega_h^2 per rotor
    Q = np.diag([10.0] * 3 + [1.0] * 4 + [1.0] * 3 + [0.1] * 3)
    kf = 0.5 * 9.81 / 4.0 / 400.0 ** 2
    R = 0.1 * (2.0 * kf * 400.0) ** 2 * np.eye(4)
    d = np.random.default_rng(17).standard_normal(13)

    def deviation(delta):
        x0 = xh + delta * d
        x0[3:7] /= np.linalg.norm(x0[3:7])
        th = np.zeros(lay["end"])
        th[lay["xbar"]:lay["xbar"] + 13] = x0
        nlp = QuatNLP(desc, th)
        st, _ = ipm.solve(nlp, opt=ipm.Options(tol=1e-11))
        assert st.status == ipm.CONVERGED
        w = st.normal.x
        xs_l, us_l = _lqr_rollout(A, B, Q, R, 10 * Q, x0 - xh, N)
        xs = w[nlp.xi.numpy()] - xh
        us = w[nlp.ui.numpy()] - uh
        dev = max(np.abs(xs - xs_l).max(), np.abs(us - us_l).max() / OMEGA_H)
        return dev, np.abs(xs_l).max()

    (e1, s1), (e2, _) = deviation(1e-3), deviation(2e-3)
    assert e1 < 0.01 * s1            # far below the size of the trajectory itself
    assert 3.5 < e2 / e1 < 4.5       # second order in the offset
