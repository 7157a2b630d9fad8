"""Pins of the oracle's quadrotor transcription against physics and libraries.

Each test checks the oracle against something other than itself: rigid-body
identities evaluated with scipy's rotation library, an ODE integrator of
scipy, the observed convergence order of RK4, and finite differences of the
autograd derivatives.
"""

import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp
from scipy.spatial.transform import Rotation

from oracle import quadrotor as Q
from workloads import ProblemDesc, make_batch

F64 = torch.float64


def rhs_np(x, u):
    return Q.quad_rhs(torch.as_tensor(x, dtype=F64), torch.as_tensor(u, dtype=F64)).numpy()


def test_hover_is_an_equilibrium():
    x = np.zeros(12)
    x[0:3] = [1.0, -2.0, 3.0]
    x[8] = 0.7  # yaw does not matter at hover
    u = np.full(4, Q.HOVER)
    assert np.allclose(rhs_np(x, u), 0.0, atol=1e-14)
    F = Q.rk4(torch.as_tensor(x), torch.as_tensor(u), 0.05).numpy()
    assert np.allclose(F, x, atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_thrust_direction_is_body_z_axis(seed):
    rng = np.random.default_rng(seed)
    eta = rng.uniform(-0.8, 0.8, 3)
    x = np.zeros(12)
    x[6:9] = eta
    u = rng.uniform(0.5, 2.0, 4)
    acc = rhs_np(x, u)[3:6]
    # ZYX convention: R = Rz(psi) Ry(theta) Rx(phi)
    R = Rotation.from_euler("ZYX", [eta[2], eta[1], eta[0]]).as_matrix()
    expect = R[:, 2] * u.sum() / Q.MASS - np.array([0, 0, Q.GRAV])
    assert np.allclose(acc, expect, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_euler_rates_match_rotation_kinematics(seed):
    """R(eta + h eta_dot) ~= R(eta) expm(h [omega]_x) to first order in h."""
    rng = np.random.default_rng(100 + seed)
    eta = rng.uniform(-0.7, 0.7, 3)
    om = rng.uniform(-2, 2, 3)
    x = np.zeros(12)
    x[6:9] = eta
    x[9:12] = om
    etad = rhs_np(x, np.full(4, Q.HOVER))[6:9]

    def rot(e):
        return Rotation.from_euler("ZYX", [e[2], e[1], e[0]]).as_matrix()

    h = 1e-6
    Rdot = (rot(eta + h * etad) - rot(eta - h * etad)) / (2 * h)
    Om = rot(eta).T @ Rdot  # = [omega]_x for body rates
    assert np.allclose([Om[2, 1], Om[0, 2], Om[1, 0]], om, rtol=1e-7, atol=1e-7)
    assert np.allclose(Om + Om.T, 0.0, atol=1e-7)


@pytest.mark.parametrize("seed", range(4))
def test_rotational_dynamics_from_rotor_geometry(seed):
    """Torques from rotor positions (cross products) and Euler's equations."""
    rng = np.random.default_rng(200 + seed)
    om = rng.uniform(-3, 3, 3)
    u = rng.uniform(0, 2.4, 4)
    x = np.zeros(12)
    x[9:12] = om
    wd = rhs_np(x, u)[9:12]
    L = Q.ARM
    arms = [np.array([L, 0, 0]), np.array([0, L, 0]), np.array([-L, 0, 0]), np.array([0, -L, 0])]
    tau = sum(np.cross(a, np.array([0, 0, f])) for a, f in zip(arms, u))
    tau[2] += Q.KAPPA * (u[0] - u[1] + u[2] - u[3])
    J = np.diag(Q.INERTIA)
    expect = np.linalg.solve(J, tau - np.cross(om, J @ om))
    assert np.allclose(wd, expect, rtol=1e-12, atol=1e-12)


def test_rk4_exact_for_constant_acceleration():
    x = np.zeros(12)
    x[3:6] = [0.3, -0.2, 0.1]
    x[6] = 0.25  # constant roll, no body rates
    u = np.array([1.0, 1.1, 1.0, 1.1])
    dt = 0.05
    a = rhs_np(x, u)[3:6]
    F = Q.rk4(torch.as_tensor(x), torch.as_tensor(u), dt).numpy()
    assert np.allclose(F[0:3], x[0:3] + dt * x[3:6] + 0.5 * dt * dt * a, atol=1e-15)
    assert np.allclose(F[3:6], x[3:6] + dt * a, atol=1e-15)


def test_rk4_is_fourth_order_against_scipy():
    rng = np.random.default_rng(7)
    x0 = np.concatenate([rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3),
                         rng.uniform(-0.4, 0.4, 3), rng.uniform(-2, 2, 3)])
    u = rng.uniform(0.8, 1.6, 4)
    errs = []
    for dt in (0.08, 0.04):
        ref = solve_ivp(lambda t, z: rhs_np(z, u), (0, dt), x0, method="DOP853",
                        rtol=1e-13, atol=1e-13).y[:, -1]
        F = Q.rk4(torch.as_tensor(x0), torch.as_tensor(u), dt).numpy()
        errs.append(np.max(np.abs(F - ref)))
    # local error of a 4th-order method scales like dt^5
    order = np.log2(errs[0] / errs[1])
    assert 4.5 < order < 5.5, (errs, order)


def _nlp(name="nav1", j=0, horizon=None):
    desc, th = make_batch(name, j + 1)
    if horizon is not None:
        d0 = desc
        desc = ProblemDesc(nq=d0.nq, horizon=horizon, dt=d0.dt, n_sph=d0.n_sph,
                           n_cyl=d0.n_cyl, pair_dist=d0.pair_dist)
        desc, th = make_batch(name, j + 1, desc=desc)
    return Q.QuadNLP(desc, th[j])


def _perturbed_point(nlp, seed):
    rng = np.random.default_rng(seed)
    w = nlp.default_start() + 0.05 * rng.standard_normal(nlp.n)
    return w


@pytest.mark.parametrize("name,horizon", [("nav1", 3), ("multi4", 2), ("track", 3)])
def test_constraint_jacobian_matches_finite_differences(name, horizon):
    nlp = _nlp(name, 0, horizon)
    w = _perturbed_point(nlp, 1)
    J = nlp.jac_c(w)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for i in range(nlp.n):
        e = np.zeros(nlp.n)
        e[i] = h
        Jfd[:, i] = (nlp.c(w + e) - nlp.c(w - e)) / (2 * h)
    assert np.allclose(J, Jfd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("name,horizon", [("nav1", 2), ("multi4", 2)])
def test_lagrangian_hessian_matches_finite_differences(name, horizon):
    nlp = _nlp(name, 0, horizon)
    w = _perturbed_point(nlp, 2)
    rng = np.random.default_rng(3)
    y = rng.standard_normal(nlp.m)
    H = nlp.hess_lag(w, y)
    assert np.allclose(H, H.T, atol=1e-12)

    def grad_lag(v):
        return nlp.grad_f(v) + nlp.jac_c(v).T @ y

    h = 1e-5
    Hfd = np.zeros_like(H)
    for i in range(nlp.n):
        e = np.zeros(nlp.n)
        e[i] = h
        Hfd[:, i] = (grad_lag(w + e) - grad_lag(w - e)) / (2 * h)
    assert np.allclose(H, Hfd, rtol=1e-5, atol=1e-5)


def test_cost_and_constraint_values_by_hand():
    nlp = _nlp("nav1", 0)
    w = nlp.default_start()
    x, u, s = nlp.split(torch.as_tensor(w))
    # at the default start every state is xbar and every input is hover:
    # the dynamics defects vanish and only the position error to the origin costs
    c = nlp.c(w)
    assert np.allclose(c, 0.0, atol=1e-12)
    p0 = nlp.xbar.numpy()[0:3]
    expect = nlp.N * 10.0 * np.sum(p0 ** 2) + 10.0 * 10.0 * np.sum(p0 ** 2)
    assert np.isclose(nlp.f(w), expect, rtol=1e-14)
    cen, rad = nlp.sph[0, 0:3].numpy(), float(nlp.sph[0, 3])
    assert np.allclose(s.numpy(), np.sum((p0 - cen) ** 2) - rad ** 2)


@pytest.mark.parametrize("case", ["nav1", "track", "pairs_cyl"])
def test_stage_assembled_derivatives_equal_whole_vector_autograd(case):
    """The oracle assembles the constraint Jacobian and the Lagrangian Hessian
    from per-stage autograd; differentiating the whole decision vector at once
    must give the same matrices (sparsity placement, signs of the dynamics rows,
    multiplier indexing, the objective factor)."""
    desc = None if case != "pairs_cyl" else ProblemDesc(nq=3, horizon=4, dt=0.05, n_sph=1, n_cyl=2, pair_dist=0.4)
    name = "multi4" if case == "pairs_cyl" else case
    d, th = make_batch(name, 1, desc=desc)
    nlp = Q.QuadNLP(d, th[0])
    rng = np.random.default_rng(7)
    x = nlp.default_start() + 0.1 * rng.standard_normal(nlp.n)
    y = rng.standard_normal(nlp.m)
    assert np.allclose(nlp.jac_c(x), nlp.jac_c_whole(x), rtol=0, atol=1e-12)
    for of in (1.0, 0.0, 2.5):
        assert np.allclose(nlp.hess_lag(x, y, of), nlp.hess_lag_whole(x, y, of), rtol=0, atol=1e-11)


def test_moving_sphere_rows_by_hand():
    """A moving sphere (c + v t, radius r) at stage k enters as |p_k - (c + v k dt)|^2 - r^2
    - s = 0.  c = (1, 2, 3), v = (0.5, -1, 2), r = 0.5, dt = 0.05: at k = 4 (t = 0.2) the
    centre is (1.1, 1.8, 3.4); with p_4 = (2, 2, 2): 0.81 + 0.04 + 1.96 - 0.25 = 2.56.
    The default start puts every slack at g(xbar) of its own stage, so those rows are 0."""
    desc = ProblemDesc(nq=1, horizon=5, dt=0.05, n_mov=1)
    th = np.zeros(18 + 7)
    th[0:3] = [0.2, -0.3, 1.0]
    th[18:25] = [1.0, 2.0, 3.0, 0.5, 0.5, -1.0, 2.0]
    nlp = Q.QuadNLP(desc, th)
    w = nlp.default_start()
    c = nlp.c(w)
    ineq_rows = [12 + k * 13 + 12 for k in range(5)]   # after each stage's dynamics rows
    assert np.allclose(c[ineq_rows], 0.0, atol=1e-14)
    x4 = np.zeros(12)
    x4[0:3] = [2.0, 2.0, 2.0]
    g = nlp.ineq(torch.as_tensor(x4).reshape(1, -1), torch.tensor([4.0])).numpy()[0]
    assert g[0] == pytest.approx(2.56, rel=1e-14)
