"""Pins of the oracle's interior-point iteration against closed forms, brute
force, a textbook LQR and independent KKT checks."""

import numpy as np
import pytest
import torch

from oracle import ipm
from oracle.generic import TorchNLP
from oracle.quadrotor import HOVER, QuadNLP
from workloads import ProblemDesc

F64 = torch.float64


def solve(nlp, **kw):
    opt = ipm.Options(**kw)
    st, hist = ipm.solve(nlp, opt=opt, record=True)
    return st, hist, opt


def test_kkt_factor_inertia_matches_eigenvalues():
    rng = np.random.default_rng(0)
    for trial in range(20):
        n = int(rng.integers(2, 9))
        m = int(rng.integers(1, n))
        H = rng.standard_normal((n, n))
        H = H + H.T + rng.uniform(-3, 3) * np.eye(n)
        J = rng.standard_normal((m, n))
        K = ipm.augmented_matrix(H, J, 0.0)
        ev = np.linalg.eigvalsh(K)
        if np.min(np.abs(ev)) < 1e-6:
            continue
        fac = ipm.KKTFactor(K)
        assert fac.n_pos == np.sum(ev > 1e-10)
        assert fac.n_neg == np.sum(ev < -1e-10)
        b = rng.standard_normal(n + m)
        assert np.allclose(fac.solve(b), np.linalg.solve(K, b), rtol=1e-9, atol=1e-9)


def test_bound_only_1d_closed_form():
    # min (x-2)^2 s.t. 0 <= x <= 1  ->  x* = 1, z_U* = 2
    nlp = TorchNLP(lambda x: (x[0] - 2.0) ** 2, None, 1, 0, xl=[0.0], xu=[1.0], x0=[0.5])
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    assert abs(st.normal.x[0] - 1.0) < 1e-6
    assert abs(st.normal.zu[0] - 2.0) < 1e-5


def test_equality_qp_closed_form():
    rng = np.random.default_rng(1)
    n, m = 6, 3
    M = rng.standard_normal((n, n))
    H = M @ M.T + np.eye(n)
    g = rng.standard_normal(n)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    Ht, gt, At, bt = (torch.as_tensor(v, dtype=F64) for v in (H, g, A, b))
    nlp = TorchNLP(lambda x: 0.5 * x @ Ht @ x + gt @ x, lambda x: At @ x - bt, n, m)
    st, _, _ = solve(nlp)
    K = np.block([[H, A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([-g, b]))
    assert st.status == ipm.CONVERGED
    assert np.allclose(st.normal.x, sol[:n], atol=1e-8)
    assert np.allclose(st.normal.y, sol[n:], atol=1e-7)


def test_capped_simplex_projection():
    # min 1/2 |x - a|^2 s.t. sum x = 1, 0 <= x <= 1: x_i = clip(a_i - t, 0, 1)
    a = np.array([0.9, 0.7, -0.3, 1.8, 0.2])
    lo, hi = -5.0, 5.0
    for _ in range(200):
        t = 0.5 * (lo + hi)
        if np.clip(a - t, 0, 1).sum() > 1:
            lo = t
        else:
            hi = t
    expect = np.clip(a - 0.5 * (lo + hi), 0, 1)
    at = torch.as_tensor(a, dtype=F64)
    nlp = TorchNLP(lambda x: 0.5 * ((x - at) ** 2).sum(), lambda x: (x.sum() - 1.0).reshape(1),
                   5, 1, xl=np.zeros(5), xu=np.ones(5), x0=np.full(5, 0.2))
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    # E_0 <= 1e-6 bounds s * z; with bound multipliers >= 0.15 an active bound is
    # met to within 1e-6 / 0.15, and the free components move by as much
    assert np.allclose(st.normal.x, expect, atol=1e-5)


def test_disk_inequality_through_slack():
    # min (x-2)^2 + (y-1)^2 s.t. x^2 + y^2 <= 1  ->  (2, 1)/sqrt(5)
    f = lambda w: (w[0] - 2.0) ** 2 + (w[1] - 1.0) ** 2
    c = lambda w: (1.0 - w[0] ** 2 - w[1] ** 2 - w[2]).reshape(1)
    nlp = TorchNLP(f, c, 3, 1, xl=[-np.inf, -np.inf, 0.0], xu=[np.inf] * 3, x0=[0.0, 0.0, 1.0])
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    assert np.allclose(st.normal.x[:2], np.array([2.0, 1.0]) / np.sqrt(5.0), atol=1e-6)


def _brute_force_min(f, g_ok, lo, hi, n=4001):
    xs = np.linspace(lo, hi, n)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    F = f(X, Y)
    F[~g_ok(X, Y)] = np.inf
    i = np.unravel_index(np.argmin(F), F.shape)
    return X[i], Y[i], F[i]


def test_rosenbrock_in_disk_brute_force():
    fn = lambda x, y: (1 - x) ** 2 + 100 * (y - x * x) ** 2
    bx, by, bf = _brute_force_min(fn, lambda x, y: x * x + y * y <= 1.0, -1.2, 1.2)
    f = lambda w: (1 - w[0]) ** 2 + 100 * (w[1] - w[0] ** 2) ** 2
    c = lambda w: (1.0 - w[0] ** 2 - w[1] ** 2 - w[2]).reshape(1)
    nlp = TorchNLP(f, c, 3, 1, xl=[-np.inf, -np.inf, 0.0], xu=[np.inf] * 3, x0=[-0.5, 0.5, 0.5])
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    x, y = st.normal.x[:2]
    # the grid has spacing 6e-4; the solver's point must be at least as good and nearby
    assert fn(x, y) <= bf + 1e-6
    assert abs(x - bx) < 2e-3 and abs(y - by) < 2e-3


def test_two_global_minima_brute_force():
    # min x y s.t. x^2 + y^2 = 1: minima +-(1/sqrt2, -1/sqrt2), value -1/2
    f = lambda w: w[0] * w[1]
    c = lambda w: (w[0] ** 2 + w[1] ** 2 - 1.0).reshape(1)
    nlp = TorchNLP(f, c, 2, 1, x0=[0.9, -0.2])
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    x, y = st.normal.x
    assert abs(x * y + 0.5) < 1e-7
    assert min(np.hypot(x - 2 ** -0.5, y + 2 ** -0.5), np.hypot(x + 2 ** -0.5, y - 2 ** -0.5)) < 1e-6


def test_wachter_biegler_example_ends_at_l1_infeasibility_minimum():
    """The classic counterexample for line-search IPMs (Wachter & Biegler 2000):
    min x1 s.t. x1^2 - x2 - 1 = 0, x1 - x3 - 1/2 = 0, x2, x3 >= 0, from (-2, 1, 1).

    Plain Newton steps stall at x1 < -1 with x2, x3 -> 0; the filter method
    enters restoration.  The l1 restoration problem is a local method and the
    point x1 = -1, x2 = x3 = 0 is a local minimiser of |c|_1 over the bounds,
    so the run must enter and leave restoration and finally report a
    restoration failure there (local infeasibility)."""
    f = lambda w: w[0]
    c = lambda w: torch.stack([w[0] ** 2 - w[1] - 1.0, w[0] - w[2] - 0.5])
    nlp = TorchNLP(f, c, 3, 2, xl=[-np.inf, 0.0, 0.0], xu=[np.inf] * 3, x0=[-2.0, 1.0, 1.0])
    st, hist, _ = solve(nlp)
    assert any(tr.get("entered_resto") for (_, tr) in hist)
    assert any(tr.get("left_resto") for (_, tr) in hist)
    assert st.status == ipm.RESTO_FAILED
    x_end = st.resto.x[:3] if st.resto is not None else st.normal.x
    assert abs(x_end[0] + 1.0) < 1e-3 and x_end[1] < 1e-4 and x_end[2] < 1e-4
    # brute force: |c|_1 over a box around (-1, 0, 0) (x2, x3 >= 0) is minimal there
    g = np.linspace(-0.2, 0.2, 81)
    best = min(abs(a * a - b - 1) + abs(a - cc - 0.5)
               for a in -1.0 + g for b in np.abs(g) for cc in np.abs(g))
    assert best >= 1.5 - 1e-12


def test_restoration_recovers_from_singular_jacobian():
    """min (x-2)^2 + (y-1)^2 s.t. x^2 + y^2 = 1, -1 <= x, y <= 3, from (0, 0):
    the constraint Jacobian vanishes at the start, no regularisation gives the
    required inertia, restoration moves off the origin and the method then
    converges to the closed form (2, 1)/sqrt(5)."""
    f = lambda w: (w[0] - 2.0) ** 2 + (w[1] - 1.0) ** 2
    c = lambda w: (w[0] ** 2 + w[1] ** 2 - 1.0).reshape(1)
    nlp = TorchNLP(f, c, 2, 1, xl=[-1.0, -1.0], xu=[3.0, 3.0], x0=[0.0, 0.0])
    st, hist, _ = solve(nlp)
    assert hist[0][1].get("ic_failed") and hist[0][1].get("entered_resto")
    assert st.n_resto_iter >= 1
    assert st.status == ipm.CONVERGED
    assert np.allclose(st.normal.x, np.array([2.0, 1.0]) / np.sqrt(5.0), atol=1e-6)


def test_locally_infeasible_problem_reports_restoration_failure():
    # x^2 + 1 = 0 has no real solution
    f = lambda w: (w[0] - 1.0) ** 2
    c = lambda w: (w[0] ** 2 + 1.0).reshape(1)
    nlp = TorchNLP(f, c, 1, 1, x0=[0.5])
    st, _, _ = solve(nlp, max_iter=200)
    assert st.status in (ipm.RESTO_FAILED, ipm.MAX_ITER)
    assert st.status == ipm.RESTO_FAILED


def _lin_quad_nlp(N, A, B, Qw, Rw, QN, x0):
    nx, nu = B.shape
    At, Bt = torch.as_tensor(A), torch.as_tensor(B)
    Qt, Rt, QNt = (torch.as_tensor(v) for v in (Qw, Rw, QN))
    x0t = torch.as_tensor(x0)
    n = nx * (N + 1) + nu * N
    m = nx * (N + 1)

    def xs_us(w):
        xs = [w[k * (nx + nu):k * (nx + nu) + nx] for k in range(N + 1)]
        us = [w[k * (nx + nu) + nx:(k + 1) * (nx + nu)] for k in range(N)]
        return xs, us

    def f(w):
        xs, us = xs_us(w)
        val = sum(xs[k] @ Qt @ xs[k] + us[k] @ Rt @ us[k] for k in range(N))
        return val + xs[N] @ QNt @ xs[N]

    def c(w):
        xs, us = xs_us(w)
        rows = [xs[0] - x0t] + [xs[k + 1] - At @ xs[k] - Bt @ us[k] for k in range(N)]
        return torch.cat(rows)

    xl = np.full(n, -np.inf)
    xu = np.full(n, np.inf)
    for k in range(N):
        xl[k * (nx + nu) + nx:(k + 1) * (nx + nu)] = -50.0
        xu[k * (nx + nu) + nx:(k + 1) * (nx + nu)] = 50.0
    return TorchNLP(f, c, n, m, xl=xl, xu=xu, x0=np.zeros(n))


def test_linear_quadratic_matches_textbook_lqr():
    """Linearised hover model without obstacles: the solution is the finite-horizon
    discrete LQR rollout (backward Riccati recursion, textbook form)."""
    nlp_q = QuadNLP(ProblemDesc(nq=1, horizon=4, dt=0.05), np.zeros(18))
    xh = torch.zeros(12, dtype=F64)
    uh = torch.full((4,), HOVER, dtype=F64)
    from oracle.quadrotor import rk4
    A = torch.func.jacfwd(lambda x: rk4(x, uh, 0.05))(xh).numpy()
    B = torch.func.jacfwd(lambda u: rk4(xh, u, 0.05))(uh).numpy()
    Qw = np.diag([10.0] * 3 + [1.0] * 6 + [0.1] * 3)
    Rw = 0.1 * np.eye(4)
    QN = 10 * Qw
    N = 6
    x0 = np.array([0.1, -0.05, 0.08, 0.02, 0.0, -0.03, 0.01, 0.02, -0.01, 0.0, 0.05, 0.0])
    # textbook LQR: P_N = QN, K_k = -(R + B'PB)^{-1} B'PA, P_k = Q + A'PA + A'PB K
    P = QN
    Ks = []
    for _ in range(N):
        K = -np.linalg.solve(Rw + B.T @ P @ B, B.T @ P @ A)
        P = Qw + A.T @ P @ A + A.T @ P @ B @ K
        Ks.append(K)
    Ks = Ks[::-1]
    xs = [x0]
    us = []
    for k in range(N):
        us.append(Ks[k] @ xs[-1])
        xs.append(A @ xs[-1] + B @ us[-1])
    nlp = _lin_quad_nlp(N, A, B, Qw, Rw, QN, x0)
    st, _, _ = solve(nlp, tol=1e-9)
    assert st.status == ipm.CONVERGED
    w = st.normal.x
    for k in range(N):
        assert np.allclose(w[k * 16:k * 16 + 12], xs[k], atol=1e-6)
        assert np.allclose(w[k * 16 + 12:k * 16 + 16], us[k], atol=1e-6)
    del nlp_q


def test_quadrotor_hover_at_goal_is_already_optimal():
    desc = ProblemDesc(nq=1, horizon=5, dt=0.05, n_sph=1)
    theta = np.zeros(22)
    theta[18:22] = [5.0, 5.0, 5.0, 0.5]  # far-away sphere
    nlp = QuadNLP(desc, theta)
    st, _, _ = solve(nlp)
    assert st.status == ipm.CONVERGED
    x, u, _ = nlp.split(torch.as_tensor(st.normal.x))
    assert np.allclose(x.numpy(), 0.0, atol=1e-5)
    assert np.allclose(u.numpy(), HOVER, atol=1e-5)
    assert nlp.f(st.normal.x) < 1e-8


def independent_kkt_residuals(nlp, st, h=1e-6):
    """Stationarity and feasibility by central finite differences (not autograd)."""
    ph = st.normal
    x = ph.x

    def lag(v):
        return nlp.f(v) + ph.y @ nlp.c(v)

    grad = np.zeros(nlp.n)
    for i in range(nlp.n):
        e = np.zeros(nlp.n)
        e[i] = h * max(1.0, abs(x[i]))
        grad[i] = (lag(x + e) - lag(x - e)) / (2 * e[i])
    stat = grad - ph.zl + ph.zu
    return np.max(np.abs(stat)), np.max(np.abs(nlp.c(x)))


@pytest.mark.parametrize("j", [0, 1])
def test_quadrotor_nav_invariants_and_kkt(j):
    from workloads import make_batch
    desc, th = make_batch("nav1", j + 1)
    nlp = QuadNLP(desc, th[j])
    st, hist, opt = solve(nlp)
    assert st.status == ipm.CONVERGED
    has_l, has_u = ipm.bound_sets(nlp)
    mus = []
    for (s, tr) in hist:
        ph = s.normal if s.mode == ipm.NORMAL else None
        if ph is None:
            continue
        sl, su = ipm.slacks(nlp, ph.x)
        assert np.all(sl[has_l] > 0) and np.all(su[has_u] > 0)
        assert np.all(ph.zl[has_l] > 0) and np.all(ph.zu[has_u] > 0)
        mus.append(ph.mu)
    assert all(a >= b for a, b in zip(mus, mus[1:]))
    stat, feas = independent_kkt_residuals(nlp, st)
    assert feas <= 1e-6
    # finite differences carry ~1e-6 error on gradients of size ~1e2
    assert stat <= 1e-3
    m = ipm.final_metrics(nlp, st)
    assert m["kkt"] <= 1e-6
