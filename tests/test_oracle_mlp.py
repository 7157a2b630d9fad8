"""Pins of the CPU warm-start network and encodings (oracle.mlp, oracle.warm).

Each test checks the oracle against something other than itself: a library's
bfloat16 conversion, central finite differences, the textbook least-squares
gradient, Adam's closed-form first steps, hand-computed features, and the NLP's
own inequality functions.
"""

import numpy as np
import pytest
import torch

from oracle import ipm, mlp, warm
from oracle.quadrotor import HOVER, QuadNLP
from workloads import ProblemDesc, make_batch, mlp_init, theta_layout


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    v32 = np.concatenate([rng.standard_normal(20000), rng.uniform(-1e3, 1e3, 20000),
                          rng.uniform(-1e-3, 1e-3, 2000)]).astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    got = mlp.bf16(v32.astype(np.float64))
    np.testing.assert_array_equal(got, ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    # unit roundoff of round-to-nearest with 8 significant bits: 2^-8
    x = rng.standard_normal(1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= 2.0 ** -8 * np.abs(x))


def _tiny(seed=1, dims=(5, 7, 6, 4), rows=3):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(mlp.n_params(dims)) * 0.5
    x = rng.standard_normal((rows, dims[0]))
    t = rng.standard_normal((rows, dims[-1]))
    return dims, flat, x, t


def test_gradient_matches_central_differences():
    dims, flat, x, t = _tiny()
    _, g = mlp.loss_and_grad(dims, flat, x, t)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = h
        lp, _ = mlp.loss_and_grad(dims, flat + e, x, t)
        lm, _ = mlp.loss_and_grad(dims, flat - e, x, t)
        fd[i] = (lp - lm) / (2 * h)
    assert np.max(np.abs(g - fd)) <= 1e-8 * max(1.0, np.max(np.abs(fd)))


def test_single_linear_layer_is_least_squares():
    rng = np.random.default_rng(2)
    dims = (6, 3)
    W = rng.standard_normal((3, 6))
    b = rng.standard_normal(3)
    x = rng.standard_normal((10, 6))
    t = rng.standard_normal((10, 3))
    loss, g = mlp.loss_and_grad(dims, np.concatenate([W.ravel(), b]), x, t)
    r = x @ W.T + b - t
    assert loss == pytest.approx(0.5 * np.sum(r * r) / 10, rel=1e-14)
    np.testing.assert_allclose(g[:18].reshape(3, 6), r.T @ x / 10, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g[18:], r.sum(0) / 10, rtol=1e-13, atol=1e-15)


def test_bf16_emulation_is_exact_on_representable_values():
    # weights and inputs on a coarse dyadic grid are bfloat16 numbers, so rounding
    # the product operands changes nothing in the first layer
    rng = np.random.default_rng(3)
    dims = (8, 4)
    flat = rng.integers(-8, 8, mlp.n_params(dims)) / 8.0
    x = rng.integers(-8, 8, (5, 8)) / 4.0
    o1, _ = mlp.forward(dims, flat, x, emulate_bf16=True)
    o2, _ = mlp.forward(dims, flat, x, emulate_bf16=False)
    np.testing.assert_array_equal(o1, o2)
    # and the emulated network stays within the rounding bound of the exact one
    dims, flat, x, t = _tiny(4, dims=(16, 32, 32, 8), rows=16)
    e1, g1 = mlp.loss_and_grad(dims, flat, x, t, emulate_bf16=True)
    e0, g0 = mlp.loss_and_grad(dims, flat, x, t)
    assert abs(e1 - e0) <= 0.05 * e0
    assert np.linalg.norm(g1 - g0) <= 0.05 * np.linalg.norm(g0)


def test_adam_first_steps_closed_form():
    # with bias correction, a constant gradient g moves every parameter by
    # lr * g / (|g| + eps) at every step
    g = np.array([0.5, -2.0, 1e-3, -4e-2])
    opt = mlp.Adam(4)
    p = np.zeros(4)
    for _ in range(3):
        q = opt.step(p, g, 0.01)
        np.testing.assert_allclose(q - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
        p = q
    # a zero gradient after one step decays the first moment by beta1 per step
    opt = mlp.Adam(1)
    p1 = opt.step(np.zeros(1), np.array([1.0]), 1.0)
    p2 = opt.step(p1, np.array([0.0]), 1.0)
    m_hat = 0.1 * 0.9 / (1 - 0.9 ** 2)
    v_hat = 0.001 * 0.999 / (1 - 0.999 ** 2)
    assert p2[0] - p1[0] == pytest.approx(-m_hat / (np.sqrt(v_hat) + 1e-8), rel=1e-12)


def test_training_reduces_the_loss():
    dims = (6, 16, 16, 3)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((64, 6))
    t = np.stack([np.sin(x[:, 0]), x[:, 1] * x[:, 2], np.cos(x[:, 3])], axis=1)
    flat = mlp_init(dims, 7).astype(np.float64)
    opt = mlp.Adam(flat.size)
    l0, _ = mlp.loss_and_grad(dims, flat, x, t)
    for _ in range(300):
        _, g = mlp.loss_and_grad(dims, flat, x, t)
        flat = opt.step(flat, g, 1e-2)
    l1, _ = mlp.loss_and_grad(dims, flat, x, t)
    assert l1 < 0.2 * l0


# ------------------------------------------------------------- encodings

CYL = ProblemDesc(nq=1, horizon=4, dt=0.05, n_cyl=4)


def _hand_theta():
    lay = theta_layout(CYL)
    th = np.zeros(lay["end"])
    th[lay["xbar"]:lay["xbar"] + 12] = [1.0, 2.0, 1.5, 0.4, -0.2, 0.0, 0.1, -0.1, 0.3, 0.2, 0.0, -0.4]
    th[lay["ref"]:lay["ref"] + 6] = [0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    # centre distances from (1, 2): 5, 1, 100 (beyond the cutoff), 2
    th[lay["cyl"]:lay["cyl"] + 12] = [4.0, 6.0, 0.3, 2.0, 2.0, 0.5, 101.0, 2.0, 0.2, 1.0, 0.0, 0.4]
    return th


def test_features_by_hand():
    f = warm.features(CYL, _hand_theta(), k_near=5)
    expect = [0.1, 0.2, 0.05, 0.2, -0.1, 0.0, 0.1, -0.1, 0.3, 0.1, 0.0, -0.2,
              0.1, 0.0, 0.5,      # distance 1
              0.0, -0.2, 0.4,     # distance 2
              0.3, 0.4, 0.3,      # distance 5
              0.0, 0.0, 0.0,      # distance 100 > cutoff
              0.0, 0.0, 0.0]      # no fifth cylinder
    np.testing.assert_allclose(f, expect, rtol=0, atol=1e-15)
    assert warm.features(CYL, _hand_theta(), k_near=2).size == 18


def test_features_rank_cylinders_by_distance():
    desc, theta = make_batch("cyl", 3)
    for th in theta:
        f = warm.features(desc, th, k_near=50)
        rel = f[12:].reshape(50, 3)
        d = np.hypot(rel[:, 0], rel[:, 1])
        real = rel[:, 2] > 0
        assert np.all(np.diff(d[real]) >= 0)
        assert real.sum() >= 20


def test_encode_decode_round_trip_and_slacks():
    desc = CYL
    th = _hand_theta()
    nlp = QuadNLP(desc, th)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(desc.n)
    x[nlp.xi[0].numpy()] = nlp.xbar.numpy()
    o = warm.encode(desc, th, x)
    assert o.size == warm.output_dim(desc) == 12 * 5 + 16
    assert np.all(o[:12] == 0.0)
    xd = warm.decode(desc, th, o, lambda s: nlp.ineq(torch.as_tensor(s)).numpy())
    xi, ui, si = (v.numpy().ravel() for v in (nlp.xi, nlp.ui, nlp.si))
    np.testing.assert_allclose(xd[xi], x[xi], rtol=0, atol=1e-14)
    np.testing.assert_allclose(xd[ui], x[ui], rtol=0, atol=1e-14)
    # slacks at the decoded states make every inequality row of c(x) vanish
    c = nlp.c(xd)
    rows = np.concatenate([desc.nx + k * (desc.nx + desc.ni) + desc.nx + np.arange(desc.ni)
                           for k in range(desc.horizon)])
    np.testing.assert_allclose(c[rows], 0.0, atol=1e-12)
    # hover input encodes to zero
    assert warm.encode(desc, th, np.where(np.isin(np.arange(desc.n), ui), HOVER, x))[60:].max() == 0.0


def test_warm_initial_point_is_centred_and_interior():
    desc, theta = make_batch("cyl", 1, desc=ProblemDesc(nq=1, horizon=6, dt=0.05, n_cyl=50))
    nlp = QuadNLP(desc, theta[0])
    opt = warm.warm_options()
    x0 = nlp.default_start()
    x0[nlp.si.numpy().ravel()[:5]] = -1.0          # a guess inside an obstacle
    st = ipm.initial_state(nlp, x0, opt)
    ph = st.normal
    has_l, has_u = ipm.bound_sets(nlp)
    sl, su = ipm.slacks(nlp, ph.x)
    assert np.all(sl[has_l] > 0) and np.all(su[has_u] > 0)
    np.testing.assert_allclose(sl[has_l] * ph.zl[has_l], opt.mu_init, rtol=1e-14)
    np.testing.assert_allclose(su[has_u] * ph.zu[has_u], opt.mu_init, rtol=1e-14)
    assert ph.mu == 1e-2
    assert np.min(sl[has_l]) == pytest.approx(1e-3)


def test_warm_start_from_the_solution_converges_quickly():
    desc, theta = make_batch("cyl", 1, desc=ProblemDesc(nq=1, horizon=8, dt=0.05, n_cyl=50))
    nlp = QuadNLP(desc, theta[0])
    cold, _ = ipm.solve(nlp)
    assert cold.status == ipm.CONVERGED
    o = warm.encode(desc, theta[0], cold.normal.x)
    x0 = warm.decode(desc, theta[0], o, lambda s: nlp.ineq(torch.as_tensor(s)).numpy())
    hot, _ = ipm.solve(nlp, x0=x0, opt=warm.warm_options())
    assert hot.status == ipm.CONVERGED
    assert hot.iter < cold.iter
    assert np.max(np.abs(hot.normal.x - cold.normal.x)) < 1e-4
