"""Pins of the oracle's step-level rules on hand-made numbers (no GPU).

Every parity test of the CUDA path compares it with the oracle step by step,
so a rule both sides read the same wrong way would pass them all.  These pins
check each rule of the iteration against values worked out by hand from its
definition (the branches of Table I and the IPOPT rules Sec. IV defers to),
chosen so that a plausible slip -- a flipped inequality, swapped exponents,
a dropped term, the wrong end of the filter -- fails at least one of them.
The expected numbers are derived in each test's docstring.
"""

import math

import numpy as np
import pytest

from oracle import ipm
from oracle.generic import TorchNLP

OPT = ipm.Options()


def rel(value, r=1e-12):
    """pytest.approx with a relative tolerance only (no absolute slack near zero)."""
    return pytest.approx(value, rel=r, abs=0.0)


def _phase(filt=(), theta_max=10.0, theta_min=1e-4):
    ph = ipm.Phase(x=np.zeros(1), y=np.zeros(0), zl=np.zeros(1), zu=np.zeros(1), mu=0.1,
                   filt=list(filt))
    ph.theta_max, ph.theta_min = theta_max, theta_min
    return ph


# ------------------------------------------------------------------ filter --

def test_filter_membership_uses_weak_dominance_and_theta_max():
    """Filter {(1, 5)}, theta_max 10.  A point is in the filter when theta >= 1 and
    phi >= 5 (ties count), or when theta >= theta_max."""
    ph = _phase([(1.0, 5.0)])
    assert ipm.in_filter(ph, 1.0, 5.0)          # the entry itself (tie in both)
    assert ipm.in_filter(ph, 2.0, 6.0)          # worse in both
    assert not ipm.in_filter(ph, 0.999, 5.0)    # better theta
    assert not ipm.in_filter(ph, 1.0, 4.999)    # better phi
    assert not ipm.in_filter(ph, 0.5, 100.0)
    assert ipm.in_filter(ph, 10.0, -1e9)        # theta >= theta_max
    assert not ipm.in_filter(ph, 9.999, -1e9)


def test_filter_add_drops_dominated_entries_and_keeps_order():
    """Adding (1.5, 4) to [(1, 5), (2, 5), (0.5, 8)]: only (2, 5) has theta >= 1.5 and
    phi >= 4, so it goes; the new pair is appended.  Adding (0.4, 2) then removes
    every entry (all have theta >= 0.4 and phi >= 2)."""
    ph = _phase([(1.0, 5.0), (2.0, 5.0), (0.5, 8.0)])
    ipm.filter_add(ph, 1.5, 4.0, OPT)
    assert ph.filt == [(1.0, 5.0), (0.5, 8.0), (1.5, 4.0)]
    ipm.filter_add(ph, 0.4, 2.0, OPT)
    assert ph.filt == [(0.4, 2.0)]


def test_full_filter_drops_its_oldest_entry():
    """With room for 3 entries, a fourth non-dominated entry pushes out the first one
    added, not the newest."""
    opt = ipm.Options(filter_cap=3)
    ph = _phase()
    for e in [(1.0, 4.0), (2.0, 3.0), (3.0, 2.0), (0.5, 5.0)]:
        ipm.filter_add(ph, *e, opt)
    assert ph.filt == [(2.0, 3.0), (3.0, 2.0), (0.5, 5.0)]


def test_filter_entry_is_the_margin_shifted_pair():
    """theta = 2, phi = 7: ((1 - 1e-5) 2, 7 - 1e-8 * 2) = (1.99998, 6.99999998)."""
    t, p = ipm.filter_entry(2.0, 7.0, OPT)
    assert t == rel(1.99998, 1e-15)
    assert p == rel(6.99999998, 1e-15)


# -------------------------------------------------------- line-search rules --

def test_alpha_min_three_cases():
    """gamma_alpha = 0.05, gamma_theta = 1e-5, gamma_phi = 1e-8, delta = 1,
    s_theta = 1.1, s_phi = 2.3.
    (a) gdx < 0, theta <= theta_min: theta = 1e-6, gdx = -1e8: the terms are 1e-5,
        1e-8 * 1e-6 / 1e8 = 1e-22 and (1e-6)^1.1 / (1e8)^2.3 = 10^-6.6 / 10^18.4 = 1e-25,
        so alpha_min = 0.05e-25 = 5e-27.
    (b) gdx < 0, theta > theta_min: theta = 1, gdx = -1e-2: min(1e-5, 1e-8 / 1e-2 = 1e-6)
        = 1e-6, alpha_min = 5e-8.
    (c) gdx >= 0: 0.05 * 1e-5 = 5e-7."""
    assert ipm.alpha_min(1e-6, -1e8, 1e-4, OPT) == rel(5e-27, 1e-12)
    assert ipm.alpha_min(1.0, -1e-2, 1e-4, OPT) == rel(5e-8, 1e-12)
    assert ipm.alpha_min(1.0, 0.3, 1e-4, OPT) == rel(5e-7, 1e-12)
    assert ipm.alpha_min(1e-6, 0.0, 1e-4, OPT) == rel(5e-7, 1e-12)


def test_switching_condition_exponents():
    """alpha = 0.5, gdx = -2: alpha (-gdx)^2.3 = 0.5 * 4.92458 = 2.46229; theta^1.1 is
    2.14355 at theta = 2 (holds) and 2.74050 at theta = 2.5 (fails).  Swapping the
    exponents would give 0.5 * 2^1.1 = 1.0718 < 2^2.3 and fail the first case."""
    assert 0.5 * 2.0 ** 2.3 == rel(2.462289, 1e-6)
    assert ipm.switching_condition(0.5, -2.0, 2.0, OPT)
    assert not ipm.switching_condition(0.5, -2.0, 2.5, OPT)
    assert not ipm.switching_condition(0.5, 2.0, 1e-9, OPT)   # ascent direction
    assert not ipm.switching_condition(1.0, 0.0, 0.0, OPT)


def test_armijo_condition_sign():
    """phi0 = 10, alpha = 0.5, gdx = -2: the bound is 10 + 1e-8 * 0.5 * (-2) = 9.99999999."""
    assert ipm.armijo_holds(9.999999985, 10.0, 0.5, -2.0, OPT)
    assert ipm.armijo_holds(9.99999999, 10.0, 0.5, -2.0, OPT)       # equality accepts
    assert not ipm.armijo_holds(9.999999995, 10.0, 0.5, -2.0, OPT)  # decrease too small
    assert not ipm.armijo_holds(10.000000005, 10.0, 0.5, -2.0, OPT)


def test_sufficient_decrease_either_measure():
    """theta = 1, phi0 = 10: theta_t <= 0.99999 or phi_t <= 10 - 1e-8."""
    assert ipm.sufficient_decrease(0.99999, 50.0, 1.0, 10.0, OPT)
    assert not ipm.sufficient_decrease(0.999995, 10.0, 1.0, 10.0, OPT)
    assert ipm.sufficient_decrease(0.999995, 9.99999999, 1.0, 10.0, OPT)
    assert not ipm.sufficient_decrease(0.999995, 9.999999995, 1.0, 10.0, OPT)


def test_trial_acceptance_branches():
    """theta_min = 1e-4.
    * A nearly feasible iterate (theta = 1e-6) with a descent direction gdx = -1 and
      alpha = 1 satisfies the switching condition (1 > 1e-6^1.1 = 2.5e-7), so the
      Armijo rule decides: phi_t = phi0 - 1e-9 fails it (needs phi0 - 1e-8) although
      theta_t = 0 is a large decrease of theta.
    * The same trial at theta = 1 (> theta_min) is judged by sufficient decrease and
      accepted.
    * A point inside the filter is rejected whatever it decreases."""
    ph = _phase([(5.0, 5.0)], theta_min=1e-4)
    # switching holds at theta = 0.5 > theta_min (1 * 10^2.3 = 199.5 > 0.5^1.1 = 0.467):
    # sufficient decrease still decides, so a trial with theta_t = 0 and phi up by 1 passes
    assert ipm.switching_condition(1.0, -10.0, 0.5, OPT)
    assert ipm.trial_acceptable(ph, 0.0, 2.0, 1.0, 0.5, 1.0, -10.0, OPT)
    assert not ipm.trial_acceptable(ph, 0.0, 1.0 - 1e-9, 1.0, 1e-6, 1.0, -1.0, OPT)
    assert ipm.trial_acceptable(ph, 0.0, 1.0 - 2e-8, 1.0, 1e-6, 1.0, -1.0, OPT)
    assert ipm.trial_acceptable(ph, 0.0, 1.0 - 1e-9, 1.0, 1.0, 1.0, -1.0, OPT)
    assert not ipm.trial_acceptable(ph, 6.0, 6.0, 1.0, 10.0, 100.0, -1.0, OPT)
    assert not ipm.trial_acceptable(ph, 0.0, np.inf, 1.0, 1.0, 1.0, -1.0, OPT)


def test_filter_augmentation_rule():
    """No augmentation only when switching and Armijo both hold (an f-type step)."""
    # switching holds (theta tiny) and Armijo holds
    assert not ipm.filter_needs_augment(1.0, 1.0 - 2e-8, 1.0, -1.0, 1e-6, OPT)
    # switching holds, Armijo fails
    assert ipm.filter_needs_augment(1.0, 1.0 - 1e-9, 1.0, -1.0, 1e-6, OPT)
    # switching fails (theta large): augment even with a big decrease of phi
    assert ipm.filter_needs_augment(1.0, -100.0, 1.0, -1.0, 10.0, OPT)


def test_second_order_correction_recursion_and_stop():
    """c_soc^1 = alpha c(x) + c(x_alpha); c_soc^{p+1} = alpha_soc^p c_soc^p + c(x_soc^p).
    alpha = 0.5, c(x) = (2, -4), c(x_alpha) = (1, 1): c_soc^1 = (2, -1); with
    alpha_soc = 0.25 and c(x_soc) = (0.5, 0): c_soc^2 = (1.0, -0.25).  Stop after
    p_max = 4 corrections, or when theta_soc > 0.99 theta_old."""
    c1 = ipm.soc_constraint_rhs(0.5, np.array([2.0, -4.0]), np.array([1.0, 1.0]))
    assert np.array_equal(c1, [2.0, -1.0])
    c2 = ipm.soc_constraint_rhs(0.25, c1, np.array([0.5, 0.0]))
    assert np.array_equal(c2, [1.0, -0.25])
    assert not ipm.soc_should_stop(1, 0.98, 1.0, OPT)
    assert ipm.soc_should_stop(1, 0.995, 1.0, OPT)
    assert ipm.soc_should_stop(4, 0.1, 1.0, OPT)
    assert not ipm.soc_should_stop(3, 0.99, 1.0, OPT)  # equality keeps going


def test_second_order_correction_solves_the_corrected_linear_system():
    """min -x1 on the unit circle x0^2 + x1^2 = 1 from (1, 0): the Newton step is
    tangent to the circle, so the trial point leaves it and theta grows (the
    situation second-order corrections exist for).  The first correction's
    right-hand side must be alpha c(x) + c(x + alpha dx), and every correction step
    d_s must satisfy the linearised constraint with it: J d_s = -c_soc."""
    nlp = TorchNLP(lambda x: -x[1], lambda x: (x[0] ** 2 + x[1] ** 2 - 1.0).reshape(1), 2, 1,
                   x0=[1.0, 0.0])
    opt = ipm.Options(trace_soc=True)
    st = ipm.initial_state(nlp, np.array([1.0, 0.0]), opt)
    logs = []
    for _ in range(6):
        tr = {}
        ipm.phase_iteration(nlp, st.normal, opt, tr, init_theta=not logs, y_ls=not logs)
        logs += tr.get("soc_log", [])
    assert logs
    first = logs[0]
    x_trial_c = first["c_trial"]
    assert np.allclose(first["c_soc"], first["alpha"] * first["c"] + x_trial_c, rtol=1e-14, atol=0)
    for e in logs:
        assert np.allclose(e["J"] @ e["dx_soc"], -e["c_soc"], rtol=1e-9, atol=1e-12)


def test_tiny_step_threshold():
    """10 eps = 2.22e-15: |dx| / (1 + |x|) = 1e-15 / 2 = 5e-16 is tiny; 1e-14 / 1 is not."""
    assert ipm.is_tiny_step(np.array([1.0, 5.0]), np.array([1e-15, 0.0]))
    assert not ipm.is_tiny_step(np.array([0.0]), np.array([1e-14]))
    assert not ipm.is_tiny_step(np.array([0.0, 0.0]), np.array([0.0, 2.3e-15]))


# ------------------------------------------------------- bound handling --

def test_fraction_to_boundary():
    """v = (1, 2, 0.5), dv = (-2, 1, -0.25), tau = 0.99: the candidates -tau v / dv over
    dv < 0 are 0.495 and 1.98, so alpha = 0.495, and v + alpha dv keeps 1% of v_0."""
    v = np.array([1.0, 2.0, 0.5])
    dv = np.array([-2.0, 1.0, -0.25])
    a = ipm.frac_to_boundary(v, dv, 0.99)
    assert a == rel(0.495, 1e-15)
    assert (v + a * dv)[0] == rel(0.01, 1e-12)
    assert ipm.frac_to_boundary(v, np.abs(dv), 0.99) == 1.0


def test_kappa_sigma_reset_clips_both_ways():
    """mu = 0.1, s = 1e-3 (lower bound x_L = 0, x = 1e-3): kappa_Sigma mu / s = 1e12 and
    mu / (kappa_Sigma s) = 1e-8, so z = 5 stays, 1e13 -> 1e12, 1e-9 -> 1e-8."""
    nlp = TorchNLP(lambda x: x.sum(), None, 3, 0, xl=[0.0, 0.0, 0.0], xu=[np.inf] * 3)
    x = np.full(3, 1e-3)
    zl, _ = ipm.kappa_sigma_reset(nlp, x, np.array([5.0, 1e13, 1e-9]), np.zeros(3), 0.1, OPT)
    assert zl[0] == 5.0
    assert zl[1] == rel(1e12, 1e-12)
    assert zl[2] == rel(1e-8, 1e-12)


def test_initial_point_bound_push():
    """kappa_1 = kappa_2 = 1e-2 on the box [0, 2.4525]: p_L = min(1e-2 max(1, 0),
    1e-2 * 2.4525) = 0.01 and p_U = min(1e-2 * 2.4525, 0.024525) = 0.024525, so 0 -> 0.01
    and 2.4525 -> 2.427975; a lower-bounded x = -1 -> 0.01; a free variable is kept."""
    u = 2.4525
    nlp = TorchNLP(lambda x: x.sum(), None, 4, 0, xl=[0.0, 0.0, 0.0, -np.inf], xu=[u, u, np.inf, np.inf])
    st = ipm.initial_state(nlp, np.array([0.0, u, -1.0, -7.0]), OPT)
    assert st.normal.x[0] == rel(0.01, 1e-15)
    assert st.normal.x[1] == rel(2.427975, 1e-14)
    assert st.normal.x[2] == rel(0.01, 1e-15)
    assert st.normal.x[3] == -7.0
    assert list(st.normal.zl) == [1.0, 1.0, 1.0, 0.0] and list(st.normal.zu) == [1.0, 1.0, 0.0, 0.0]


def test_least_squares_multipliers_and_cap():
    """J = (1, 1), grad f = (1, 3), z = 0: y minimises |g + J^T y| -> y = -(1 + 3)/2 = -2.
    With grad f = (3000, 3000), y = -3000 exceeds y_max = 1e3 and is replaced by 0."""
    nlp = TorchNLP(lambda x: x.sum(), lambda x: (x[0] + x[1]).reshape(1), 2, 1)
    J = np.array([[1.0, 1.0]])
    y = ipm.least_squares_y(nlp, np.array([1.0, 3.0]), J, np.zeros(2), np.zeros(2), OPT)
    assert y[0] == rel(-2.0, 1e-14)
    y = ipm.least_squares_y(nlp, np.array([3000.0, 3000.0]), J, np.zeros(2), np.zeros(2), OPT)
    assert y[0] == 0.0


# --------------------------------------------------------- error measure --

def test_scaled_optimality_error_by_hand():
    """Three variables: x0 in [0, 1] (two bounds), x1 and x2 free (n = 3, n_b = 2);
    one equality with J = (1, 2, 0).  x = (0.5, 0, 0), y = (300), z_L = (200, 0, 0),
    z_U = (50, 0, 0), grad f = (1, 0, 0), c = (0.02), mu = 24.
    |z|_1 = 250, |y|_1 = 300: s_d = max(100, 550 / (m + n_b) = 183.33) / 100 = 1.8333,
    s_c = max(100, 250 / n_b = 125) / 100 = 1.25.
    grad L = g + J^T y - z_L + z_U = (151, 600, 0): dual = 600 / 1.8333 = 327.27.
    comp: |0.5 * 200 - 24| = 76, |0.5 * 50 - 24| = 1: 76 / 1.25 = 60.8.
    E_24 = max(327.27, 0.02, 60.8) = 327.27.
    With y = 0 and grad f = (150, 0, 0): grad L = 0, E_24 = 60.8; at mu = 0 the
    complementarity is 100 and 25: E_0 = 100 / 1.25 = 80."""
    nlp = TorchNLP(lambda x: x.sum(), lambda x: (x[0] + 2 * x[1]).reshape(1), 3, 1,
                   xl=[0.0, -np.inf, -np.inf], xu=[1.0, np.inf, np.inf])
    x = np.array([0.5, 0.0, 0.0])
    zl, zu = np.array([200.0, 0.0, 0.0]), np.array([50.0, 0.0, 0.0])
    J = np.array([[1.0, 2.0, 0.0]])
    c = np.array([0.02])
    e = ipm.opt_error(nlp, x, np.array([300.0]), zl, zu, np.array([1.0, 0.0, 0.0]), J, c, 24.0, OPT)
    assert e == rel(600.0 / (550.0 / 300.0), 1e-14)
    g0 = np.array([150.0, 0.0, 0.0])
    assert ipm.opt_error(nlp, x, np.array([0.0]), zl, zu, g0, J, c, 24.0, OPT) == rel(76.0 / 1.25, 1e-14)
    assert ipm.opt_error(nlp, x, np.array([0.0]), zl, zu, g0, J, c, 0.0, OPT) == rel(80.0, 1e-14)


# --------------------------------------------------------- barrier update --

def test_barrier_update_fast_decrease_loop():
    """kappa_mu = 0.2, theta_mu = 1.5, kappa_eps = 10.  mu_+ = min(0.2 mu, mu^1.5):
    0.1 -> 0.02 -> 0.02^1.5 = 0.0028284 -> 0.0028284^1.5 = 1.50424e-4 -> ...
    With a fixed E_mu = 0.01 the loop continues while 0.01 <= 10 mu: it stops at
    1.50424e-4 (0.01 > 1.5e-3) after three decreases.  With E_mu = 0 it reaches the
    floor tol / 10 = 1e-7: 1.50424e-4^1.5 = 1.84493e-6, then max(1e-7, 2.5e-9) = 1e-7."""
    mu, dec, stall = ipm.barrier_update(0.1, lambda m: 0.01, False, OPT)
    assert dec and not stall
    assert mu == rel((0.02 ** 1.5) ** 1.5, 1e-14)
    assert mu == rel(1.504241e-4, 1e-6)
    mu, dec, stall = ipm.barrier_update(0.1, lambda m: 0.0, False, OPT)
    assert mu == 1e-7 and dec and not stall
    # not solved: no change
    mu, dec, stall = ipm.barrier_update(0.1, lambda m: 5.0, False, OPT)
    assert mu == 0.1 and not dec and not stall


def test_barrier_update_after_a_tiny_step():
    """A tiny step forces one decrease even if E_mu > kappa_eps mu; at the floor it is
    reported as a stall (status TINY_STEP)."""
    mu, dec, stall = ipm.barrier_update(0.1, lambda m: 5.0, True, OPT)
    assert mu == rel(0.02, 1e-15) and dec and not stall
    mu, dec, stall = ipm.barrier_update(1e-7, lambda m: 5.0, True, OPT)
    assert stall and mu == 1e-7


# ------------------------------------------------------- inertia correction --

def test_inertia_correction_sequence():
    """Algorithm IC.  A matrix that needs delta_w >= 0.5:
    * no previous delta_w: 0 (fails), 1e-4, 1e-2 (x100), 1 (x100) -> 1.0 after 3 retries;
    * previous delta_w = 0.3: max(1e-20, 0.3/3) = 0.1 (fails), x8 = 0.8 -> 0.8 after 2;
    * previous delta_w = 3e-21: max(1e-20, 1e-21) = 1e-20 is the floor.
    A matrix no delta_w fixes ends when delta_w would pass 1e40."""
    seen = []

    def need(th):
        def ok(dw):
            seen.append(dw)
            return dw >= th
        return ok

    dw, n = ipm.inertia_correction(need(0.5), 0.0, OPT)
    assert dw == rel(1.0, 1e-12) and n == 3
    assert seen == [0.0, 1e-4, pytest.approx(1e-2), pytest.approx(1.0)]
    dw, n = ipm.inertia_correction(need(0.5), 0.3, OPT)
    assert dw == rel(0.8, 1e-12) and n == 2
    seen.clear()
    dw, n = ipm.inertia_correction(need(1.0), 3e-21, OPT)
    assert seen[1] == 1e-20
    dw, n = ipm.inertia_correction(lambda d: False, 0.0, OPT)
    assert dw is None
    # 1e-4 * 100^k <= 1e40 for k <= 22: 23 retries, then 1e-4 * 100^23 = 1e42 > 1e40
    assert n == 23
    assert ipm.inertia_correction(lambda d: True, 0.7, OPT) == (0.0, 0)


# ------------------------------------------------------- restoration entry --

@pytest.mark.parametrize("c", [-3.0, 0.0, 1e-8, 5.0, 1234.5])
def test_restoration_elastics_solve_their_optimality_conditions(c):
    """p, n minimise rho (p + n) - mu (ln p + ln n) on p - n = c: p, n > 0, c - p + n = 0,
    and the two stationarity conditions rho - mu/p - lam = 0, rho - mu/n + lam = 0 add
    to mu/p + mu/n = 2 rho."""
    rho, mu = 1000.0, 0.37
    p, n = ipm.resto_elastics(np.array([c]), mu, rho)
    p, n = float(p[0]), float(n[0])
    assert p > 0 and n > 0
    assert c - p + n == pytest.approx(0.0, abs=1e-12 * max(1.0, abs(c)))
    assert mu / p + mu / n == rel(2 * rho, 1e-9)


def test_restoration_start_state():
    """Entering restoration at x with c(x) = (0.5, -2), mu = 0.04: mu_R = max(mu,
    |c|_inf) = 2, zeta = sqrt(0.04) = 0.2, y = 0, z_p = mu_R / p, z_n = mu_R / n, z_x clipped
    at rho = 1000, and the original filter gains the entry of (theta, phi)."""
    import torch

    b = torch.tensor([0.5, -2.0], dtype=torch.float64)
    nlp = TorchNLP(lambda x: (x ** 2).sum(), lambda x: x[:2] - b, 3, 2, xl=[0.0, -np.inf, -np.inf],
                   xu=[np.inf] * 3)
    st = ipm.initial_state(nlp, np.array([1.0, 0.0, 0.0]), OPT)
    st.normal.mu = 0.04
    st.normal.zl = np.array([5000.0, 0.0, 0.0])
    st.normal.theta_max = 1e4
    ipm.resto_start(nlp, st, OPT)
    r = st.resto
    assert st.mode == ipm.RESTO
    assert r.mu == 2.0 and st.zeta == rel(0.2, 1e-15)
    assert np.all(r.y == 0)
    p, n = r.x[3:5], r.x[5:7]
    assert np.allclose(nlp.c(r.x[:3]) - p + n, 0.0, atol=1e-14)
    assert np.allclose(r.zl[3:5] * p, 2.0) and np.allclose(r.zl[5:7] * n, 2.0)
    assert r.zl[0] == 1000.0
    theta = 0.5 + 2.0
    phi = ipm.barrier_phi(nlp, st.normal.x, nlp.f(st.normal.x), 0.04, OPT)
    assert st.normal.filt[-1] == pytest.approx(ipm.filter_entry(theta, phi, OPT))
    assert np.allclose(ipm.resto_scaling(np.array([0.5, -4.0, 0.0])), [1.0, 0.25, 1.0])


def test_restoration_return_test():
    """Return when theta <= 0.9 theta(x_R) and the point is not in the original filter."""
    ph = _phase([(0.5, 1.0)], theta_max=100.0)
    assert ipm.resto_may_return(ph, 0.45, 0.0, 1.0, OPT)      # 0.45 <= 0.9, not in filter
    assert not ipm.resto_may_return(ph, 0.95, 0.0, 1.0, OPT)  # not enough reduction
    assert not ipm.resto_may_return(ph, 0.6, 2.0, 1.0, OPT)   # dominated by (0.5, 1)
    assert not ipm.resto_may_return(ph, 0.1, np.inf, 1.0, OPT)
    assert math.isclose(OPT.kappa_resto, 0.9)


# ------------------------------------- watchdog and soft restoration (rows 3, 5) --

def test_primal_dual_error_by_hand():
    """x0 in [0, 1], x1 free; J = (1, 2); x = (0.25, 3), y = (2), z_L = (4, 0), z_U = (1, 0),
    grad f = (0.5, -1), c = (0.1), mu = 0.5.
    grad L = g + J^T y - z_L + z_U = (0.5 + 2 - 4 + 1, -1 + 4) = (-0.5, 3): |.|_1 = 3.5.
    complementarity: |0.25 * 4 - 0.5| = 0.5, |0.75 * 1 - 0.5| = 0.25.
    E_pd = 3.5 + 0.1 + 0.75 = 4.35."""
    nlp = TorchNLP(lambda x: x.sum(), lambda x: (x[0] + 2 * x[1]).reshape(1), 2, 1,
                   xl=[0.0, -np.inf], xu=[1.0, np.inf])
    e = ipm.primal_dual_error(nlp, np.array([0.25, 3.0]), np.array([2.0]), np.array([4.0, 0.0]),
                              np.array([1.0, 0.0]), np.array([0.5, -1.0]), np.array([[1.0, 2.0]]),
                              np.array([0.1]), 0.5)
    assert e == rel(4.35, 1e-14)


def test_soft_restoration_acceptance_threshold():
    """kappa_soft = 1e-4: accept when E_pd(trial) <= 0.9999 E_pd(current)."""
    assert ipm.soft_resto_accepts(0.9999, 1.0, OPT)
    assert not ipm.soft_resto_accepts(0.99995, 1.0, OPT)
    assert ipm.soft_resto_accepts(0.5, 1.0, OPT)


def test_watchdog_start_and_end_rules():
    """The watchdog starts after 10 consecutive shortened steps when it is enabled;
    a barrier decrease or restoration entry ends it and the soft phase."""
    opt = ipm.Options(watchdog=True)
    ph = _phase()
    ph.wd_short = 9
    assert not ipm.watchdog_should_start(ph, opt)
    ph.wd_short = 10
    assert ipm.watchdog_should_start(ph, opt)
    assert not ipm.watchdog_should_start(ph, OPT)  # disabled by default
    ph.wd_active, ph.wd_trials, ph.wd_store = True, 2, {"x": 0}
    assert not ipm.watchdog_should_start(ph, opt)
    ph.soft_active, ph.soft_iters = True, 3
    ipm.end_globalization(ph)
    assert (ph.wd_active, ph.wd_trials, ph.wd_store, ph.wd_short) == (False, 0, None, 0)
    assert (ph.soft_active, ph.soft_iters) == (False, 0)


def _nonconvex_chain():
    """min sum (x_i - 2)^2 s.t. x_i^2 + x_{i+1}^2 = 1 (i = 0, 1): curved constraints whose
    steps are often shortened."""
    import torch

    n = 3
    return TorchNLP(lambda x: ((x - 2.0) ** 2).sum(),
                    lambda x: torch.stack([x[0] ** 2 + x[1] ** 2 - 1.0, x[1] ** 2 + x[2] ** 2 - 1.0]), n, 2,
                    x0=[3.0, -2.0, 1.5])


def test_watchdog_first_step_is_the_full_step():
    """Once started, the watchdog takes the full step alpha_max: the new iterate is
    x + alpha_max dx whether or not the filter tests accept it, and the stored
    iterate is the one it started from."""
    nlp = _nonconvex_chain()
    opt = ipm.Options(watchdog=True)
    st = ipm.initial_state(nlp, nlp.default_start(), opt)
    tr = {}
    ipm.phase_iteration(nlp, st.normal, opt, tr, init_theta=True, y_ls=True, globalize=True)
    x0 = st.normal.x.copy()
    st.normal.wd_short = opt.wd_trigger
    tr = {}
    out = ipm.phase_iteration(nlp, st.normal, opt, tr, globalize=True)
    assert out == ipm._Outcome.ACCEPTED and tr.get("wd_start")
    ph = st.normal
    if tr.get("wd_accepted"):
        assert not ph.wd_active
    else:
        assert tr.get("wd_step") and ph.wd_active and ph.wd_trials == 1
        assert np.array_equal(ph.wd_store["x"], x0)
        # the accepted step is the full one along the stored direction
        assert np.allclose(ph.x, x0 + ph.wd_store["a_max"] * ph.wd_store["dx"], rtol=0, atol=1e-15)
    assert tr["alpha"] == pytest.approx(tr["alpha"])


def test_watchdog_gives_up_after_the_trial_steps_and_backtracks_from_the_stored_point():
    """A watchdog whose reference values no trial can satisfy (theta_W = phi_W = -inf
    rejects every point) takes wd_trial_max = 3 unconditional steps and then returns
    to the stored iterate, searching along its stored step from half its full step."""
    nlp = _nonconvex_chain()
    opt = ipm.Options(watchdog=True)
    st = ipm.initial_state(nlp, nlp.default_start(), opt)
    ph = st.normal
    ipm.phase_iteration(nlp, ph, opt, {}, init_theta=True, y_ls=True, globalize=True)
    ph.wd_short = opt.wd_trigger
    # a filter entry that dominates every point: no trial passes the filter test
    ph.filt = [(-1.0, -np.inf)]
    x_start = ph.x.copy()
    steps = []
    for _ in range(opt.wd_trial_max + 1):
        tr = {}
        ipm.phase_iteration(nlp, ph, opt, tr, globalize=True)
        steps.append(tr)
        if ph.wd_store is not None:
            W = ph.wd_store
        if ph.mu != steps[0].get("mu", ph.mu):
            break
    assert steps[0].get("wd_start")
    assert [bool(t.get("wd_step")) for t in steps[:3]] == [True, True, True]
    assert steps[3].get("wd_return")
    assert not ph.wd_active and ph.wd_store is None
    # the search ran from the stored point along its step: every trial was
    # rejected by the filter, so the line search failed there
    assert np.array_equal(W["x"], x_start)


def test_soft_restoration_step_reduces_the_primal_dual_error():
    """On the Wachter-Biegler problem the line search fails and soft restoration
    (Table I row 5) is tried before hard restoration.  Every soft step recorded must
    use alpha_s = min(alpha_max, alpha_z_max) for primal and dual alike, and an
    accepted one must lower E_pd, recomputed here at the recorded trial point
    x + alpha_s dx (multipliers likewise), by the factor 1 - 1e-4."""
    import torch

    nlp = TorchNLP(lambda x: x[0], lambda x: torch.stack([x[0] ** 2 - x[1] - 1.0, x[0] - x[2] - 0.5]), 3, 2,
                   xl=[-np.inf, 0.0, 0.0], xu=[np.inf] * 3, x0=[-2.0, 1.0, 1.0])
    opt = ipm.Options(soft_resto=True, trace_soc=True)
    st = ipm.initial_state(nlp, nlp.default_start(), opt)
    tried, checked = 0, 0
    for _ in range(40):
        if st.mode != ipm.NORMAL or st.status != ipm.RUNNING:
            break
        tr = ipm.step(nlp, st, opt)
        tried += bool(tr.get("soft_trial"))
        L = tr.get("soft_log")
        if L is None:
            continue
        assert L["alpha"] == min(L["a_max"], L["az_max"])
        a = L["alpha"]
        xt, yt = L["x"] + a * L["dx"], L["y"] + a * L["dy"]
        zlt, zut = L["zl"] + a * L["dzl"], L["zu"] + a * L["dzu"]
        e_t = ipm.primal_dual_error(nlp, xt, yt, zlt, zut, nlp.grad_f(xt), nlp.jac_c(xt), nlp.c(xt), L["mu"])
        assert e_t == rel(L["e_trial"], 1e-12)
        if tr.get("soft_step"):
            checked += 1
            assert e_t <= (1 - opt.kappa_soft) * L["e_current"]
    assert tried >= 1


# ------------------------------------------ adaptive barrier update (row 7) --

def test_loqo_centrality_rule():
    """xi = min / average; sigma = 0.1 min(0.05 (1 - xi) / xi, 2)^3; mu = sigma * average.
    avg = 1, min = 0.5: xi = 0.5, 0.05 * 0.5 / 0.5 = 0.05, sigma = 0.1 * 1.25e-4 = 1.25e-5.
    avg = 2, min = 0.02: xi = 0.01, 0.05 * 0.99 / 0.01 = 4.95 -> 2, sigma = 0.8, mu = 1.6.
    Perfect centrality (min = avg) gives mu = 0."""
    assert ipm.loqo_mu(1.0, 0.5) == rel(1.25e-5, 1e-12)
    assert ipm.loqo_mu(2.0, 0.02) == rel(1.6, 1e-14)
    assert ipm.loqo_mu(3.0, 3.0) == 0.0
    assert ipm.loqo_mu(1.0, 0.0) == rel(0.8, 1e-15)


def test_complementarity_statistics():
    """x0 in [0, 2] at 0.5 with z_L = 2, z_U = 1; x1 >= 0 at 3 with z_L = 0.1: products
    1.0, 1.5 and 0.3 -> average 0.9333, minimum 0.3."""
    nlp = TorchNLP(lambda x: x.sum(), None, 2, 0, xl=[0.0, 0.0], xu=[2.0, np.inf])
    avg, mn = ipm.complementarity_stats(nlp, np.array([0.5, 3.0]), np.array([2.0, 0.1]), np.array([1.0, 0.0]))
    assert avg == rel(2.8 / 3.0, 1e-15) and mn == rel(0.3, 1e-15)


def test_progress_test_and_references():
    """Progress: E_0 <= 0.9999 max(refs); empty refs always progress; at most four kept."""
    refs = []
    assert ipm.sufficient_progress(5.0, refs, OPT)
    for e in (4.0, 3.0, 2.0, 1.0, 0.5):
        ipm.remember_reference(refs, e, OPT)
    assert refs == [3.0, 2.0, 1.0, 0.5]
    assert ipm.sufficient_progress(2.9997, refs, OPT)
    assert not ipm.sufficient_progress(2.9998, refs, OPT)


def test_adaptive_barrier_update_modes():
    """Free mode with progress: mu = LOQO, clipped to [1e-11, mu_max]; without progress
    (or after a tiny step) the fixed mode starts at 0.8 * average complementarity;
    fixed mode returns to free mode once the barrier problem is solved with progress,
    and otherwise follows the monotone rule."""
    opt = ipm.Options(mu_strategy="adaptive")
    ph = _phase()
    ph.mu, ph.mu_max = 0.1, 10.0
    mu, changed, stall = ipm.adaptive_barrier_update(ph, 1.0, lambda m: 0.0, 2.0, 0.02, False, opt)
    assert (mu, ph.mu_free, ph.mu_refs) == (pytest.approx(1.6), True, [1.0]) and changed and not stall
    ph.mu = mu
    ph.mu_max = 1.0  # the cap applies
    mu, _, _ = ipm.adaptive_barrier_update(ph, 0.5, lambda m: 0.0, 2.0, 0.02, False, opt)
    assert mu == 1.0 and ph.mu_refs == [1.0, 0.5]
    ph.mu = mu
    # no progress (0.99995 > 0.9999 * 1.0): fixed mode at 0.8 * average
    mu, changed, _ = ipm.adaptive_barrier_update(ph, 0.99995, lambda m: 0.0, 0.5, 0.1, False, opt)
    assert not ph.mu_free and mu == rel(0.4, 1e-15) and changed
    ph.mu = mu
    # fixed mode, barrier problem not solved (E_mu > 10 mu): unchanged
    mu, changed, _ = ipm.adaptive_barrier_update(ph, 0.1, lambda m: 100.0, 0.5, 0.1, False, opt)
    assert mu == 0.4 and not changed and not ph.mu_free
    # solved, but no progress against the references: the monotone rule, whose fast
    # decrease (E_mu = 0 at every mu) runs down to the floor tol / 10
    mu, changed, _ = ipm.adaptive_barrier_update(ph, 5.0, lambda m: 0.0, 0.5, 0.1, False, opt)
    assert changed and not ph.mu_free and mu == 1e-7
    ph.mu = mu
    # solved with progress: free mode again, references restart from E_0
    mu, changed, _ = ipm.adaptive_barrier_update(ph, 0.1, lambda m: 0.0, 2.0, 0.02, False, opt)
    assert ph.mu_free and ph.mu_refs == [0.1] and mu == rel(1.0, 1e-15)  # LOQO 1.6 capped at 1.0
    # a tiny step in free mode switches to the fixed mode
    ph.mu = mu
    ipm.adaptive_barrier_update(ph, 0.01, lambda m: 0.0, 0.5, 0.1, True, opt)
    assert not ph.mu_free
