"""Plain FP64 interior-point iteration, one problem at a time (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

This follows the paper's review of IPOPT (Sec. IV) step by step:

* barrier objective phi_mu (Eq. 3) with IPOPT's linear damping term for
  variables bounded on one side only (the footnote of Sec. IV points to
  IPOPT's handling of one-sided bounds);
* Lagrangian and iterate (x, y_c, z_L, z_U) (Eq. 4);
* optimality conditions (Eq. 5) measured by IPOPT's scaled error E_mu;
* Newton system (Eq. 6) reduced to the augmented system (Eq. 7) by
  eliminating the bound-multiplier steps (text after Eq. 6), solved by a
  symmetric indefinite LDL^T whose inertia is checked and corrected by the
  regularisation delta_x I (text after Eq. 7; IPOPT's Algorithm IC);
* the branches of Table I: (1) backtracking filter line search,
  (2) second-order correction, (3) the watchdog and (5) soft feasibility
  restoration (options, off by default; the original problem only),
  (4) tiny step, (6) hard feasibility restoration (a nested interior-point
  solve of the l1 restoration problem; a restoration inside restoration is
  reported as a failure), and (7) the monotone barrier update.  The adaptive
  barrier rule is not part of this method.

Every constant is IPOPT's published default as listed in ``Options``.
One call of ``step`` is one iteration; the complete state between iterations
is ``SolverState`` (the state-injection test of Sec. VI, Eq. 8, loads it).
"""

from __future__ import annotations

import copy
import dataclasses
import math

import numpy as np
from scipy.linalg import eigvalsh_tridiagonal, ldl, solve_triangular

# status codes (shared meaning with the library, not shared code)
RUNNING, CONVERGED, MAX_ITER, RESTO_FAILED, EVAL_ERROR, TINY_STEP = 0, 1, 2, 3, 4, 5
NORMAL, RESTO = 0, 1
EPS_MACH = np.finfo(np.float64).eps


@dataclasses.dataclass
class Options:
    tol: float = 1e-6
    max_iter: int = 500
    mu_init: float = 0.1
    s_max: float = 100.0
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    kappa_sigma: float = 1e10
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-8
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-8
    gamma_alpha: float = 0.05
    kappa_soc: float = 0.99
    p_max: int = 4
    kappa_d: float = 1e-4
    dw_init: float = 1e-4
    dw_min: float = 1e-20
    dw_max: float = 1e40
    kappa_w_minus: float = 1.0 / 3.0
    kappa_w_plus: float = 8.0
    kappa_w_plus_bar: float = 100.0
    bound_push: float = 1e-2
    bound_frac: float = 1e-2
    y_max: float = 1e3
    z_init: float = 1.0
    z_centred: bool = False  # warm start: z = mu_init / (distance to the bound) instead of z_init
    rho: float = 1000.0
    kappa_resto: float = 0.9
    filter_cap: int = 64
    ls_max_trials: int = 60
    trace_cond: bool = False  # record the 2-norm condition number of each step's matrix
    trace_soc: bool = False   # record the linear systems of the second-order corrections
    # watchdog (Table I row 3) and soft feasibility restoration (row 5); off by default
    watchdog: bool = False
    wd_trigger: int = 10      # consecutive shortened steps that start the watchdog
    wd_trial_max: int = 3     # unconditional steps before the watchdog gives up
    soft_resto: bool = False
    kappa_soft: float = 1e-4  # required relative decrease of the primal-dual error
    soft_max: int = 10        # soft restoration steps before hard restoration
    # barrier update (Table I row 7): "monotone" (Fiacco-McCormick) or "adaptive"
    # (free mode with the LOQO centrality rule, monotone fallback)
    mu_strategy: str = "monotone"
    mu_min_adaptive: float = 1e-11   # floor of mu in free mode
    mu_max_fact: float = 1e3         # mu <= mu_max_fact * (average complementarity at the start)
    refs_red_fact: float = 0.9999    # required reduction of E_0 against the reference values
    num_refs_max: int = 4            # reference values kept
    mu_monotone_init: float = 0.8    # fixed mode starts at this fraction of the average complementarity


@dataclasses.dataclass
class Phase:
    """Iterate and line-search memory of one barrier solve (original or restoration)."""

    x: np.ndarray
    y: np.ndarray
    zl: np.ndarray
    zu: np.ndarray
    mu: float
    filt: list
    theta_max: float = 0.0
    theta_min: float = 0.0
    dw_last: float = 0.0
    tiny: bool = False
    # watchdog: consecutive shortened steps, active flag, unconditional steps
    # taken, and the stored iterate with its step and reference values
    wd_short: int = 0
    wd_active: bool = False
    wd_trials: int = 0
    wd_store: dict | None = None
    # soft restoration: active flag and soft steps taken in the current phase
    soft_active: bool = False
    soft_iters: int = 0
    # adaptive barrier update: free mode flag, reference values of E_0 and the cap of mu
    mu_free: bool = True
    mu_refs: list = dataclasses.field(default_factory=list)
    mu_max: float = 0.0


@dataclasses.dataclass
class SolverState:
    normal: Phase
    mode: int = NORMAL
    resto: Phase | None = None
    x_ref: np.ndarray | None = None      # x_R, the point where restoration started
    zeta: float = 0.0
    need_init: bool = True               # theta_max/theta_min and y still to be set
    need_y_ls: bool = True               # least-squares y at the next evaluation
    iter: int = 0
    status: int = RUNNING
    # counters (reported, not part of the algorithm)
    n_soc: int = 0
    n_resto_iter: int = 0
    n_inertia_corr: int = 0
    n_tiny: int = 0


# ---------------------------------------------------------------- helpers --

def bound_sets(nlp):
    has_l = np.isfinite(nlp.xl)
    has_u = np.isfinite(nlp.xu)
    return has_l, has_u


def slacks(nlp, x):
    """s_L = x - x_L and s_U = x_U - x on the bounded components (0 elsewhere)."""
    has_l, has_u = bound_sets(nlp)
    sl = np.where(has_l, x - np.where(has_l, nlp.xl, 0.0), 0.0)
    su = np.where(has_u, np.where(has_u, nlp.xu, 0.0) - x, 0.0)
    return sl, su


def barrier_phi(nlp, x, f, mu, opt):
    """phi_mu (Eq. 3) plus kappa_d * mu * (distance to the only bound) per one-sided variable."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    if np.any(sl[has_l] <= 0) or np.any(su[has_u] <= 0):
        return np.inf
    val = f - mu * np.sum(np.log(sl[has_l])) - mu * np.sum(np.log(su[has_u]))
    only_l = has_l & ~has_u
    only_u = has_u & ~has_l
    val += opt.kappa_d * mu * (np.sum(sl[only_l]) + np.sum(su[only_u]))
    return val


def barrier_grad(nlp, x, g, mu, opt):
    """Gradient of barrier_phi: grad f - mu S_L^{-1} e + mu S_U^{-1} e (+ damping)."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    out = g.copy()
    out[has_l] -= mu / sl[has_l]
    out[has_u] += mu / su[has_u]
    only_l = has_l & ~has_u
    only_u = has_u & ~has_l
    out[only_l] += opt.kappa_d * mu
    out[only_u] -= opt.kappa_d * mu
    return out


def theta_of(c):
    """Constraint violation used by the filter: l1 norm of c."""
    return float(np.sum(np.abs(c)))


def opt_error(nlp, x, y, zl, zu, g, J, c, mu, opt):
    """IPOPT's scaled optimality error E_mu of the conditions Eq. 5."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    grad_lag = g + J.T @ y - zl + zu
    nb = int(has_l.sum() + has_u.sum())
    z1 = float(np.sum(np.abs(zl[has_l])) + np.sum(np.abs(zu[has_u])))
    s_d = max(opt.s_max, (float(np.sum(np.abs(y))) + z1) / max(1, nlp.m + nb)) / opt.s_max
    s_c = max(opt.s_max, z1 / max(1, nb)) / opt.s_max
    e_dual = float(np.max(np.abs(grad_lag))) / s_d if grad_lag.size else 0.0
    e_prim = float(np.max(np.abs(c))) if c.size else 0.0
    comp = 0.0
    if has_l.any():
        comp = max(comp, float(np.max(np.abs(sl[has_l] * zl[has_l] - mu))))
    if has_u.any():
        comp = max(comp, float(np.max(np.abs(su[has_u] * zu[has_u] - mu))))
    return max(e_dual, e_prim, comp / s_c)


def frac_to_boundary(v, dv, tau):
    """Largest alpha in (0, 1] with v + alpha dv >= (1 - tau) v, over components with dv < 0."""
    neg = dv < 0
    if not np.any(neg):
        return 1.0
    return float(min(1.0, np.min(-tau * v[neg] / dv[neg])))


def is_tiny_step(x, dx):
    """Tiny-step test (Table I row 4): max_i |dx_i| / (1 + |x_i|) < 10 eps_mach."""
    return bool(np.max(np.abs(dx) / (1.0 + np.abs(x))) < 10.0 * EPS_MACH)


# ----------------------------------------------------- line-search rules --
# The acceptance rules of the backtracking filter line search (Table I row 1;
# IPOPT's Algorithm A with its Eqs. for the switching condition, the Armijo
# and sufficient-decrease tests and the minimal step size).  theta is the
# constraint violation and phi the barrier objective at the current iterate,
# gdx = grad phi^T dx the directional derivative along the primal step.

def alpha_min(theta, gdx, theta_min, opt):
    """Smallest trial step before the line search gives up (IPOPT's Eq. 23, three cases)."""
    if gdx < 0 and theta <= theta_min:
        return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta / (-gdx),
                                     opt.delta * theta ** opt.s_theta / (-gdx) ** opt.s_phi)
    if gdx < 0:
        return opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta / (-gdx))
    return opt.gamma_alpha * opt.gamma_theta


def switching_condition(alpha, gdx, theta, opt):
    """gdx < 0 and alpha (-gdx)^s_phi > delta theta^s_theta."""
    return gdx < 0 and alpha * (-gdx) ** opt.s_phi > opt.delta * theta ** opt.s_theta


def armijo_holds(phi_t, phi0, alpha, gdx, opt):
    """Armijo condition on the barrier objective: phi(x_a) <= phi + eta_phi alpha gdx."""
    return phi_t <= phi0 + opt.eta_phi * alpha * gdx


def sufficient_decrease(theta_t, phi_t, theta, phi0, opt):
    """Sufficient reduction of theta or phi with respect to the current iterate."""
    return theta_t <= (1.0 - opt.gamma_theta) * theta or phi_t <= phi0 - opt.gamma_phi * theta


def trial_acceptable(ph, theta_t, phi_t, alpha, theta, phi0, gdx, opt):
    """A trial point is accepted if it is not in the filter and, when the switching
    condition holds at a nearly feasible iterate (theta <= theta_min), satisfies the
    Armijo condition, otherwise the sufficient-decrease test."""
    if not np.isfinite(phi_t) or in_filter(ph, theta_t, phi_t):
        return False
    if switching_condition(alpha, gdx, theta, opt) and theta <= ph.theta_min:
        return armijo_holds(phi_t, phi0, alpha, gdx, opt)
    return sufficient_decrease(theta_t, phi_t, theta, phi0, opt)


def filter_needs_augment(alpha, phi_t, phi0, gdx, theta, opt):
    """The filter is augmented after an accepted step unless the switching condition
    and the Armijo condition both hold."""
    return not (switching_condition(alpha, gdx, theta, opt) and armijo_holds(phi_t, phi0, alpha, gdx, opt))


def filter_entry(theta, phi, opt):
    """The pair stored in the filter for an iterate with (theta, phi)."""
    return (1.0 - opt.gamma_theta) * theta, phi - opt.gamma_phi * theta


def soc_constraint_rhs(alpha_prev, c_soc_prev, c_trial):
    """Right-hand side of the next second-order correction (Table I row 2):
    c_soc <- alpha c_soc + c(x_soc); the first one is alpha c(x) + c(x_alpha)."""
    return alpha_prev * c_soc_prev + c_trial


def soc_should_stop(p, theta_soc, theta_old, opt):
    """Stop correcting after p_max corrections or when theta no longer shrinks by kappa_soc."""
    return p >= opt.p_max or theta_soc > opt.kappa_soc * theta_old


def primal_dual_error(nlp, x, y, zl, zu, g, J, c, mu):
    """1-norm primal-dual error of the barrier problem at mu (the conditions of
    Eq. 5 with mu): |grad L|_1 + |c|_1 + |S_L z_L - mu e|_1 + |S_U z_U - mu e|_1.
    Soft restoration accepts a step that reduces it."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    gl = g + J.T @ y - zl + zu
    comp = float(np.sum(np.abs(sl[has_l] * zl[has_l] - mu)) + np.sum(np.abs(su[has_u] * zu[has_u] - mu)))
    return float(np.sum(np.abs(gl)) + np.sum(np.abs(c))) + comp


def soft_resto_accepts(e_trial, e_current, opt):
    """Soft restoration's acceptance: E_pd(trial) <= (1 - kappa_soft) E_pd(current)."""
    return e_trial <= (1.0 - opt.kappa_soft) * e_current


def watchdog_should_start(ph, opt):
    """The watchdog starts after wd_trigger consecutive shortened steps."""
    return opt.watchdog and not ph.wd_active and ph.wd_short >= opt.wd_trigger


def end_globalization(ph):
    """A barrier-parameter decrease (or entering restoration) ends an active watchdog
    and soft restoration and clears the shortened-step count."""
    ph.wd_active, ph.wd_trials, ph.wd_store, ph.wd_short = False, 0, None, 0
    ph.soft_active, ph.soft_iters = False, 0


# ------------------------------------------------------ barrier update --

def barrier_update(mu, err_at, tiny, opt):
    """Monotone barrier update (Table I row 7, monotone schedule).

    While the barrier problem at mu is solved to E_mu <= kappa_eps mu (err_at(mu)
    is E_mu), or once after a tiny step, mu <- max(tol/10, min(kappa_mu mu,
    mu^theta_mu)) and the filter is reset.  Returns (mu, decreased, stalled):
    stalled means a tiny step happened at the floor value of mu."""
    mu_floor = opt.tol / 10.0
    first = True
    decreased = False
    while True:
        if (err_at(mu) <= opt.kappa_eps * mu) or (first and tiny):
            if mu <= mu_floor:
                return mu, decreased, bool(first and tiny)
            mu = max(mu_floor, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
            decreased = True
            first = False
            tiny = False
            continue
        return mu, decreased, False


def complementarity_stats(nlp, x, zl, zu):
    """(average, minimum) of the complementarity products s_i z_i over all bounds."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    prod = np.concatenate([sl[has_l] * zl[has_l], su[has_u] * zu[has_u]])
    if prod.size == 0:
        return 0.0, 0.0
    return float(np.mean(prod)), float(np.min(prod))


def loqo_mu(avg, minimum):
    """LOQO's centrality rule (Vanderbei & Shanno): mu = sigma * average
    complementarity with sigma = 0.1 min(0.05 (1 - xi) / xi, 2)^3, xi = min / average."""
    if avg <= 0.0:
        return 0.0
    xi = minimum / avg
    t = min(0.05 * (1.0 - xi) / xi, 2.0) if xi > 0 else 2.0
    return 0.1 * t * t * t * avg


def sufficient_progress(err, refs, opt):
    """Free-mode progress: E_0 at most refs_red_fact times the largest of the stored
    reference values (no reference yet counts as progress)."""
    return not refs or err <= opt.refs_red_fact * max(refs)


def remember_reference(refs, err, opt):
    """Append E_0 of an accepted free-mode iterate; keep the last num_refs_max."""
    refs.append(err)
    if len(refs) > opt.num_refs_max:
        refs.pop(0)


def adaptive_barrier_update(ph, err0, err_at, avg, minimum, tiny, opt):
    """Adaptive barrier update (Table I row 7).  Free mode: mu = max(mu_min, min(mu_max,
    LOQO(x))) every iteration while E_0 keeps falling (sufficient_progress); without
    progress, or after a tiny step, the fixed (monotone) mode starts at mu =
    mu_monotone_init * average complementarity.  Fixed mode: the monotone rule, except
    that once the barrier problem is solved (E_mu <= kappa_eps mu) with progress of
    E_0 against the references, free mode resumes.  Returns (mu, changed, stalled)."""
    mu_old = ph.mu
    if ph.mu_free:
        if sufficient_progress(err0, ph.mu_refs, opt) and not tiny:
            remember_reference(ph.mu_refs, err0, opt)
            mu = max(opt.mu_min_adaptive, min(ph.mu_max, loqo_mu(avg, minimum)))
            return mu, mu != mu_old, False
        ph.mu_free = False
        mu = max(opt.tol / 10.0, opt.mu_monotone_init * avg)
        return mu, mu != mu_old, False
    # fixed mode
    if err_at(ph.mu) <= opt.kappa_eps * ph.mu and sufficient_progress(err0, ph.mu_refs, opt):
        ph.mu_free = True
        ph.mu_refs = [err0]
        mu = max(opt.mu_min_adaptive, min(ph.mu_max, loqo_mu(avg, minimum)))
        return mu, mu != mu_old, False
    mu, decreased, stalled = barrier_update(ph.mu, err_at, tiny, opt)
    return mu, decreased, stalled


# ------------------------------------------------- inertia correction --

def inertia_correction(factor_ok, dw_last, opt):
    """IPOPT's Algorithm IC with delta_w only: the smallest delta_w of its sequence
    for which factor_ok(delta_w) holds.  Returns (delta_w, n_retries) or
    (None, n_retries) when delta_w would exceed delta_w_max."""
    if factor_ok(0.0):
        return 0.0, 0
    dw = opt.dw_init if dw_last == 0.0 else max(opt.dw_min, opt.kappa_w_minus * dw_last)
    n = 0
    while True:
        n += 1
        if factor_ok(dw):
            return dw, n
        dw *= opt.kappa_w_plus_bar if dw_last == 0.0 else opt.kappa_w_plus
        if dw > opt.dw_max:
            return None, n


# ------------------------------------------------ restoration entry --

def resto_elastics(c, mu_r, rho):
    """Closed-form start of the restoration elastics p, n for c(x) - p + n = 0: the
    minimiser of rho (p + n) - mu_R (ln p + ln n) on p - n = c (IPOPT Sec. 3.3)."""
    a = (mu_r - rho * c) / (2.0 * rho)
    nn = a + np.sqrt(a * a + mu_r * c / (2.0 * rho))
    return c + nn, nn


def resto_scaling(x_ref):
    """D_R = diag(min(1, 1/|x_R|)) of the restoration objective's proximity term."""
    return np.minimum(1.0, 1.0 / np.maximum(np.abs(x_ref), 1e-300))


def resto_may_return(ph_orig, theta, phi, theta_ref, opt):
    """Restoration ends when the original constraint violation fell to
    kappa_resto theta(x_R) and the point is acceptable to the original filter."""
    return bool(np.isfinite(phi) and theta <= opt.kappa_resto * theta_ref and not in_filter(ph_orig, theta, phi))


# ------------------------------------------------------------ linear algebra --

class KKTFactor:
    """Bunch-Kaufman LDL^T of the augmented matrix of Eq. 7 with its inertia."""

    def __init__(self, K):
        self.K = K
        lu, d, perm = ldl(K, lower=True)
        self.L = lu[perm]
        self.perm = perm
        self.d = d
        diag = np.diag(d).copy()
        off = np.diag(d, -1).copy()
        ev = eigvalsh_tridiagonal(diag, off) if K.shape[0] > 1 else diag
        self.n_pos = int(np.sum(ev > 0))
        self.n_neg = int(np.sum(ev < 0))
        self.n_zero = int(np.sum(ev == 0))

    def solve(self, rhs):
        b = rhs[self.perm]
        w = solve_triangular(self.L, b, lower=True, unit_diagonal=True)
        n = self.d.shape[0]
        ab = np.zeros((3, n))
        ab[0, 1:] = np.diag(self.d, 1)
        ab[1, :] = np.diag(self.d)
        ab[2, :-1] = np.diag(self.d, -1)
        from scipy.linalg import solve_banded
        v = solve_banded((1, 1), ab, w)
        u = solve_triangular(self.L.T, v, lower=False, unit_diagonal=True)
        out = np.empty_like(u)
        out[self.perm] = u
        return out


def augmented_matrix(Wsig, J, dw):
    n = Wsig.shape[0]
    m = J.shape[0]
    K = np.zeros((n + m, n + m))
    K[:n, :n] = Wsig + dw * np.eye(n)
    K[n:, :n] = J
    K[:n, n:] = J.T
    return K


# ------------------------------------------------------- restoration NLP --

class RestoNLP:
    """The l1 feasibility-restoration problem of IPOPT, built on an NLP.

    min rho * sum(p + n) + zeta/2 * |D_R (x - x_R)|^2
    s.t. c(x) - p + n = 0,  x_L <= x <= x_U,  p, n >= 0,
    with D_R = diag(min(1, 1/|x_R|)) and zeta = sqrt(mu) at the start of the phase.
    Variables are stacked as w = (x, p, n).
    """

    def __init__(self, nlp, x_ref, zeta, rho):
        self.inner = nlp
        self.x_ref = x_ref.copy()
        self.zeta = zeta
        self.rho = rho
        nx, m = nlp.n, nlp.m
        self.nx0 = nx
        self.n = nx + 2 * m
        self.m = m
        self.dr = resto_scaling(x_ref)
        self.xl = np.concatenate([nlp.xl, np.zeros(2 * m)])
        self.xu = np.concatenate([nlp.xu, np.full(2 * m, np.inf)])

    def parts(self, w):
        nx, m = self.nx0, self.m
        return w[:nx], w[nx:nx + m], w[nx + m:]

    def f(self, w):
        x, p, n = self.parts(w)
        return self.rho * float(np.sum(p) + np.sum(n)) + \
            0.5 * self.zeta * float(np.sum((self.dr * (x - self.x_ref)) ** 2))

    def c(self, w):
        x, p, n = self.parts(w)
        return self.inner.c(x) - p + n

    def grad_f(self, w):
        x, _, _ = self.parts(w)
        gx = self.zeta * self.dr ** 2 * (x - self.x_ref)
        return np.concatenate([gx, np.full(2 * self.m, self.rho)])

    def jac_c(self, w):
        x, _, _ = self.parts(w)
        Jx = self.inner.jac_c(x)
        return np.hstack([Jx, -np.eye(self.m), np.eye(self.m)])

    def hess_lag(self, w, y, obj_factor=1.0):
        x, _, _ = self.parts(w)
        H = np.zeros((self.n, self.n))
        H[:self.nx0, :self.nx0] = self.inner.hess_lag(x, y, obj_factor=0.0) + \
            obj_factor * np.diag(self.zeta * self.dr ** 2)
        return H


# ------------------------------------------------------------- the solver --

def initial_state(nlp, x0, opt: Options) -> SolverState:
    """Starting point: x pushed inside its bounds, z = 1 (or centred on mu_init for a
    warm start), y set at the first iteration."""
    x = np.asarray(x0, dtype=np.float64).copy()
    has_l, has_u = bound_sets(nlp)
    k1, k2 = opt.bound_push, opt.bound_frac
    for i in range(nlp.n):
        if has_l[i] and has_u[i]:
            width = nlp.xu[i] - nlp.xl[i]
            pl = min(k1 * max(1.0, abs(nlp.xl[i])), k2 * width)
            pu = min(k1 * max(1.0, abs(nlp.xu[i])), k2 * width)
            x[i] = min(max(x[i], nlp.xl[i] + pl), nlp.xu[i] - pu)
        elif has_l[i]:
            x[i] = max(x[i], nlp.xl[i] + k1 * max(1.0, abs(nlp.xl[i])))
        elif has_u[i]:
            x[i] = min(x[i], nlp.xu[i] - k1 * max(1.0, abs(nlp.xu[i])))
    if opt.z_centred:
        sl, su = slacks(nlp, x)
        zl = np.where(has_l, opt.mu_init / np.where(has_l, sl, 1.0), 0.0)
        zu = np.where(has_u, opt.mu_init / np.where(has_u, su, 1.0), 0.0)
    else:
        zl = np.where(has_l, opt.z_init, 0.0)
        zu = np.where(has_u, opt.z_init, 0.0)
    ph = Phase(x=x, y=np.zeros(nlp.m), zl=zl, zu=zu, mu=opt.mu_init, filt=[])
    return SolverState(normal=ph)


def least_squares_y(nlp, g, J, zl, zu, opt):
    """y minimising |grad f - z_L + z_U + J^T y| via [[I, J^T], [J, 0]]; 0 if too large."""
    n, m = nlp.n, nlp.m
    K = augmented_matrix(np.zeros((n, n)), J, 1.0)
    rhs = np.concatenate([-(g - zl + zu), np.zeros(m)])
    try:
        sol = np.linalg.solve(K, rhs)
    except np.linalg.LinAlgError:
        return np.zeros(m)  # rank-deficient constraint Jacobian: no estimate
    y = sol[n:]
    if m and np.max(np.abs(y)) > opt.y_max:
        y = np.zeros(m)
    return y


def filter_add(ph: Phase, theta, phi, opt):
    """Add (theta, phi) to the filter, dropping entries it dominates; oldest goes when full."""
    ph.filt = [(t, p) for (t, p) in ph.filt if not (t >= theta and p >= phi)]
    ph.filt.append((theta, phi))
    if len(ph.filt) > opt.filter_cap:
        ph.filt.pop(0)


def in_filter(ph: Phase, theta, phi):
    if not (theta < ph.theta_max):
        return True
    return any(theta >= t and phi >= p for (t, p) in ph.filt)


def kappa_sigma_reset(nlp, x, zl, zu, mu, opt):
    """z <- max(min(z, kappa_Sigma mu / s), mu / (kappa_Sigma s)) componentwise."""
    has_l, has_u = bound_sets(nlp)
    sl, su = slacks(nlp, x)
    zl = zl.copy()
    zu = zu.copy()
    ks = opt.kappa_sigma
    zl[has_l] = np.maximum(np.minimum(zl[has_l], ks * mu / sl[has_l]), mu / (ks * sl[has_l]))
    zu[has_u] = np.maximum(np.minimum(zu[has_u], ks * mu / su[has_u]), mu / (ks * su[has_u]))
    return zl, zu


class _Outcome:
    ACCEPTED, CONVERGED, LS_FAILED, EVAL_ERROR, TINY_STALL = range(5)


def phase_iteration(nlp, ph: Phase, opt: Options, trace: dict, init_theta=False,
                    y_ls=False, globalize=False):
    """One iteration of the barrier method on `nlp` from phase state `ph`.

    globalize: the watchdog and soft restoration (when enabled in opt) take part
    in this phase's line search (the original problem; the restoration phase's
    line search is the plain backtracking filter search).
    Returns an _Outcome; on ACCEPTED, `ph` holds the next iterate.
    """
    x, y, zl, zu = ph.x, ph.y, ph.zl, ph.zu
    has_l, has_u = bound_sets(nlp)
    f = nlp.f(x)
    c = nlp.c(x)
    g = nlp.grad_f(x)
    J = nlp.jac_c(x)
    if not (np.isfinite(f) and np.all(np.isfinite(c)) and np.all(np.isfinite(g))
            and np.all(np.isfinite(J))):
        return _Outcome.EVAL_ERROR
    if y_ls:
        y = least_squares_y(nlp, g, J, zl, zu, opt)
        ph.y = y
    theta = theta_of(c)
    if init_theta:
        ph.theta_max = 1e4 * max(1.0, theta)
        ph.theta_min = 1e-4 * max(1.0, theta)

    # overall convergence (Eq. 5 with mu = 0)
    if opt_error(nlp, x, y, zl, zu, g, J, c, 0.0, opt) <= opt.tol:
        return _Outcome.CONVERGED

    # barrier update (Table I row 7): monotone, repeated while the subproblem is
    # solved; or adaptive (free mode with the monotone fallback) on the original problem
    err_at = lambda mu: opt_error(nlp, x, y, zl, zu, g, J, c, mu, opt)  # noqa: E731
    if globalize and opt.mu_strategy == "adaptive":
        avg, minimum = complementarity_stats(nlp, x, zl, zu)
        if ph.mu_max == 0.0:
            ph.mu_max = opt.mu_max_fact * max(avg, opt.tol)
        was_free = ph.mu_free
        mu_new, decreased, stalled = adaptive_barrier_update(ph, err_at(0.0), err_at, avg, minimum, ph.tiny, opt)
        trace["mu_free"] = ph.mu_free
        if was_free != ph.mu_free:
            trace["mu_mode_switch"] = True
    else:
        mu_new, decreased, stalled = barrier_update(ph.mu, err_at, ph.tiny, opt)
    if stalled:
        return _Outcome.TINY_STALL
    if decreased:
        ph.mu = mu_new
        ph.filt = []
        ph.tiny = False
        end_globalization(ph)
    mu = ph.mu
    tau = max(opt.tau_min, 1.0 - mu)

    # augmented system (Eq. 7)
    sl, su = slacks(nlp, x)
    sigma = np.zeros(nlp.n)
    sigma[has_l] += zl[has_l] / sl[has_l]
    sigma[has_u] += zu[has_u] / su[has_u]
    W = nlp.hess_lag(x, y, 1.0)
    Wsig = W + np.diag(sigma)
    gphi = barrier_grad(nlp, x, g, mu, opt)
    rhs = -np.concatenate([gphi + J.T @ y, c])

    # inertia correction (IPOPT Algorithm IC); delta_c is never used
    facs = {}

    def factor_ok(dw_try):
        fac_try = KKTFactor(augmented_matrix(Wsig, J, dw_try))
        facs[dw_try] = fac_try
        return fac_try.n_pos == nlp.n and fac_try.n_neg == nlp.m and fac_try.n_zero == 0

    dw, n_retry = inertia_correction(factor_ok, ph.dw_last, opt)
    if n_retry:
        trace["n_inertia_corr"] = trace.get("n_inertia_corr", 0) + n_retry
    if dw is None:
        trace["ic_failed"] = True
        return _Outcome.LS_FAILED
    if n_retry:
        ph.dw_last = dw
    fac = facs[dw]
    trace["delta_w"] = dw
    if opt.trace_cond:
        trace["cond"] = float(np.linalg.cond(fac.K))

    def solve(rhs_vec):
        sol = fac.solve(rhs_vec)
        return sol[:nlp.n], sol[nlp.n:]

    def z_step(dx):
        dzl = np.zeros(nlp.n)
        dzu = np.zeros(nlp.n)
        dzl[has_l] = mu / sl[has_l] - zl[has_l] - zl[has_l] / sl[has_l] * dx[has_l]
        dzu[has_u] = mu / su[has_u] - zu[has_u] + zu[has_u] / su[has_u] * dx[has_u]
        return dzl, dzu

    def alpha_primal_max(dx):
        return min(frac_to_boundary(sl[has_l], dx[has_l], tau),
                   frac_to_boundary(su[has_u], -dx[has_u], tau))

    def alpha_dual_max(dzl, dzu):
        return min(frac_to_boundary(zl[has_l], dzl[has_l], tau),
                   frac_to_boundary(zu[has_u], dzu[has_u], tau))

    dx, dy = solve(rhs)
    dzl, dzu = z_step(dx)
    a_max = alpha_primal_max(dx)

    def accept(alpha, dx_, dy_, dzl_, dzu_, augment, theta0, phi0, az=None):
        x_new = x + alpha * dx_
        y_new = y + alpha * dy_
        if az is None:
            az = alpha_dual_max(dzl_, dzu_)
        zl_new = zl + az * dzl_
        zu_new = zu + az * dzu_
        zl_new, zu_new = kappa_sigma_reset(nlp, x_new, zl_new, zu_new, mu, opt)
        if augment:
            filter_add(ph, *filter_entry(theta0, phi0, opt), opt)
        ph.x, ph.y, ph.zl, ph.zu = x_new, y_new, zl_new, zu_new
        trace["alpha"] = alpha
        trace["alpha_z"] = az

    # tiny step (Table I row 4)
    if is_tiny_step(x, dx):
        trace["tiny"] = True
        accept(a_max, dx, dy, dzl, dzu, False, 0.0, 0.0)
        ph.tiny = True
        ph.wd_short = 0
        return _Outcome.ACCEPTED
    ph.tiny = False

    # backtracking filter line search (Table I row 1) with SOC (row 2)
    phi0 = barrier_phi(nlp, x, f, mu, opt)
    gdx = float(gphi @ dx)
    a_min = alpha_min(theta, gdx, ph.theta_min, opt)

    def trial_values(xt):
        ft = nlp.f(xt)
        ct = nlp.c(xt)
        if not (np.isfinite(ft) and np.all(np.isfinite(ct))):
            return None
        return theta_of(ct), barrier_phi(nlp, xt, ft, mu, opt), ct

    def acceptable(theta_t, phi_t, alpha):
        return trial_acceptable(ph, theta_t, phi_t, alpha, theta, phi0, gdx, opt)

    def needs_augment(alpha, phi_t):
        return filter_needs_augment(alpha, phi_t, phi0, gdx, theta, opt)

    def soft_resto_step():
        """Soft restoration (Table I row 5): the primal-dual step with one step size
        alpha_s = min(alpha_max, alpha_z_max), accepted if the trial point passes the
        original acceptance tests (which ends the soft phase) or reduces the
        primal-dual error E_pd (which continues it)."""
        a_s = min(a_max, alpha_dual_max(dzl, dzu))
        xt = x + a_s * dx
        tv = trial_values(xt)
        trace["soft_trial"] = True
        if tv is None:
            return False
        theta_t, phi_t, c_t = tv
        if trial_acceptable(ph, theta_t, phi_t, 0.0, theta, phi0, gdx, opt):
            accept(a_s, dx, dy, dzl, dzu, True, theta, phi0, az=a_s)
            ph.soft_active, ph.soft_iters = False, 0
            trace["soft_left"] = True
            return True
        yt, zlt, zut = y + a_s * dy, zl + a_s * dzl, zu + a_s * dzu
        gt, Jt = nlp.grad_f(xt), nlp.jac_c(xt)
        if not (np.all(np.isfinite(gt)) and np.all(np.isfinite(Jt))):
            return False
        e_t = primal_dual_error(nlp, xt, yt, zlt, zut, gt, Jt, c_t, mu)
        e_0 = primal_dual_error(nlp, x, y, zl, zu, g, J, c, mu)
        if opt.trace_soc:
            trace["soft_log"] = {"alpha": a_s, "a_max": a_max, "az_max": alpha_dual_max(dzl, dzu),
                                 "x": x.copy(), "y": y.copy(), "zl": zl.copy(), "zu": zu.copy(),
                                 "dx": dx.copy(), "dy": dy.copy(), "dzl": dzl.copy(), "dzu": dzu.copy(),
                                 "mu": mu, "e_trial": e_t, "e_current": e_0}
        if not soft_resto_accepts(e_t, e_0, opt):
            return False
        accept(a_s, dx, dy, dzl, dzu, True, theta, phi0, az=a_s)
        ph.soft_active = True
        ph.soft_iters += 1
        trace["soft_step"] = True
        return True

    if globalize and ph.soft_active:
        # in the soft restoration phase the soft step replaces the line search
        if ph.soft_iters < opt.soft_max and soft_resto_step():
            return _Outcome.ACCEPTED
        return _Outcome.LS_FAILED

    if globalize and watchdog_should_start(ph, opt):
        ph.wd_active, ph.wd_trials, ph.wd_short = True, 0, 0
        ph.wd_store = {"x": x.copy(), "y": y.copy(), "zl": zl.copy(), "zu": zu.copy(), "dx": dx.copy(),
                       "dy": dy.copy(), "dzl": dzl.copy(), "dzu": dzu.copy(), "theta": theta, "phi": phi0,
                       "gdx": gdx, "a_max": a_max, "a_min": a_min}
        trace["wd_start"] = True
    if globalize and ph.wd_active:
        # watchdog (Table I row 3): the full step, judged against the stored iterate
        W = ph.wd_store
        tv = trial_values(x + a_max * dx)
        if tv is not None and trial_acceptable(ph, tv[0], tv[1], a_max, W["theta"], W["phi"], W["gdx"], opt):
            accept(a_max, dx, dy, dzl, dzu,
                   filter_needs_augment(a_max, tv[1], W["phi"], W["gdx"], W["theta"], opt), W["theta"], W["phi"])
            ph.wd_active, ph.wd_trials, ph.wd_store = False, 0, None
            trace["wd_accepted"] = True
            return _Outcome.ACCEPTED
        ph.wd_trials += 1
        if ph.wd_trials <= opt.wd_trial_max:
            accept(a_max, dx, dy, dzl, dzu, False, 0.0, 0.0)
            trace["wd_step"] = True
            return _Outcome.ACCEPTED
        # give up: back to the stored iterate and a backtracking search along its step
        ph.wd_active, ph.wd_trials, ph.wd_store = False, 0, None
        trace["wd_return"] = True
        return _watchdog_return(nlp, ph, opt, trace, W, mu, tau)

    alpha = a_max
    n_trial = 0
    while True:
        n_trial += 1
        xt = x + alpha * dx
        tv = trial_values(xt)
        if tv is not None:
            theta_t, phi_t, c_t = tv
            if acceptable(theta_t, phi_t, alpha):
                accept(alpha, dx, dy, dzl, dzu, needs_augment(alpha, phi_t), theta, phi0)
                trace["ls_trials"] = n_trial
                ph.wd_short = ph.wd_short + 1 if alpha < a_max else 0
                return _Outcome.ACCEPTED
            # second-order correction on the first trial when theta did not decrease
            if n_trial == 1 and not (theta_t < theta):
                c_soc = soc_constraint_rhs(alpha, c, c_t)
                theta_old = theta
                for p in range(1, opt.p_max + 1):
                    trace["n_soc"] = trace.get("n_soc", 0) + 1
                    dx_s, dy_s = solve(-np.concatenate([gphi + J.T @ y, c_soc]))
                    if opt.trace_soc:
                        trace.setdefault("soc_log", []).append(
                            {"alpha": alpha, "c": c.copy(), "c_trial": c_t.copy(), "c_soc": c_soc.copy(),
                             "dx": dx.copy(), "dx_soc": dx_s.copy(), "J": J.copy()})
                    a_soc = alpha_primal_max(dx_s)
                    xs = x + a_soc * dx_s
                    sv = trial_values(xs)
                    if sv is None:
                        break
                    theta_s, phi_s, c_s = sv
                    if acceptable(theta_s, phi_s, alpha):
                        dzl_s, dzu_s = z_step(dx_s)
                        accept(a_soc, dx_s, dy_s, dzl_s, dzu_s, needs_augment(alpha, phi_s),
                               theta, phi0)
                        trace["soc_accepted"] = True
                        trace["ls_trials"] = n_trial
                        ph.wd_short = 0
                        return _Outcome.ACCEPTED
                    if soc_should_stop(p, theta_s, theta_old, opt):
                        break
                    c_soc = soc_constraint_rhs(a_soc, c_soc, c_s)
                    theta_old = theta_s
        alpha *= 0.5
        if alpha < a_min or n_trial >= opt.ls_max_trials:
            trace["ls_trials"] = n_trial
            if globalize and opt.soft_resto and soft_resto_step():
                return _Outcome.ACCEPTED
            return _Outcome.LS_FAILED


def _watchdog_return(nlp, ph, opt, trace, W, mu, tau):
    """The watchdog gave up: the iterate returns to the one stored when it started,
    and a backtracking filter line search runs along that iterate's step, judged
    against its reference values, from half its full step (the full step was the
    watchdog's first step).  The stored factorisation is gone, so no second-order
    correction is tried.  Returns the outcome of that search."""
    has_l, has_u = bound_sets(nlp)
    x, y, zl, zu = W["x"], W["y"], W["zl"], W["zu"]
    ph.x, ph.y, ph.zl, ph.zu = x, y, zl, zu
    theta, phi0, gdx = W["theta"], W["phi"], W["gdx"]

    def alpha_dual_max(dzl_, dzu_):
        return min(frac_to_boundary(zl[has_l], dzl_[has_l], tau), frac_to_boundary(zu[has_u], dzu_[has_u], tau))

    alpha = 0.5 * W["a_max"]
    n_trial = 0
    while alpha >= W["a_min"] and n_trial < opt.ls_max_trials:
        n_trial += 1
        xt = x + alpha * W["dx"]
        ft, ct = nlp.f(xt), nlp.c(xt)
        if np.isfinite(ft) and np.all(np.isfinite(ct)):
            theta_t, phi_t = theta_of(ct), barrier_phi(nlp, xt, ft, mu, opt)
            if trial_acceptable(ph, theta_t, phi_t, alpha, theta, phi0, gdx, opt):
                az = alpha_dual_max(W["dzl"], W["dzu"])
                x_new = xt
                zl_new, zu_new = kappa_sigma_reset(nlp, x_new, zl + az * W["dzl"], zu + az * W["dzu"], mu, opt)
                if filter_needs_augment(alpha, phi_t, phi0, gdx, theta, opt):
                    filter_add(ph, *filter_entry(theta, phi0, opt), opt)
                ph.x, ph.y, ph.zl, ph.zu = x_new, y + alpha * W["dy"], zl_new, zu_new
                trace["alpha"], trace["alpha_z"], trace["ls_trials"] = alpha, az, n_trial
                return _Outcome.ACCEPTED
        alpha *= 0.5
    trace["ls_trials"] = n_trial
    return _Outcome.LS_FAILED


def resto_start(nlp, st: SolverState, opt: Options):
    """Enter restoration from the current original iterate (IPOPT Sec. 3.3 reading)."""
    ph = st.normal
    x = ph.x
    c = nlp.c(x)
    f = nlp.f(x)
    theta = theta_of(c)
    phi = barrier_phi(nlp, x, f, ph.mu, opt)
    filter_add(ph, *filter_entry(theta, phi, opt), opt)
    zeta = math.sqrt(ph.mu)
    rnlp = RestoNLP(nlp, x, zeta, opt.rho)
    mu_r = max(ph.mu, float(np.max(np.abs(c))) if c.size else 0.0)
    rho = opt.rho
    pp, nn = resto_elastics(c, mu_r, rho)
    w = np.concatenate([x, pp, nn])
    has_l, has_u = bound_sets(nlp)
    zl = np.concatenate([np.where(has_l, np.minimum(rho, ph.zl), 0.0), mu_r / pp, mu_r / nn])
    zu = np.concatenate([np.where(has_u, np.minimum(rho, ph.zu), 0.0), np.zeros(2 * nlp.m)])
    rph = Phase(x=w, y=np.zeros(nlp.m), zl=zl, zu=zu, mu=mu_r, filt=[])
    theta_r = theta_of(rnlp.c(w))
    rph.theta_max = 1e4 * max(1.0, theta_r)
    rph.theta_min = 1e-4 * max(1.0, theta_r)
    st.resto = rph
    st.x_ref = x.copy()
    st.zeta = zeta
    st.mode = RESTO
    return rnlp


def make_resto_nlp(nlp, st: SolverState, opt: Options):
    return RestoNLP(nlp, st.x_ref, st.zeta, opt.rho)


def step(nlp, st: SolverState, opt: Options) -> dict:
    """Advance `st` by one iteration in place; returns a trace of what happened."""
    trace = {"mode": st.mode}
    if st.status != RUNNING:
        return trace
    if st.mode == NORMAL:
        ph = st.normal
        out = phase_iteration(nlp, ph, opt, trace, init_theta=st.need_init,
                              y_ls=st.need_y_ls, globalize=True) if st.iter < opt.max_iter else None
        if out is None:
            # the iteration cap is tested after the convergence test of the same point
            out = _check_only(nlp, ph, opt, st)
            if out == _Outcome.CONVERGED:
                st.status = CONVERGED
            elif out == _Outcome.EVAL_ERROR:
                st.status = EVAL_ERROR
            else:
                st.status = MAX_ITER
            return trace
        st.need_init = False
        st.need_y_ls = False
        if out == _Outcome.CONVERGED:
            st.status = CONVERGED
        elif out == _Outcome.EVAL_ERROR:
            st.status = EVAL_ERROR
        elif out == _Outcome.TINY_STALL:
            st.status = TINY_STEP
        elif out == _Outcome.ACCEPTED:
            st.iter += 1
            if trace.get("tiny"):
                st.n_tiny += 1
        elif out == _Outcome.LS_FAILED:
            c = nlp.c(ph.x)
            if theta_of(c) <= opt.tol:
                st.status = RESTO_FAILED
            else:
                end_globalization(ph)
                resto_start(nlp, st, opt)
                trace["entered_resto"] = True
                st.iter += 1
        st.n_soc += trace.get("n_soc", 0)
        st.n_inertia_corr += trace.get("n_inertia_corr", 0)
        return trace

    # restoration mode
    rnlp = make_resto_nlp(nlp, st, opt)
    rph = st.resto
    if st.iter >= opt.max_iter:
        st.status = MAX_ITER
        return trace
    out = phase_iteration(rnlp, rph, opt, trace)
    st.n_soc += trace.get("n_soc", 0)
    st.n_inertia_corr += trace.get("n_inertia_corr", 0)
    if out in (_Outcome.CONVERGED, _Outcome.LS_FAILED, _Outcome.TINY_STALL):
        st.status = RESTO_FAILED
        return trace
    if out == _Outcome.EVAL_ERROR:
        st.status = EVAL_ERROR
        return trace
    st.iter += 1
    st.n_resto_iter += 1
    # return test: enough reduction of the original infeasibility and acceptable
    # to the original filter at the original barrier parameter
    x = rph.x[:nlp.n]
    c = nlp.c(x)
    f = nlp.f(x)
    th = theta_of(c)
    ph = st.normal
    phi = barrier_phi(nlp, x, f, ph.mu, opt)
    th_ref = theta_of(nlp.c(st.x_ref))
    if resto_may_return(ph, th, phi, th_ref, opt):
        zl, zu = kappa_sigma_reset(nlp, x, rph.zl[:nlp.n], rph.zu[:nlp.n], ph.mu, opt)
        ph.x, ph.zl, ph.zu = x.copy(), zl, zu
        ph.y = rph.y.copy()
        st.need_y_ls = True
        st.mode = NORMAL
        st.resto = None
        trace["left_resto"] = True
    return trace


def _check_only(nlp, ph, opt, st):
    """Convergence test alone (used when the iteration cap is reached)."""
    x = ph.x
    f = nlp.f(x)
    c = nlp.c(x)
    g = nlp.grad_f(x)
    J = nlp.jac_c(x)
    if not (np.isfinite(f) and np.all(np.isfinite(c))):
        return _Outcome.EVAL_ERROR
    y = ph.y
    if st.need_y_ls:
        y = least_squares_y(nlp, g, J, ph.zl, ph.zu, opt)
    if opt_error(nlp, x, y, ph.zl, ph.zu, g, J, c, 0.0, opt) <= opt.tol:
        return _Outcome.CONVERGED
    return None


def solve(nlp, x0=None, opt: Options | None = None, record=False):
    """Run to termination from x0 (default: the NLP's default start)."""
    opt = opt or Options()
    st = initial_state(nlp, nlp.default_start() if x0 is None else x0, opt)
    history = []
    while st.status == RUNNING:
        if record:
            history.append(copy.deepcopy(st))
        tr = step(nlp, st, opt)
        if record:
            history[-1] = (history[-1], tr)
    if record:
        history.append((copy.deepcopy(st), {}))
    return st, history


def final_metrics(nlp, st: SolverState, opt: Options | None = None):
    """Objective, scaled KKT error E_0 and infeasibility at the final original iterate."""
    opt = opt or Options()
    ph = st.normal
    x = ph.x
    g = nlp.grad_f(x)
    J = nlp.jac_c(x)
    c = nlp.c(x)
    return {
        "obj": nlp.f(x),
        "kkt": opt_error(nlp, x, ph.y, ph.zl, ph.zu, g, J, c, 0.0, opt),
        "inf": float(np.max(np.abs(c))) if c.size else 0.0,
    }
