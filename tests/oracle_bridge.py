"""Test helpers that move solver states between the oracle and the library.

Test infrastructure only: it reads oracle states and writes the equivalent
bipm_iterate record, and builds the comparison vectors of the state-injection
test (Sec. VI, Eq. 8).
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import ipm
from oracle.quadrotor import QuadNLP
from oracle.quat13 import QuatNLP


def oracle_to_iterate(nlp, st: ipm.SolverState) -> dict:
    n, m = nlp.n, nlp.m
    ph = st.normal
    out = {
        "mode": st.mode, "status": st.status, "iter": st.iter,
        "need_init": int(st.need_init), "need_y_ls": int(st.need_y_ls),
        "tiny": int(ph.tiny), "mu": ph.mu, "dw_last": ph.dw_last,
        "theta_max": ph.theta_max, "theta_min": ph.theta_min,
        "filter": np.array(ph.filt, dtype=np.float64).reshape(-1, 2),
        "wd_short": int(ph.wd_short), "wd_active": int(ph.wd_active), "wd_trials": int(ph.wd_trials),
        "soft_active": int(ph.soft_active), "soft_iters": int(ph.soft_iters),
        "mu_free": int(ph.mu_free), "mu_refs": list(ph.mu_refs), "mu_max": ph.mu_max,
    }
    if ph.wd_store is not None:
        W = ph.wd_store
        out.update(wd_x=W["x"], wd_y=W["y"], wd_zl=W["zl"], wd_zu=W["zu"], wd_dx=W["dx"], wd_dy=W["dy"],
                   wd_theta=W["theta"], wd_phi=W["phi"], wd_gdx=W["gdx"], wd_amax=W["a_max"],
                   wd_amin=W["a_min"])
    if st.mode == ipm.NORMAL:
        out.update(x=ph.x, y=ph.y, zl=ph.zl, zu=ph.zu)
    else:
        r = st.resto
        out.update(x=r.x[:n], p=r.x[n:n + m], nn=r.x[n + m:], y=r.y,
                   zl=r.zl[:n], zp=r.zl[n:n + m], zn=r.zl[n + m:], zu=r.zu[:n],
                   x_ref=st.x_ref, zeta=st.zeta, mu_r=r.mu, dw_last_r=r.dw_last,
                   theta_max_r=r.theta_max, theta_min_r=r.theta_min, tiny_r=int(r.tiny),
                   filter_r=np.array(r.filt, dtype=np.float64).reshape(-1, 2),
                   theta_ref=float(np.sum(np.abs(nlp.c(st.x_ref)))))
    return out


def compare_vector(state: dict) -> np.ndarray:
    """Quantities compared by e_v: the active iterate and the barrier parameter(s),
    and the watchdog's stored iterate and step while it is active."""
    parts = [state["x"], state["y"], state["zl"], state["zu"], [state["mu"]]]
    if state["mode"] == ipm.RESTO:
        parts += [state["p"], state["nn"], state["zp"], state["zn"], [state["mu_r"]]]
    refs = list(state.get("mu_refs", []))
    parts += [refs, [state.get("mu_max", 0.0)]]
    if state.get("wd_active"):
        parts += [state["wd_x"], state["wd_y"], state["wd_zl"], state["wd_zu"], state["wd_dx"], state["wd_dy"],
                  [state["wd_theta"], state["wd_phi"], state["wd_gdx"], state["wd_amax"], state["wd_amin"]]]
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def globalization_state(state: dict) -> tuple:
    """The discrete watchdog / soft-restoration state of an iterate record."""
    return tuple(int(state.get(k, 0)) for k in ("wd_short", "wd_active", "wd_trials", "soft_active", "soft_iters",
                                                 "mu_free")) + (len(state.get("mu_refs", [])),)


def e_v(v, v_ref) -> float:
    """Largest scaled elementwise deviation, Eq. 8."""
    v = np.asarray(v)
    v_ref = np.asarray(v_ref)
    if v.size == 0:
        return 0.0
    return float(np.max(np.abs(v - v_ref) / (1.0 + np.abs(v_ref))))


def _single_thread():
    import torch

    torch.set_num_threads(1)


def nlp_of(desc, theta):
    """The oracle NLP of a problem: the 12-state model, or the 13-state one for a
    QuatProblemDesc."""
    return QuatNLP(desc, theta) if getattr(desc, "model", "euler12") == "quat13" else QuadNLP(desc, theta)


def _solve_one(args):
    desc, theta, record, opt_kw = args
    _single_thread()
    nlp = nlp_of(desc, theta)
    opt = ipm.Options(**opt_kw)
    st, hist = ipm.solve(nlp, opt=opt, record=record)
    res = {
        "status": st.status, "iter": st.iter, "resto": st.n_resto_iter, "soc": st.n_soc,
        "ic": st.n_inertia_corr, "x": st.normal.x.copy(), "y": st.normal.y.copy(),
        "metrics": ipm.final_metrics(nlp, st, opt) if st.status == ipm.CONVERGED else None,
    }
    if record:
        res["history"] = [(oracle_to_iterate(nlp, s), tr) for (s, tr) in hist]
    return res


def oracle_solve_batch(desc, theta, record=False, processes=None, **opt_kw):
    """Oracle solves of every row of theta, in a spawn process pool."""
    jobs = [(desc, theta[j], record, opt_kw) for j in range(theta.shape[0])]
    if processes == 1 or len(jobs) <= 1:
        return [_solve_one(j) for j in jobs]
    ctx = mp.get_context("spawn")
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # one thread per worker process
    with ctx.Pool(processes=processes or min(len(jobs), mp.cpu_count())) as pool:
        return pool.map(_solve_one, jobs)


def straight_line_guess(desc, theta):
    """A deliberately poor primal starting point: positions on the straight line
    from the start to the goal (through any obstacle on the way), zero velocity
    and attitude, hover thrust, zero slacks.  Input construction only."""
    from workloads import theta_layout

    lay = theta_layout(desc)
    nq, N, nx, nu, ni = desc.nq, desc.horizon, desc.nx, desc.nu, desc.ni
    x0 = np.zeros(desc.n)
    pos = 0
    for k in range(N + 1):
        t = k / N
        for q in range(nq):
            p0 = theta[lay["xbar"] + 12 * q:lay["xbar"] + 12 * q + 3]
            goal = theta[lay["ref"] + 6 * q:lay["ref"] + 6 * q + 3]
            x0[pos + 12 * q:pos + 12 * q + 3] = (1 - t) * p0 + t * goal
        pos += nx
        if k < N:
            x0[pos:pos + nu] = 0.5 * 9.81 / 4.0
            pos += nu
        if k >= 1:
            pos += ni
    return x0


def oracle_kkt_error(desc, theta, x, y, zl, zu, tol=1e-6):
    """IPOPT's scaled optimality error E_0 of a returned iterate, evaluated with
    the oracle's own model and autograd derivatives (an independent KKT check)."""
    nlp = QuadNLP(desc, theta)
    opt = ipm.Options(tol=tol)
    g = nlp.grad_f(x)
    J = nlp.jac_c(x)
    c = nlp.c(x)
    return ipm.opt_error(nlp, np.asarray(x), np.asarray(y), np.asarray(zl), np.asarray(zu), g, J, c,
                         0.0, opt)


def oracle_warm_case(job):
    """Oracle cold solve of one problem, a perturbed encoding of its solution
    decoded to a warm starting point, and the oracle's warm-started solve from
    it.  Returns (guess, status, iterations, x, cold iterations)."""
    import torch

    from oracle import warm

    desc, theta, j = job
    nlp = QuadNLP(desc, theta)
    cold, _ = ipm.solve(nlp)
    o = warm.encode(desc, theta, cold.normal.x)
    rng = np.random.default_rng(100 + j)
    o = (o + 0.05 * rng.standard_normal(o.size)).astype(np.float32).astype(np.float64)
    guess = warm.decode(desc, theta, o, lambda s: nlp.ineq(torch.as_tensor(s)).numpy())
    st, _ = ipm.solve(nlp, x0=guess, opt=warm.warm_options())
    return guess, st.status, st.iter, st.normal.x, cold.iter


def check_outcome(desc, theta, status, x, y, zl, zu, oracle_status, tol=1e-6):
    """Outcome rule of a GPU solve against the oracle's solve of the same problem.

    * The oracle converged: the GPU must converge too, to a point that the
      oracle's own KKT evaluation accepts (E_0 <= tol).
    * The oracle ended in a failure status: the GPU must end in the same one, or
      converge to a point the oracle's KKT test accepts.  The second case is a
      path split: a failing run passes through numerically singular steps,
      where two backward-stable solvers may round onto different paths.
    Returns True for a path split (the caller bounds how many it accepts)."""
    if status == ipm.CONVERGED:
        err = oracle_kkt_error(desc, theta, x, y, zl, zu, tol)
        assert err <= tol, ("GPU point fails the oracle's KKT test", err)
        return oracle_status != ipm.CONVERGED
    assert oracle_status != ipm.CONVERGED, ("oracle converged, GPU ended with status", status)
    assert status == oracle_status, ("failure statuses differ", status, oracle_status)
    return False
