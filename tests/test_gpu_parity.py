"""Parity of the CUDA solver with the CPU oracle (GPU tests, through the C ABI).

* State injection (Sec. VI "Correctness", Eq. 8): every recorded oracle state
  is loaded into a slot, the library advances it by exactly one iteration,
  and the result must equal the oracle's next state: same mode, status and
  iteration counter, the same filter, and e_v <= 1e-6 on the iterate and
  barrier parameter.  It runs on the navigation workload with both team
  schedules, and on the benchmark's tracking workload (N = 30, three
  spheres), four quadrotors with pairwise separation, the cluttered
  environment (cylinders) and a hover problem whose steps are tiny steps
  (Table I row 4); each case asserts the branches of Table I it reaches.
* Full solves against the oracle's solves of the same problems.  The outcome
  rule (oracle_bridge.check_outcome): where the oracle converges the GPU must
  converge to a point that the oracle's own KKT evaluation accepts
  (E_0 <= 1e-6); where the oracle fails the GPU must fail with the same
  status, or converge to a point the oracle's KKT test accepts (a path split
  in the numerically singular steps of a failing run; each test bounds how
  many it accepts).  Where the iteration counts agree, FP64 solutions agree
  to e_v <= 1e-6.
* Mixed-precision forms: every converged point passes the oracle's KKT test,
  and the distance from the oracle's solution is reported per problem.
* Full-size workloads in the benchmark's launch configuration: every problem
  checked by properties that hold at any size (status, E_0), a spread sample
  against the oracle one by one.
"""

import dataclasses
import json
import os

import numpy as np
import pytest

from oracle import ipm
from workloads import ProblemDesc, make_batch

from oracle_bridge import (check_outcome, compare_vector, e_v, globalization_state, oracle_kkt_error,
                           oracle_solve_batch, oracle_to_iterate)

pytestmark = pytest.mark.gpu

TOL_EV = 1e-6  # Eq. 8 deviation per state-injection step
EPS = 2.220446049250313e-16
# Two backward-stable solvers of the same augmented system (the oracle's dense
# Bunch-Kaufman and the library's Riccati recursion) agree to about
# cond * eps relative, cond the 2-norm condition number of the step's matrix
# (recorded by the oracle).  A step is therefore compared within
# max(TOL_EV, 10 eps cond); at cond > COND_SINGULAR = 1 / (10 eps) that bound
# passes 1: the matrix is numerically singular and the step is not determined
# by the data, so only the discrete outcome (mode, status, iteration, filter
# length) is compared.  Such steps occur only in runs that end in
# restoration failure.
COND_SINGULAR = 1.0 / (10.0 * EPS)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def bipm():
    import torch

    assert torch.cuda.is_available()
    from paper_2606_26341_gb300 import bipm as b

    b.load_library()
    return b


def _inject(bipm, desc, theta, histories, precision=0, schedule=1, **opt_kw):
    """One library step from every recorded oracle state; returns (pairs, gpu states)."""
    pairs = [(j, k) for j, h in enumerate(histories) for k in range(len(h) - 1)]
    with bipm.Batch(desc, len(pairs), bipm.Options(precision=precision, schedule=schedule, **opt_kw)) as b:
        b.set_problems(np.ascontiguousarray(np.stack([theta[j] for j, _ in pairs])))
        for s, (j, k) in enumerate(pairs):
            b.set_iterate(s, histories[j][k][0])
        b.step(1)
        got = [b.get_iterate(s) for s in range(len(pairs))]
    return pairs, got


def _check_injection(pairs, got, histories):
    """Returns (worst e_v of the steps compared at 1e-6, steps compared within the
    conditioning bound, worst ratio e_v / bound there, numerically singular steps).
    A numerically singular step's direction is not determined by the data, so even
    its discrete outcome (accept vs. restoration) may differ; such steps are
    counted, and a differing outcome is reported, not failed."""
    worst, n_cond, worst_ratio, n_sing = 0.0, 0, 0.0, 0
    for (j, k), g in zip(pairs, got):
        ref = histories[j][k + 1][0]
        tr = histories[j][k][1]
        cond = tr.get("cond", 0.0)
        if cond > COND_SINGULAR:
            n_sing += 1
            if (g["mode"], g["status"], g["iter"]) != (ref["mode"], ref["status"], ref["iter"]):
                print(f"numerically singular step ({j}, {k}), cond {cond:.1e}: outcome differs "
                      f"(mode {g['mode']} / {ref['mode']}, status {g['status']} / {ref['status']})")
            continue
        assert g["mode"] == ref["mode"], (j, k, "mode", g["mode"], ref["mode"])
        assert g["status"] == ref["status"], (j, k, "status", g["status"], ref["status"])
        assert g["iter"] == ref["iter"], (j, k)
        assert globalization_state(g) == globalization_state(ref), (j, k, globalization_state(g),
                                                                    globalization_state(ref))
        assert len(g["filter"]) == len(ref["filter"]), (j, k)
        if ref["mode"] == ipm.RESTO:
            assert len(g["filter_r"]) == len(ref["filter_r"]), (j, k)
        ev = e_v(compare_vector(g), compare_vector(ref))
        tol = max(TOL_EV, 10.0 * EPS * cond)
        assert ev <= tol, (j, k, ev, tol, tr)
        if len(ref["filter"]):
            assert _filter_ev(g["filter"], ref["filter"]) <= tol
        if tol > TOL_EV:
            n_cond += 1
            worst_ratio = max(worst_ratio, ev / tol)
        else:
            worst = max(worst, ev)
    return worst, n_cond, worst_ratio, n_sing


def _filter_ev(a, b):
    """e_v of two filters; entries that are equal (infinite ones included) count as 0."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    same = a == b
    if same.all():
        return 0.0
    return e_v(np.where(same, 0.0, a), np.where(same, 0.0, b))


def _report(label, pairs, checked):
    worst, n_cond, ratio, n_sing = checked
    print(f"{label}: {len(pairs)} steps; {len(pairs) - n_cond - n_sing} at 1e-6 (worst e_v {worst:.2e}), "
          f"{n_cond} within 10 eps cond (worst fraction of the bound {ratio:.2f}), {n_sing} numerically singular")


def _branches(histories):
    return {k for h in histories for (_, tr) in h for k in tr if k in
            ("n_soc", "soc_accepted", "entered_resto", "left_resto", "n_inertia_corr", "tiny")}


@pytest.fixture(scope="module")
def nav_oracle():
    desc, theta = make_batch("nav1", 64)
    res = oracle_solve_batch(desc, theta, record=True, trace_cond=True)
    return desc, theta, res


@pytest.mark.parametrize("schedule", [1, 2], ids=["warp_team", "block_team"])
def test_state_injection_nav1(bipm, nav_oracle, schedule):
    """Every problem whose oracle run took an SOC, restoration or failure
    branch, plus every fourth problem; one step by a warp per problem and by a
    256-thread block per problem."""
    desc, theta, res = nav_oracle
    sel = sorted(set(range(0, 64, 4)) | {j for j, r in enumerate(res)
                                          if r["soc"] or r["resto"] or r["status"] != ipm.CONVERGED})
    hist = [res[j]["history"] for j in sel]
    pairs, got = _inject(bipm, desc, theta[sel], hist, schedule=schedule)
    _report("nav1", pairs, _check_injection(pairs, got, hist))
    branches = _branches(hist)
    print(f"branches {sorted(branches)}")
    # the selection must exercise the branches of Table I this workload reaches
    assert {"n_soc", "entered_resto", "left_resto", "n_inertia_corr"} <= branches


def _injection_case(name):
    """(desc, theta, branches the case must reach) of the state-injection workloads.
    The problem ids were picked from oracle runs of the first problems of each
    workload: the ones whose runs take the branches listed, plus plain ones."""
    if name == "track":
        desc, theta = make_batch("track", 48)
        ids = TRACK_IDS
        need = {"n_soc", "n_inertia_corr", "entered_resto"}
    elif name == "multi4":
        desc = ProblemDesc(nq=4, horizon=8, dt=0.05, pair_dist=0.4)
        _, theta = make_batch("multi4", 8, desc=desc)
        # 4 ends in restoration failure after 78 corrections, 5 takes two corrections
        ids = [0, 1, 5, 4]
        need = {"n_soc", "n_inertia_corr", "entered_resto"}
    elif name == "cyl":
        d0, _ = make_batch("cyl", 1)
        desc = dataclasses.replace(d0, horizon=12)
        _, theta = make_batch("cyl", 32, desc=desc)
        ids = CYL_IDS
        need = {"n_soc", "n_inertia_corr", "entered_resto"}
    elif name == "track_moving":
        desc, theta = make_batch("track_moving", 24)
        ids = TRACK_MOVING_IDS
        need = {"n_soc", "n_inertia_corr"}
    elif name == "swap2":
        desc, theta = make_batch("swap2", 3)
        ids = [0, 1, 2]
        need = {"n_inertia_corr"}
    else:  # hover: a quadrotor at rest at its goal takes tiny steps only
        desc = ProblemDesc(nq=1, horizon=10, dt=0.05)
        theta = np.zeros((3, 18))
        theta[1, 0:3] = [1.0, -1.0, 0.5]
        theta[2, 0:3] = [-0.5, 0.25, -1.0]
        ids = [0, 1, 2]
        need = {"tiny"}
    return desc, np.ascontiguousarray(theta[ids]), need


# problem 27 ends in restoration failure (33 restoration iterations), 37 takes eight
# corrections and 32 inertia corrections, 9 and 25 three corrections each
TRACK_IDS = [27, 37, 9, 25, 0, 1]
# cluttered environment at N = 12: problem 13 ends in restoration failure after
# corrections and inertia corrections; 0-2 converge plainly
CYL_IDS = [13, 0, 1, 2]


# tracking with three moving spheres (the time-varying obstacles of Sec. VI): 9 and 20
# take five and four corrections, 3 and 10 over thirty inertia corrections
TRACK_MOVING_IDS = [9, 20, 3, 10, 0, 1]


@pytest.mark.parametrize("case", ["track", "multi4", "cyl", "hover", "track_moving", "swap2"])
def test_state_injection_workloads(bipm, case):
    """State injection on the benchmark's own workload and the other families."""
    desc, theta, need = _injection_case(case)
    res = oracle_solve_batch(desc, theta, record=True, trace_cond=True)
    hist = [r["history"] for r in res]
    pairs, got = _inject(bipm, desc, theta, hist)
    _report(case, pairs, _check_injection(pairs, got, hist))
    branches = _branches(hist)
    print(f"branches {sorted(branches)}")
    assert need <= branches, (need, branches)


def _watchdog_history(desc, theta, start_iter, block_all, steps=6):
    """Oracle states of a watchdog scenario on one problem: the oracle runs with
    the watchdog on to iteration start_iter, the shortened-step count is set to its
    trigger there (and, with block_all, the filter gets an entry that rejects every
    trial point), and the oracle's next `steps` iterations are recorded.  The
    scenario is the oracle's: the library must reproduce each step from each state."""
    import copy

    from oracle.quadrotor import QuadNLP

    nlp = QuadNLP(desc, theta)
    opt = ipm.Options(watchdog=True, soft_resto=False, trace_cond=True)
    st = ipm.initial_state(nlp, nlp.default_start(), opt)
    for _ in range(start_iter):
        ipm.step(nlp, st, opt)
    st.normal.wd_short = opt.wd_trigger
    if block_all:
        st.normal.filt = [(-1.0, -np.inf)]
    hist = []
    for _ in range(steps):
        if st.status != ipm.RUNNING:
            break
        s0 = copy.deepcopy(st)
        tr = ipm.step(nlp, st, opt)
        hist.append((oracle_to_iterate(nlp, s0), tr))
    hist.append((oracle_to_iterate(nlp, st), {}))
    return hist


@pytest.mark.parametrize("scenario", ["soft_restoration", "watchdog", "watchdog_gives_up"])
def test_state_injection_globalization(bipm, scenario):
    """Watchdog (Table I row 3) and soft restoration (row 5) by state injection.
    * soft_restoration: the tracking problem whose line search fails repeatedly
      (problem 27), solved by the oracle with soft restoration on: soft steps,
      their acceptance by the primal-dual error, and hard restoration after.
    * watchdog: nav1 problems with the watchdog triggered at their third
      iteration: the stored iterate, the full steps and their acceptance.
    * watchdog_gives_up: the same with every trial rejected by the filter: three
      unconditional steps, the return to the stored iterate, its failed
      backtracking search and restoration from the stored point."""
    if scenario == "soft_restoration":
        desc, theta = make_batch("track", 28)
        theta = np.ascontiguousarray(theta[[27]])
        res = oracle_solve_batch(desc, theta, record=True, trace_cond=True, soft_resto=True)
        hist = [res[0]["history"]]
        kw = {"soft_resto": 1}
        need = {"soft_trial", "soft_step", "entered_resto"}
    else:
        desc, theta = make_batch("nav1", 4)
        block = scenario == "watchdog_gives_up"
        hist = [_watchdog_history(desc, theta[j], 3, block) for j in range(4)]
        kw = {"watchdog": 1}
        need = {"wd_start", "wd_step", "wd_return", "entered_resto"} if block else {"wd_start"}
    pairs, got = _inject(bipm, desc, theta, hist, **kw)
    _report(scenario, pairs, _check_injection(pairs, got, hist))
    seen = {k for h in hist for (_, tr) in h for k in tr}
    print(f"branches {sorted(k for k in seen if k.startswith(('wd_', 'soft_', 'entered')))}")
    assert need <= seen, (need, seen)


def test_state_injection_adaptive_barrier(bipm, nav_oracle):
    """The adaptive barrier update (Table I row 7, free mode with the monotone
    fallback) by state injection: nav1 problems solved by the oracle with
    mu_strategy adaptive, every step of every run loaded and advanced once;
    the runs must switch between free and fixed mode.  Then full solves of the
    64 problems under the outcome rule."""
    desc, theta, _ = nav_oracle
    sel = list(range(0, 64, 4)) + [8]
    res = oracle_solve_batch(desc, theta[sel], record=True, trace_cond=True, mu_strategy="adaptive")
    hist = [r["history"] for r in res]
    pairs, got = _inject(bipm, desc, theta[sel], hist, mu_strategy=1)
    _report("adaptive mu", pairs, _check_injection(pairs, got, hist))
    switches = sum(bool(tr.get("mu_mode_switch")) for h in hist for (_, tr) in h)
    print(f"free/fixed switches {switches}")
    assert switches >= 5
    with bipm.Batch(desc, len(sel), bipm.Options(precision=0, mu_strategy=1)) as b:
        b.set_problems(np.ascontiguousarray(theta[sel]))
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    for t, j in enumerate(sel):
        if _singular_run(res[t]) and st["status"][t] != bipm.CONVERGED:
            continue
        assert not check_outcome(desc, theta[j], st["status"][t], x[t], y[t], zl[t], zu[t], res[t]["status"])
        if st["iters"][t] == res[t]["iter"]:
            assert e_v(x[t], res[t]["x"]) <= 1e-6


def _singular_run(r):
    """True if the oracle's run passed through a numerically singular step."""
    return any(tr.get("cond", 0.0) > COND_SINGULAR for (_, tr) in r["history"])


def test_full_solve_nav1_matches_oracle(bipm, nav_oracle):
    desc, theta, res = nav_oracle
    with bipm.Batch(desc, 64, bipm.Options(precision=0)) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    same_path, splits = 0, 0
    for j in range(64):
        r = res[j]
        if _singular_run(r) and st["status"][j] != bipm.CONVERGED:
            continue  # outcome of a numerically singular path: either side may fail
        splits += check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], r["status"])
        if st["iters"][j] == r["iter"] and st["status"][j] == r["status"]:
            same_path += 1
            assert e_v(x[j], r["x"]) <= 1e-6, (j, e_v(x[j], r["x"]))
    # paths may split where a decision sits at a floating-point tie; require
    # the overwhelming majority to follow the oracle's path exactly
    assert same_path >= 60, same_path
    assert splits <= 2, splits


@pytest.mark.parametrize("form", ["fp32_refined", "fp32_blocks_fp64_factor", "double_float"])
def test_mixed_precision_nav1_against_oracle(bipm, nav_oracle, form):
    """Mixed-precision forms take inexact Newton steps (FP32-rounded derivative
    blocks; FP32 or double-float factors), so their iterates leave the oracle's
    path at the level of that rounding.  What they must deliver is the same
    accuracy: every converged point passes the oracle's own KKT test, outcomes
    follow the rule above, and the distance of each solution from the oracle's
    is reported (it is bounded by the KKT tolerance's sensitivity, not 1e-6)."""
    desc, theta, res = nav_oracle
    opt = {"fp32_refined": bipm.Options(precision=1),
           "fp32_blocks_fp64_factor": bipm.Options(precision=1, fp32_switch=-1.0),
           "double_float": bipm.Options(precision=2)}[form]
    with bipm.Batch(desc, 64, opt) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    errs, same_it, splits, singular = [], 0, 0, []
    for j in range(64):
        if _singular_run(res[j]):
            # the oracle's own path runs through numerically singular steps: an
            # inexact Newton step may end elsewhere, in either direction; a
            # converged GPU point must still pass the oracle's KKT test
            singular.append((j, int(st["status"][j]), res[j]["status"]))
            if st["status"][j] == bipm.CONVERGED:
                assert oracle_kkt_error(desc, theta[j], x[j], y[j], zl[j], zu[j]) <= 1e-6, j
            continue
        splits += check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], res[j]["status"])
        if res[j]["status"] == ipm.CONVERGED:
            ev = e_v(x[j], res[j]["x"])
            errs.append(ev)
            if st["iters"][j] == res[j]["iter"]:
                same_it += 1
                # same iteration count: the inexact steps stayed on the oracle's path
                assert ev <= 1e-6, (j, ev)
    errs = np.array(errs)
    print(f"{form}: e_v vs oracle max {errs.max():.2e} median {np.median(errs):.2e} "
          f"p90 {np.percentile(errs, 90):.2e}; same iteration count {same_it}/{len(errs)}; splits {splits}; "
          f"singular oracle runs (j, gpu, oracle) {singular}")
    assert splits <= 1
    assert same_it >= len(errs) - 3


def test_degenerate_and_error_cases(bipm):
    desc, theta = make_batch("nav1", 4)
    th = theta.copy()
    th[1, 0] = np.nan  # non-finite parameter -> EVAL_ERROR for that problem only
    # problem 2 already sits at its goal: hover at the origin, obstacle far away
    th[2, :] = 0.0
    th[2, 18:22] = [5.0, 5.0, 5.0, 0.5]
    with bipm.Batch(desc, 4, bipm.Options(precision=0)) as b:
        b.set_problems(th)
        b.solve()
        st = b.get_stats()
    assert st["status"][1] == bipm.EVAL_ERROR
    assert st["status"][0] == bipm.CONVERGED and st["status"][3] == bipm.CONVERGED
    assert st["status"][2] == bipm.CONVERGED and st["iters"][2] <= 10
    # iteration cap 0: only the convergence test runs
    with bipm.Batch(desc, 2, bipm.Options(max_iter=0)) as b:
        b.set_problems(theta[:2])
        b.solve()
        st = b.get_stats()
    assert list(st["status"]) == [bipm.MAX_ITER, bipm.MAX_ITER]
    # empty batch and empty loads are no-ops
    with bipm.Batch(desc, 0) as b:
        b.solve()
    with bipm.Batch(desc, 3) as b:
        b.set_problems(theta[:0])
        with pytest.raises(bipm.BipmError):
            b.set_problems(theta[:3], first_slot=1)  # past capacity


def test_short_horizon_and_ragged_batch(bipm):
    """N = 1 (a single interval) and a batch that is not a multiple of the warps per block."""
    desc = ProblemDesc(nq=1, horizon=1, dt=0.05, n_sph=1)
    _, theta = make_batch("nav1", 5, desc=desc)
    res = oracle_solve_batch(desc, theta, processes=1)
    with bipm.Batch(desc, 5) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    for j in range(5):
        assert not check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], res[j]["status"])
        if st["iters"][j] == res[j]["iter"]:
            assert e_v(x[j], res[j]["x"]) <= 1e-6


def _sample_ids(batch, k):
    return sorted(set(np.linspace(0, batch - 1, k).astype(int).tolist()))


@pytest.mark.parametrize("precision", [2, 1, 0])
def test_track_full_size_bench_configuration(bipm, precision):
    """4096 tracking problems (N = 30, three spheres) in the benchmark's launch
    configuration: every problem must end CONVERGED with E_0 <= 1e-6 or in a
    failure status; 12 spread problems are solved by the oracle one by one and
    compared under the outcome rule."""
    desc, theta = make_batch("track", 4096)
    with bipm.Batch(desc, 4096, bipm.Options(precision=precision)) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    conv = st["status"] == bipm.CONVERGED
    assert np.all(st["kkt_err"][conv] <= 1e-6)
    assert conv.mean() >= 0.95, conv.mean()
    ids = _sample_ids(4096, 12)
    res = oracle_solve_batch(desc, theta[ids])
    splits = 0
    for r, j in zip(res, ids):
        splits += check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], r["status"])
        if precision == 0 and r["status"] == ipm.CONVERGED and st["iters"][j] == r["iter"]:
            assert e_v(x[j], r["x"]) <= 1e-6, (j, e_v(x[j], r["x"]))
    assert splits <= 1


def test_multi_quad_sample(bipm):
    """Four quadrotors with pairwise separation (block-diagonal dynamics, coupled
    inequality rows), horizon shortened to N = 8 so the oracle stays quick,
    against the oracle on a small batch."""
    desc = ProblemDesc(nq=4, horizon=8, dt=0.05, pair_dist=0.4)
    _, theta = make_batch("multi4", 4, desc=desc)
    res = oracle_solve_batch(desc, theta)
    with bipm.Batch(desc, 4, bipm.Options(precision=0)) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    for j, r in enumerate(res):
        assert not check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], r["status"])
        if r["status"] == ipm.CONVERGED and st["iters"][j] == r["iter"]:
            assert e_v(x[j], r["x"]) <= 1e-6


def _golden_outcomes(bipm, fname, desc, count, precision=0):
    with open(os.path.join(GOLDEN, fname)) as fh:
        golden = json.load(fh)
    _, theta = make_batch("multi4", count, desc=desc)
    with bipm.Batch(desc, count, bipm.Options(precision=precision)) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    splits, same = 0, 0
    for j in range(count):
        splits += check_outcome(desc, theta[j], st["status"][j], x[j], y[j], zl[j], zu[j], golden["status"][j])
        if golden["status"][j] == ipm.CONVERGED and st["iters"][j] == golden["iters"][j]:
            same += 1
            if precision == 0:
                assert e_v(x[j], np.asarray(golden["x"][j])) <= 1e-6, j
    return st, golden, splits, same


def test_multi_quad_n12_outcomes_match_stored_oracle(bipm):
    """Four quadrotors at horizon 12: the oracle's outcomes (two of eight
    problems end in restoration failure), stored by
    tests/golden/make_multi4.py, are reproduced problem by problem."""
    desc = ProblemDesc(nq=4, horizon=12, dt=0.05, pair_dist=0.4)
    _, _, splits, _ = _golden_outcomes(bipm, "multi4_n12_oracle.json", desc, 8)
    assert splits == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_quad_n25_outcomes_match_stored_oracle(bipm, precision):
    """Configuration 3 at its own horizon: four quadrotors, pairwise separation
    0.4, N = 25 (1798 variables, 1398 equalities).  The oracle's outcomes of
    the first problems, stored by tests/golden/make_multi4.py, are reproduced
    under the outcome rule, in FP64 and in the FP32-refinement form."""
    desc = ProblemDesc(nq=4, horizon=25, dt=0.05, pair_dist=0.4)
    with open(os.path.join(GOLDEN, "multi4_n25_oracle.json")) as fh:
        count = len(json.load(fh)["status"])
    st, golden, splits, same = _golden_outcomes(bipm, "multi4_n25_oracle.json", desc, count, precision)
    print(f"multi4 N=25 precision {precision}: statuses {list(st['status'])} vs {golden['status']}; "
          f"same iteration count {same}; splits {splits}")
    assert splits <= 1


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_queue_matches_batch_solve(bipm, nav_oracle, precision):
    """Iteration-level batching (a queue through fewer slots than problems)
    gives every problem the result a plain batch solve gives it."""
    import torch

    desc, theta, res = nav_oracle
    theta_dev = torch.as_tensor(theta, device="cuda")
    # warp teams only, like the queue, so both run the same code per problem
    with bipm.Batch(desc, 64, bipm.Options(precision=precision, schedule=1)) as b:
        b.set_problems(theta)
        b.solve()
        st = b.get_stats()
        x_b, _, _, _ = b.get_solution()
    with bipm.Batch(desc, 8, bipm.Options(precision=precision)) as b:  # 8 slots, 64 problems
        x_q = torch.empty((64, desc.n), dtype=torch.float64, device="cuda")
        raw = torch.empty(64 * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        b.solve_queue(theta_dev, x_q, raw)
        rq = bipm.results_from_bytes(raw.cpu().numpy())
        # host-pointer variant of the same call
        x_h = np.empty((64, desc.n))
        rh = b.solve_queue(theta, x_h)
    assert np.array_equal(rq["status"], st["status"])
    assert np.array_equal(rh["status"], st["status"])
    assert np.array_equal(rq["iters"], st["iters"])
    conv = st["status"] == bipm.CONVERGED
    for j in np.flatnonzero(conv):
        assert e_v(x_q[j].cpu().numpy(), x_b[j]) <= 1e-9
        assert e_v(x_h[j], x_b[j]) <= 1e-9
    assert np.all(rq["kkt_err"][conv] <= 1e-6)


def test_queue_parks_stragglers_for_block_teams(bipm):
    """The benchmark's queue shape (more slots than resident warps): problems
    still running after the warp visit are parked and finished by block teams.
    Every problem gets a result; the long-running (parked) ones agree with the
    batch solve of the same problems and, on a sample, with the oracle."""
    desc, theta = make_batch("track", 8192)
    res = bipm.Batch(desc, 4096, bipm.Options(precision=1, fp32_switch=-1.0))
    x = np.empty((8192, desc.n))
    r = res.solve_queue(theta, x)
    res.close()
    assert np.all(r["status"] != bipm.RUNNING) and np.all(r["status"] != bipm.EMPTY)
    conv = r["status"] == bipm.CONVERGED
    assert conv.mean() >= 0.95
    assert np.all(r["kkt_err"][conv] <= 1e-6)
    long_ids = np.nonzero(r["iters"] > 96)[0]
    assert len(long_ids) >= 20, len(long_ids)
    sel = long_ids[:256]
    with bipm.Batch(desc, len(sel), bipm.Options(precision=1, fp32_switch=-1.0)) as b:
        b.set_problems(np.ascontiguousarray(theta[sel]))
        b.solve()
        st = b.get_stats()
        xb, yb, zlb, zub = b.get_solution()
    same = r["status"][sel] == st["status"]
    assert same.mean() >= 0.95
    both = same & (st["status"] == bipm.CONVERGED) & (r["iters"][sel] == st["iters"])
    for j in np.nonzero(both)[0]:
        assert e_v(x[sel[j]], xb[j]) <= 1e-6
    # four parked problems against the oracle, with the batch solve's multipliers
    pick = np.linspace(0, len(sel) - 1, 4).astype(int)
    ores = oracle_solve_batch(desc, theta[sel[pick]])
    splits = 0
    for o, t in zip(ores, pick):
        j = int(sel[t])
        splits += check_outcome(desc, theta[j], st["status"][t], xb[t], yb[t], zlb[t], zub[t], o["status"])
    assert splits <= 1
