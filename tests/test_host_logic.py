"""Host-side logic around the CUDA library (CPU): result-record parsing of the
binding, the autotuner's choice, the warm-start network's shape, and the
dense enumeration of bounded variables the kernels iterate over (restated
here from its definition: inputs, then slacks, then elastics)."""

import ctypes

import numpy as np
import pytest

from paper_2606_26341_gb300 import autotune, bipm, warmstart
from workloads import ProblemDesc, make_batch


def test_result_records_round_trip_through_bytes():
    n = 5
    arr = (bipm.ResultC * n)()
    for j in range(n):
        arr[j].status = j % 3
        arr[j].iters = 10 * j
        arr[j].warm = j % 2
        arr[j].warm_iters = 7 * j
        arr[j].obj = 0.5 * j
        arr[j].kkt_err = 1e-7 * j
    raw = ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(arr))
    r = bipm.results_from_bytes(raw)
    assert list(r["status"]) == [j % 3 for j in range(n)]
    assert list(r["iters"]) == [10 * j for j in range(n)]
    assert list(r["warm_iters"]) == [7 * j for j in range(n)]
    np.testing.assert_array_equal(r["obj"], 0.5 * np.arange(n))
    assert bipm.RESULT_DTYPE.itemsize == ctypes.sizeof(bipm.ResultC)


def test_autotuner_picks_the_fastest_candidate(monkeypatch):
    """Precision forms first, then one schedule knob at a time from the best so far."""
    rates = {(2, 0.0, 0): 10.0, (1, -1.0, 0): 30.0, (1, 100.0, 0): 20.0, (1, -1.0, 1): 25.0, (0, 0.0, 1): 5.0}

    def fake(desc, th, o, cap, stream=None):
        r = rates[(o.precision, o.fp32_switch, o.mu_strategy)]
        # a faster schedule: visit cap 160 and 128-thread teams, 1.25x the slots
        r += 2.0 * (o.visit_cap == 160) + 1.0 * (o.team_threads == 128) + 0.5 * (cap == 125)
        r -= 3.0 * (o.warps_per_sm in (16, 20))
        return r

    monkeypatch.setattr(autotune, "measure", fake)
    best, table = autotune.autotune(None, None, 100)
    o = best.options
    assert (o.precision, o.fp32_switch) == (1, -1.0)
    assert (o.visit_cap, o.team_threads, o.warps_per_sm or 24, best.slots) == (160, 128, 24, 125)
    assert [row["solves_per_s"] for row in table[:5]] == [10.0, 30.0, 20.0, 25.0, 5.0]
    # 5 forms + 2 visit caps + 2 warp counts + 1 team size + 1 slot count
    assert len(table) == 11
    assert {row["stage"] for row in table} == {"precision", "visit_cap", "warps_per_sm", "team_threads",
                                                "slot_factor"}
    # without the schedule search only the forms are measured
    best, table = autotune.autotune(None, None, 100, schedule=False)
    assert len(table) == 5 and best.slots == 100


def test_warm_start_network_shape_follows_the_family():
    desc, _ = make_batch("cyl", 1)
    assert warmstart.widths(desc) == (162, 256, 256, 256, 652)
    short = ProblemDesc(nq=1, horizon=12, dt=0.05, n_cyl=50)
    assert warmstart.widths(short, k_near=10) == (42, 256, 256, 256, 12 * 13 + 4 * 12)


def _bounded_dense(desc, resto):
    """Positions of the bounded entries in the order the kernels enumerate them."""
    N, nx, nu, ni, n, m = desc.horizon, desc.nx, desc.nu, desc.ni, desc.n, desc.m

    def off_x(k):
        return 0 if k == 0 else (nx + nu) + (k - 1) * (nx + nu + ni)

    out = [off_x(k) + nx + a for k in range(N) for a in range(nu)]
    out += [off_x(k) + nx + (nu if k < N else 0) + r for k in range(1, N + 1) for r in range(ni)]
    if resto:
        out += list(range(n, n + 2 * m))
    return out


@pytest.mark.parametrize("name", ["nav1", "track", "multi4"])
def test_bounded_entries_are_exactly_the_inputs_and_slacks(name):
    """The dense numbering covers each bounded variable once and no free one."""
    from oracle.quadrotor import QuadNLP

    desc, theta = make_batch(name, 1, desc=None if name != "multi4" else
                             ProblemDesc(nq=4, horizon=6, dt=0.05, pair_dist=0.4))
    nlp = QuadNLP(desc, theta[0])
    pos = _bounded_dense(desc, resto=False)
    assert len(pos) == len(set(pos))
    bounded = set(np.nonzero(np.isfinite(nlp.xl) | np.isfinite(nlp.xu))[0])
    assert set(pos) == bounded
    assert len(_bounded_dense(desc, resto=True)) == len(pos) + 2 * desc.m


def test_iteration_summary_of_the_benchmark():
    import bench

    r = {"iters": np.array([5, 12, 25, 25, 40, 150, 500]), "status": np.array([1, 1, 1, 1, 1, 3, 2]),
         "obj": np.array([1.0, 2.0, 3.0, 4.0, 5.0, 100.0, 100.0])}
    s = bench.iteration_summary(r)
    assert s["max"] == 500 and s["p50"] == 25.0
    assert sum(s["histogram"].values()) == 7
    assert s["histogram"]["0-9"] == 1 and s["histogram"]["20-29"] == 2 and s["histogram"][">=500"] == 1
    assert s["objective_mean_converged"] == 3.0
