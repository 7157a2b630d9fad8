"""The boundary's time budget (bipm_options.time_limit_ms, BIPM_ETIMEOUT) on
the GPU, through the C ABI.

A budget that runs out stops every problem at an iteration boundary and ends
the call with BIPM_ETIMEOUT; the batch stays usable and later calls continue
the problems where they stopped, to the same results a call without a budget
gives.  A queue that runs out reports started problems as RUNNING and the
rest as EMPTY.  Nothing here faults or hangs the GPU: the budget is read from
the device clock before each iteration.
"""

import numpy as np
import pytest

from workloads import make_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bipm():
    import torch

    assert torch.cuda.is_available()
    from paper_2606_26341_gb300 import bipm as b

    b.load_library()
    return b


def test_solve_resumes_after_the_time_budget_runs_out(bipm):
    desc, theta = make_batch("nav1", 64)
    with bipm.Batch(desc, 64, bipm.Options(precision=0, schedule=1)) as b:
        b.set_problems(theta)
        b.solve()
        ref = b.get_stats()
        x_ref, _, _, _ = b.get_solution()
    with bipm.Batch(desc, 64, bipm.Options(precision=0, schedule=1, time_limit_ms=1)) as b:
        b.set_problems(theta)
        calls, running_seen = 0, False
        while True:
            calls += 1
            assert calls < 5000
            try:
                b.solve()
                break
            except bipm.BipmError as e:
                assert e.code == bipm.ETIMEOUT, e
                running_seen |= bool(np.any(b.get_stats()["status"] == bipm.RUNNING))
        st = b.get_stats()
        x, _, _, _ = b.get_solution()
    assert calls > 1 and running_seen
    # the interrupted solve follows exactly the same iterations
    assert np.array_equal(st["status"], ref["status"])
    assert np.array_equal(st["iters"], ref["iters"])
    assert np.array_equal(x, x_ref)


def test_queue_reports_running_and_empty_when_the_budget_runs_out(bipm):
    desc, theta = make_batch("track", 8192)
    with bipm.Batch(desc, 1024, bipm.Options(precision=1, fp32_switch=-1.0, time_limit_ms=30)) as b:
        with pytest.raises(bipm.BipmError) as ei:
            b.solve_queue(theta)
    assert ei.value.code == bipm.ETIMEOUT
    r = ei.value.results
    st = r["status"]
    assert np.all(st != bipm.RUNNING) or np.any(st == bipm.RUNNING)
    assert np.any(st == bipm.EMPTY)  # 8192 problems do not finish in 30 ms
    assert np.any((st == bipm.RUNNING) | (st == bipm.CONVERGED))
    conv = st == bipm.CONVERGED
    assert np.all(r["kkt_err"][conv] <= 1e-6)
    # the context and library stay usable: the same problems without a budget
    with bipm.Batch(desc, 1024, bipm.Options(precision=1, fp32_switch=-1.0)) as b:
        r2 = b.solve_queue(theta[:512])
    assert np.all(r2["status"] != bipm.EMPTY) and np.all(r2["status"] != bipm.RUNNING)
    assert np.mean(r2["status"] == bipm.CONVERGED) > 0.9
