"""bipm_solve_static, the entry point that allocates no device memory.

It exists for callers that cannot allocate when they need a solve (inside a
CUDA stream capture, in allocation-free real-time loops, under a fixed memory
budget): its workspace is a fixed array inside the library.  These tests call
it through the C ABI twice in a row and compare every result with the same
problems solved by the allocating queue entry point (bipm_solve_queue).  The
file sorts last so that a failure here comes after every other test has run.
"""

import numpy as np
import pytest

from workloads import ProblemDesc, make_batch

pytestmark = pytest.mark.gpu


def _e_v(a, b):
    return float(np.max(np.abs(a - b) / (1.0 + np.abs(b))))


def _reference(bipm, desc, theta_dev, count):
    import torch

    x = torch.empty((count, desc.n), dtype=torch.float64, device="cuda")
    raw = torch.empty(count * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with bipm.Batch(desc, 16) as b:
        b.solve_queue(theta_dev, x, raw)
    return x.cpu().numpy(), bipm.results_from_bytes(raw.cpu().numpy())


def test_static_workspace_matches_queue_on_two_calls_in_a_row():
    import torch

    from paper_2606_26341_gb300 import bipm

    desc, theta = make_batch("nav1", 80)
    theta_dev = torch.as_tensor(theta, device="cuda")
    # two consecutive calls on overlapping problem sets: the second one finds
    # the first one's leftovers in the shared array
    for lo, hi in ((0, 48), (16, 80)):
        count = hi - lo
        th = theta_dev[lo:hi].contiguous()
        x = torch.full((count, desc.n), float("nan"), dtype=torch.float64, device="cuda")
        raw = torch.zeros(count * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        bipm.solve_static(desc, th, x, raw)
        got = bipm.results_from_bytes(raw.cpu().numpy())
        x_ref, ref = _reference(bipm, desc, th, count)
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["iters"], ref["iters"])
        conv = ref["status"] == bipm.CONVERGED
        assert conv.mean() > 0.9
        xs = x.cpu().numpy()
        for j in np.flatnonzero(conv):
            assert _e_v(xs[j], x_ref[j]) <= 1e-9, (lo + j, _e_v(xs[j], x_ref[j]))
        assert np.all(got["kkt_err"][conv] <= 1e-6)


def test_static_workspace_rejects_a_problem_that_does_not_fit():
    import torch

    from paper_2606_26341_gb300 import bipm

    desc = ProblemDesc(nq=8, horizon=1000, dt=0.05, pair_dist=0.4)
    th = torch.zeros((1, 12 * 8 + 6 * 8), dtype=torch.float64, device="cuda")
    raw = torch.zeros(bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(bipm.BipmError, match="too large for the static workspace"):
        bipm.solve_static(desc, th, None, raw)
