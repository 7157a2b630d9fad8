"""bipm_solve_static, the entry point that allocates no device memory.

It is for callers that cannot allocate when they need a solve: real-time
control loops that must stay out of the CUDA allocator, and processes whose
device memory is budgeted up front.  Its workspace is a fixed array inside the
library.  These tests call it through the C ABI and compare every result with
the same problems solved by the allocating queue entry point
(bipm_solve_queue): twice in a row in each precision form, and once where the
array holds fewer slots than there are problems, so that slots are refilled
from the queue.  The file sorts last so that a failure here comes after every
other test has run.
"""

import numpy as np
import pytest

from workloads import ProblemDesc, make_batch

pytestmark = pytest.mark.gpu


def _e_v(a, b):
    return float(np.max(np.abs(a - b) / (1.0 + np.abs(b))))


def _reference(bipm, desc, theta_dev, count, options):
    import torch

    x = torch.empty((count, desc.n), dtype=torch.float64, device="cuda")
    raw = torch.empty(count * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with bipm.Batch(desc, 16, options) as b:
        b.solve_queue(theta_dev, x, raw)
    return x.cpu().numpy(), bipm.results_from_bytes(raw.cpu().numpy())


def _compare(bipm, desc, th, options):
    import torch

    count = th.shape[0]
    x = torch.full((count, desc.n), float("nan"), dtype=torch.float64, device="cuda")
    raw = torch.zeros(count * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    bipm.solve_static(desc, th, x, raw, options)
    got = bipm.results_from_bytes(raw.cpu().numpy())
    x_ref, ref = _reference(bipm, desc, th, count, options)
    assert np.array_equal(got["status"], ref["status"])
    assert np.array_equal(got["iters"], ref["iters"])
    xs = x.cpu().numpy()
    conv = ref["status"] == bipm.CONVERGED
    for j in np.flatnonzero(conv):
        assert _e_v(xs[j], x_ref[j]) <= 1e-9, (j, _e_v(xs[j], x_ref[j]))
    assert np.all(got["kkt_err"][conv] <= 1e-6)
    return conv


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_static_workspace_matches_queue_on_two_calls_in_a_row(precision):
    import torch

    from paper_2606_26341_gb300 import bipm

    desc, theta = make_batch("nav1", 80)
    theta_dev = torch.as_tensor(theta, device="cuda")
    opt = bipm.Options(precision=precision)
    # two consecutive calls on overlapping problem sets: the second one finds
    # the first one's leftovers in the shared array
    for lo, hi in ((0, 48), (16, 80)):
        conv = _compare(bipm, desc, theta_dev[lo:hi].contiguous(), opt)
        assert conv.mean() > 0.9


def test_static_workspace_refills_slots_when_fewer_fit_than_problems():
    """Four quadrotors at horizon 12: one problem's workspace is 1.38 MB, so the
    64 MiB array holds 48 slots and the 56 problems pass through them as a
    queue."""
    import torch

    from paper_2606_26341_gb300 import bipm

    desc = ProblemDesc(nq=4, horizon=12, dt=0.05, pair_dist=0.4)
    _, theta = make_batch("multi4", 56, desc=desc)
    _compare(bipm, desc, torch.as_tensor(theta, device="cuda"), bipm.Options(precision=0))


def test_static_workspace_rejects_a_problem_that_does_not_fit():
    import torch

    from paper_2606_26341_gb300 import bipm

    desc = ProblemDesc(nq=8, horizon=1000, dt=0.05, pair_dist=0.4)
    th = torch.zeros((1, 12 * 8 + 6 * 8), dtype=torch.float64, device="cuda")
    raw = torch.zeros(bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(bipm.BipmError, match="too large for the static workspace"):
        bipm.solve_static(desc, th, None, raw)
