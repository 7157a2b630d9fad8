"""Measured selection of the solver's execution options for one workload.

The library exposes the choices that decide throughput on a given problem
family: the factorisation precision (FP64; FP32 with FP64 refinement;
double-float) and, for the FP32 form, the barrier scale above which an
iteration falls back to an FP64 factorisation (``fp32_switch``; negative =
FP32 derivative blocks with an FP64 factorisation).  ``autotune`` runs each candidate on a sample of the
workload through the queue (iteration-level batching) path and returns the
fastest in converged solves per second.  The sample should hold at least twice
as many problems as the batch has slots, so that it runs in the same regime as
a long queue (every resident warp busy, spare slots for stragglers) rather
than in the ramp-down at its end.  Everything it runs is the CUDA path.
"""

from __future__ import annotations

import time

import numpy as np

from . import bipm

DEFAULT_CANDIDATES = (
    bipm.Options(precision=2),
    bipm.Options(precision=1, fp32_switch=-1.0),
    bipm.Options(precision=1, fp32_switch=1e2),
)


def measure(desc, theta_dev, options, capacity, stream=None):
    """Converged solves/s of one queue solve of theta_dev (device tensor)."""
    import torch

    n = theta_dev.shape[0]
    res = torch.empty(n * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=theta_dev.device)
    with bipm.Batch(desc, capacity, options, stream=stream) as b:
        b.solve_queue(theta_dev[: min(n, 256)], None, res)  # warm-up (module load, caches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.solve_queue(theta_dev, None, res)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    r = bipm.results_from_bytes(res.cpu().numpy())
    return float(np.sum(r["status"] == bipm.CONVERGED)) / dt


def autotune(desc, theta_dev, capacity, candidates=DEFAULT_CANDIDATES, stream=None):
    """Returns (best Options, [(Options, solves/s), ...]) for this workload sample."""
    table = [(o, measure(desc, theta_dev, o, capacity, stream)) for o in candidates]
    best = max(table, key=lambda t: t[1])[0]
    return best, table
