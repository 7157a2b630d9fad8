"""Measured selection of the solver's execution options for one workload.

The library exposes the choices that decide throughput on a given problem
family.  The precision form and the barrier update change the iteration path
but not the accuracy a converged problem is held to (E_0 <= tol in FP64); the
schedule changes no result beyond the order of floating-point sums:

* the precision form: FP32 derivative blocks with an FP64 factorisation
  (``precision=1, fp32_switch<0``), FP32 factorisation with FP64 refinement
  (``precision=1``, FP64 above the barrier scale ``fp32_switch``), or the
  double-float factorisation (``precision=2``), each with the monotone or the
  adaptive barrier update (``mu_strategy``; this changes the iteration path,
  not the accuracy a converged problem is held to);
* the schedule of the persistent queue (iteration-level batching, Sec. V):
  the visit cap after which a straggler is parked for the block teams, the
  resident warps per SM, the block-team size, and the number of slots (every
  slot beyond the resident warps is a spare slot that takes a parked
  straggler).

``autotune`` measures each precision form on a sample of the workload through
the queue path, then improves the schedule of the fastest form one knob at a
time (coordinate search: each knob's candidates with the others fixed at the
best so far).  The sample should hold at least twice as many problems as the
batch has slots, so that it runs in the regime of a long queue (every resident
warp busy, spare slots for stragglers) rather than in the ramp-down at its
end.  Everything it runs is the CUDA path.
"""

from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import bipm

DEFAULT_CANDIDATES = (
    bipm.Options(precision=2),
    bipm.Options(precision=1, fp32_switch=-1.0),
    bipm.Options(precision=1, fp32_switch=1e2),
    # the adaptive barrier update (Table I row 7) changes the path, not the accuracy
    # (converged = E_0 <= tol either way)
    bipm.Options(precision=1, fp32_switch=-1.0, mu_strategy=1),
    bipm.Options(precision=0, mu_strategy=1),
)

# schedule knobs and the values tried for each (the first is the library default)
SCHEDULE_KNOBS = (
    ("visit_cap", (96, 64, 160)),
    ("warps_per_sm", (24, 20, 16)),
    ("team_threads", (256, 128)),
    ("slot_factor", (1.0, 1.25)),   # slots = slot_factor x the batch size
)


@dataclasses.dataclass(frozen=True)
class Schedule:
    """Options plus the slot count of the queue they run in."""

    options: bipm.Options
    slots: int


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


def _row(options, slots, rate, stage):
    return {"stage": stage, "precision": options.precision, "fp32_switch": options.fp32_switch,
            "mu_strategy": "adaptive" if options.mu_strategy else "monotone",
            "visit_cap": options.visit_cap or 96, "warps_per_sm": options.warps_per_sm or 24,
            "team_threads": options.team_threads or 256, "slots": slots, "solves_per_s": rate}


def autotune(desc, theta_dev, capacity, candidates=DEFAULT_CANDIDATES, stream=None, schedule=True):
    """Returns (best Schedule, table of every measured candidate) for this workload sample.

    capacity is the batch size the caller solves per step; the schedule search
    may choose more slots than that (spare slots for stragglers)."""
    table = []
    rates = []
    for o in candidates:
        r = measure(desc, theta_dev, o, capacity, stream)
        rates.append(r)
        table.append(_row(o, capacity, r, "precision"))
    i = int(np.argmax(rates))
    best_opt, best_slots, best_rate = candidates[i], capacity, rates[i]
    if schedule:
        for knob, values in SCHEDULE_KNOBS:
            for v in values[1:]:
                if knob == "slot_factor":
                    opt, slots = best_opt, int(round(capacity * v))
                else:
                    opt, slots = dataclasses.replace(best_opt, **{knob: v}), best_slots
                r = measure(desc, theta_dev, opt, slots, stream)
                table.append(_row(opt, slots, r, knob))
                if r > best_rate:
                    best_opt, best_slots, best_rate = opt, slots, r
    return Schedule(best_opt, best_slots), table
