"""Seeded synthetic inputs for the batched quadrotor NMPC workloads.

This package only draws random problem parameters (initial states, references,
obstacle positions and radii).  It holds none of the solver's arithmetic: no
dynamics, no cost, no constraint and no derivative.  Both the CUDA path (through
its Python binding) and the CPU oracle take their inputs from here, so the two
sides see identical problems.

Every problem is drawn from its own counter-based SplitMix64 stream keyed by
(workload seed, problem id), so problem j can be regenerated alone.
"""

from .mlp_init import mlp_init  # noqa: F401
from .quadrotor import (  # noqa: F401
    WORKLOADS,
    ProblemDesc,
    QuatProblemDesc,
    SplitMix64,
    make_batch,
    make_mixed,
    mixed_classes,
    n_theta,
    theta_layout,
)
