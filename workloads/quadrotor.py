"""Random problem parameters for the quadrotor NMPC workloads.

The paper evaluates on quadrotor NMPC scenarios it describes only in words
(Sec. VI: navigation past obstacles, reference tracking with obstacles,
multi-quadrotor swaps).  No dataset exists, so the workloads below stand in for
them with seeded synthetic draws of the same shape.

Parameter vector theta of one problem (float64), in this order:
    xbar    nx      initial state of every quadrotor: (p, v, eta, omega), 12 per
                    quadrotor; (p, q, v, omega), 13 per quadrotor, for the
                    quaternion model of QuatProblemDesc
    ref      6*nq   per quadrotor reference circle (cx, cy, cz, radius, rate, phase);
                    radius 0 means a fixed goal at (cx, cy, cz)
    spheres  4*n_sph  (cx, cy, cz, r) of every spherical obstacle
    cyls     3*n_cyl  (cx, cy, r) of every vertical cylinder
    moving   7*n_mov  (cx, cy, cz, r, vx, vy, vz) of every moving sphere: its centre
                      at time t is c + v t (the time-varying obstacles of Sec. VI)
Shared (not per problem): nq, horizon N, dt, n_sph, n_cyl and the pairwise
minimum distance d (0 disables the pairwise constraints).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1)) % (hi - lo + 1)


def problem_stream(seed: int, problem_id: int) -> SplitMix64:
    """Independent stream for problem `problem_id` of workload `seed`."""
    mix = SplitMix64(seed * 0x1000003 + 0x51ED2701)
    base = mix.next_u64()
    return SplitMix64(base ^ ((problem_id * 0xD1342543DE82EF95) & MASK64))


@dataclasses.dataclass(frozen=True)
class ProblemDesc:
    """Shared structure of one batch of problems (identical f, c and bounds)."""

    nq: int = 1
    horizon: int = 10
    dt: float = 0.05
    n_sph: int = 0
    n_cyl: int = 0
    pair_dist: float = 0.0
    n_mov: int = 0  # moving spheres (centre c + v t at stage time t = k dt)

    @property
    def nx(self) -> int:
        return 12 * self.nq

    @property
    def nu(self) -> int:
        return 4 * self.nq

    # the model of the problem class: the 12-state Euler-angle quadrotor (the one
    # the CUDA path solves) or the 13-state quaternion one (QuatProblemDesc)
    model = "euler12"

    @property
    def n_pairs(self) -> int:
        return self.nq * (self.nq - 1) // 2 if self.pair_dist > 0 else 0

    @property
    def ni(self) -> int:
        return self.nq * (self.n_sph + self.n_cyl + self.n_mov) + self.n_pairs

    @property
    def n(self) -> int:
        return self.nx * (self.horizon + 1) + (self.nu + self.ni) * self.horizon

    @property
    def m(self) -> int:
        return self.nx * (self.horizon + 1) + self.ni * self.horizon


@dataclasses.dataclass(frozen=True)
class QuatProblemDesc(ProblemDesc):
    """ProblemDesc of the 13-state quaternion quadrotor model of Sec. VI (state
    (p, q, v, omega) per quadrotor, four rotor speeds as inputs); the same
    fields, 13 states per quadrotor."""

    model = "quat13"

    @property
    def nx(self) -> int:
        return 13 * self.nq


def theta_layout(desc: ProblemDesc) -> dict:
    """Offsets of the parameter groups inside theta."""
    o_x = 0
    o_ref = o_x + desc.nx
    o_sph = o_ref + 6 * desc.nq
    o_cyl = o_sph + 4 * desc.n_sph
    o_mov = o_cyl + 3 * desc.n_cyl
    end = o_mov + 7 * desc.n_mov
    return {"xbar": o_x, "ref": o_ref, "sph": o_sph, "cyl": o_cyl, "mov": o_mov, "end": end}


def n_theta(desc: ProblemDesc) -> int:
    return theta_layout(desc)["end"]


# ---------------------------------------------------------------- workloads --
# Seeds follow 1000 + workload number.

def _nav1(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """Single quadrotor flying to the origin past one sphere of radius 0.5."""
    th = np.zeros(n_theta(desc))
    lay = theta_layout(desc)
    r = 0.5
    while True:
        p0 = np.array([rng.uniform(-3, 3) for _ in range(3)])
        c = 0.5 * p0 + np.array([rng.uniform(-0.25, 0.25) for _ in range(3)])
        if np.linalg.norm(p0 - c) >= r + 0.2 and np.linalg.norm(c) >= r + 0.2:
            break
    th[lay["xbar"]:lay["xbar"] + 3] = p0
    th[lay["ref"]:lay["ref"] + 6] = 0.0
    th[lay["sph"]:lay["sph"] + 4] = [c[0], c[1], c[2], r]
    return th


def _circle_point(ref, t):
    cx, cy, cz, rad, rate, ph = ref
    a = rate * t + ph
    p = np.array([cx + rad * math.cos(a), cy + rad * math.sin(a), cz])
    v = np.array([-rad * rate * math.sin(a), rad * rate * math.cos(a), 0.0])
    return p, v


def _track(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """Tracking a random circular reference at 1-2 m/s past spheres near the path."""
    th = np.zeros(n_theta(desc))
    lay = theta_layout(desc)
    cx, cy, cz = rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(1, 2)
    rad = rng.uniform(1.5, 3.0)
    speed = rng.uniform(1.0, 2.0)
    ref = (cx, cy, cz, rad, speed / rad, rng.uniform(0, 2 * math.pi))
    p_ref0, v_ref0 = _circle_point(ref, 0.0)
    p0 = p_ref0 + np.array([rng.uniform(-0.5, 0.5) for _ in range(3)])
    th[lay["xbar"]:lay["xbar"] + 3] = p0
    th[lay["xbar"] + 3:lay["xbar"] + 6] = v_ref0
    th[lay["ref"]:lay["ref"] + 6] = ref
    t_end = desc.horizon * desc.dt
    for j in range(desc.n_sph):
        while True:
            r = rng.uniform(0.3, 0.8)
            pj, _ = _circle_point(ref, rng.uniform(0, t_end))
            c = pj + np.array([rng.uniform(-0.4, 0.4) for _ in range(3)])
            if np.linalg.norm(p0 - c) >= r + 0.1:
                break
        th[lay["sph"] + 4 * j:lay["sph"] + 4 * j + 4] = [c[0], c[1], c[2], r]
    return th


def _track_moving(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """Reference tracking with time-varying obstacles (the scaling-difficulty task of
    Sec. VI): the tracking workload's circle (speed U[1, 2] m/s, the paper's range of
    the reference velocity) with spheres that move at constant velocity
    U[-0.5, 0.5]^3 m/s and pass near the reference: sphere j is at p_ref(t_j) +
    U[-0.3, 0.3]^3 at t_j ~ U[0, N dt], radius U[0.3, 0.6]; redrawn until it stays
    0.1 m clear of the start at t = 0."""
    th = _track(rng, dataclasses.replace(desc, n_sph=0, n_mov=0))
    th = np.concatenate([th, np.zeros(n_theta(desc) - th.size)])
    lay = theta_layout(desc)
    ref = th[lay["ref"]:lay["ref"] + 6]
    p0 = th[lay["xbar"]:lay["xbar"] + 3]
    t_end = desc.horizon * desc.dt
    for j in range(desc.n_mov):
        while True:
            r = rng.uniform(0.3, 0.6)
            tj = rng.uniform(0, t_end)
            pj, _ = _circle_point(ref, tj)
            v = np.array([rng.uniform(-0.5, 0.5) for _ in range(3)])
            cj = pj + np.array([rng.uniform(-0.3, 0.3) for _ in range(3)])
            c0 = cj - v * tj
            if np.linalg.norm(p0 - c0) >= r + 0.1:
                break
        th[lay["mov"] + 7 * j:lay["mov"] + 7 * j + 7] = [c0[0], c0[1], c0[2], r, v[0], v[1], v[2]]
    return th


def _track_quat(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """The tracking workload for the 13-state quaternion model: the same draws as
    _track (reference circle, start, spheres), the start state written as
    (p, q = (1, 0, 0, 0), v, omega = 0): level attitude at zero yaw, where the body
    frame's velocity equals the world frame's."""
    d12 = dataclasses.replace(ProblemDesc(), nq=desc.nq, horizon=desc.horizon, dt=desc.dt, n_sph=desc.n_sph)
    t12 = _track(rng, d12)
    l12, lay = theta_layout(d12), theta_layout(desc)
    th = np.zeros(n_theta(desc))
    x12 = t12[l12["xbar"]:l12["xbar"] + 12]
    th[lay["xbar"]:lay["xbar"] + 3] = x12[0:3]
    th[lay["xbar"] + 3] = 1.0
    th[lay["xbar"] + 7:lay["xbar"] + 10] = x12[3:6]
    th[lay["ref"]:] = t12[l12["ref"]:]
    return th


def _spread_points(rng: SplitMix64, count: int, lo, hi, min_gap: float):
    pts = []
    while len(pts) < count:
        q = np.array([rng.uniform(lo[i], hi[i]) for i in range(3)])
        if all(np.linalg.norm(q - o) >= min_gap for o in pts):
            pts.append(q)
    return pts


def _multi(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """nq quadrotors flying from random starts to random goals in a 10 m cube."""
    th = np.zeros(n_theta(desc))
    lay = theta_layout(desc)
    starts = _spread_points(rng, desc.nq, (0, 0, 0), (10, 10, 10), 1.0)
    goals = _spread_points(rng, desc.nq, (0, 0, 0), (10, 10, 10), 1.0)
    for i in range(desc.nq):
        th[lay["xbar"] + 12 * i:lay["xbar"] + 12 * i + 3] = starts[i]
        th[lay["ref"] + 6 * i:lay["ref"] + 6 * i + 3] = goals[i]
    for j in range(desc.n_sph):
        # one obstacle between the first start and its goal (single-quad case)
        while True:
            c = 0.5 * (starts[0] + goals[0]) + np.array([rng.uniform(-0.25, 0.25) for _ in range(3)])
            if all(np.linalg.norm(s - c) >= 0.7 for s in starts) and all(
                np.linalg.norm(g - c) >= 0.7 for g in goals
            ):
                break
            goals = _spread_points(rng, desc.nq, (0, 0, 0), (10, 10, 10), 1.0)
            for i in range(desc.nq):
                th[lay["ref"] + 6 * i:lay["ref"] + 6 * i + 3] = goals[i]
        th[lay["sph"] + 4 * j:lay["sph"] + 4 * j + 4] = [c[0], c[1], c[2], 0.5]
    return th


def _cyl(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """Single quadrotor to (0, 0, 1) through 20-50 cylinders in a 20 m x 20 m area.

    Problems with fewer than desc.n_cyl cylinders are padded with far-away
    cylinders (centre 1000 m out, radius 0.2), which never become active.
    """
    th = np.zeros(n_theta(desc))
    lay = theta_layout(desc)
    n_real = rng.randint(20, min(50, desc.n_cyl)) if desc.n_cyl >= 20 else desc.n_cyl
    cyl = []
    while len(cyl) < n_real:
        c = (rng.uniform(-10, 10), rng.uniform(-10, 10), rng.uniform(0.2, 0.6))
        if math.hypot(c[0], c[1]) >= c[2] + 0.3:
            cyl.append(c)
    while True:
        p0 = (rng.uniform(-10, 10), rng.uniform(-10, 10), rng.uniform(0.5, 2.0))
        if all(math.hypot(p0[0] - c[0], p0[1] - c[1]) >= c[2] + 0.3 for c in cyl):
            break
    th[lay["xbar"]:lay["xbar"] + 3] = p0
    th[lay["ref"]:lay["ref"] + 6] = [0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    for j in range(desc.n_cyl):
        c = cyl[j] if j < n_real else (1000.0 + 10.0 * j, 1000.0, 0.2)
        th[lay["cyl"] + 3 * j:lay["cyl"] + 3 * j + 3] = c
    return th


def _swap(rng: SplitMix64, desc: ProblemDesc) -> np.ndarray:
    """The multi-quadrotor swap (consensus) task of the paper's dimension-scaling
    experiment: nq quadrotors start evenly spaced on a horizontal circle (radius
    U[1.5, 2.5] m, height U[1, 2] m, rotated by a random angle, each start
    perturbed by U[-0.1, 0.1]^3) and each must reach the antipodal start, so every
    path crosses the centre and the pairwise minimum-distance rows are active."""
    th = np.zeros(n_theta(desc))
    lay = theta_layout(desc)
    rad, h, rot = rng.uniform(1.5, 2.5), rng.uniform(1.0, 2.0), rng.uniform(0, 2 * math.pi)
    pts = []
    for i in range(desc.nq):
        a = rot + 2 * math.pi * i / desc.nq
        pts.append(np.array([rad * math.cos(a), rad * math.sin(a), h]))
    for i in range(desc.nq):
        p0 = pts[i] + np.array([rng.uniform(-0.1, 0.1) for _ in range(3)])
        goal = pts[(i + desc.nq // 2) % desc.nq] if desc.nq % 2 == 0 else -pts[i] + np.array([0, 0, 2 * h])
        th[lay["xbar"] + 12 * i:lay["xbar"] + 12 * i + 3] = p0
        th[lay["ref"] + 6 * i:lay["ref"] + 6 * i + 3] = goal
    return th


WORKLOADS = {
    # name: (seed, desc, drawer, default batch)
    "nav1": (1001, ProblemDesc(nq=1, horizon=10, dt=0.05, n_sph=1), _nav1, 64),
    "track": (1002, ProblemDesc(nq=1, horizon=30, dt=0.05, n_sph=3), _track, 4096),
    "multi4": (1003, ProblemDesc(nq=4, horizon=25, dt=0.05, pair_dist=0.4), _multi, 1024),
    "cyl": (1005, ProblemDesc(nq=1, horizon=40, dt=0.05, n_cyl=50), _cyl, 16384),
    # the paper's swap task (Sec. VI, dimension scaling) with 2 and 4 quadrotors, horizon 30
    "swap2": (1006, ProblemDesc(nq=2, horizon=30, dt=0.05, pair_dist=0.4), _swap, 1024),
    "swap4": (1007, ProblemDesc(nq=4, horizon=30, dt=0.05, pair_dist=0.4), _swap, 1024),
    # reference tracking with three time-varying (moving) spherical obstacles
    "track_moving": (1008, ProblemDesc(nq=1, horizon=30, dt=0.05, n_mov=3), _track_moving, 4096),
    # the tracking workload on the paper's 13-state quaternion model at its dt = 0.1 s and
    # horizon 30 (oracle side only: the CUDA path solves the 12-state model)
    "track_quat": (1009, QuatProblemDesc(nq=1, horizon=30, dt=0.1, n_sph=3), _track_quat, 4096),
}


def make_batch(name: str, count: int | None = None, first_id: int = 0,
               desc: ProblemDesc | None = None):
    """Draw `count` problems of workload `name` starting at problem id `first_id`.

    Returns (desc, theta) with theta of shape (count, n_theta(desc)).
    `desc` may override the workload's structure (e.g. a shorter horizon for
    quick tests); the drawing rules stay those of the named workload.
    """
    seed, base_desc, drawer, default_count = WORKLOADS[name]
    desc = desc or base_desc
    count = default_count if count is None else count
    th = np.stack([drawer(problem_stream(seed, first_id + j), desc) for j in range(count)]) \
        if count > 0 else np.zeros((0, n_theta(desc)))
    return desc, np.ascontiguousarray(th, dtype=np.float64)


# --------------------------------------------------------- uneven queue --
# Structure classes of the uneven queue: 1-8 quadrotors x horizons 10, 20, 30,
# 50, configured as the multi-quadrotor workload (pairwise distance 0.4); a
# single quadrotor flies past one sphere instead.
MIXED_SEED = 1004
MIXED_HORIZONS = (10, 20, 30, 50)


def mixed_classes(max_quads: int = 8, horizons=MIXED_HORIZONS):
    """The structure classes (nq, horizon), nq = 1..max_quads, in that order
    (32 classes for the default arguments)."""
    out = []
    for nq in range(1, max_quads + 1):
        for N in horizons:
            out.append(ProblemDesc(nq=nq, horizon=N, dt=0.05, n_sph=1 if nq == 1 else 0,
                                   pair_dist=0.0 if nq == 1 else 0.4))
    return out


def make_mixed(count: int, first_id: int = 0, max_quads: int = 8, horizons=MIXED_HORIZONS):
    """Draw `count` problems of the uneven queue: each draws its quadrotor count
    (uniform 1..max_quads) and horizon (uniform over `horizons`) from its own
    stream, then its parameters as the multi-quadrotor workload.

    Returns (classes, cls, theta_packed): the class list of
    mixed_classes(max_quads, horizons), the class index of every problem and the
    concatenated parameter rows."""
    classes = mixed_classes(max_quads, horizons)
    index = {(c.nq, c.horizon): k for k, c in enumerate(classes)}
    cls = np.zeros(count, dtype=np.int32)
    rows = []
    for j in range(count):
        rng = problem_stream(MIXED_SEED, first_id + j)
        nq = rng.randint(1, max_quads)
        N = horizons[rng.randint(0, len(horizons) - 1)]
        k = index[(nq, N)]
        cls[j] = k
        rows.append(_multi(rng, classes[k]))
    theta = np.concatenate(rows) if rows else np.zeros(0)
    return classes, cls, np.ascontiguousarray(theta, dtype=np.float64)
