"""Python binding of the bipm C ABI (include/bipm.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and back.  It fails loudly when the
library cannot be built or loaded: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

RUNNING, CONVERGED, MAX_ITER, RESTO_FAILED, EVAL_ERROR, TINY_STEP, EMPTY, FP64_ESCALATION_FAILED = range(8)
STATUS_NAMES = {RUNNING: "running", CONVERGED: "converged", MAX_ITER: "max_iter",
                RESTO_FAILED: "resto_failed", EVAL_ERROR: "eval_error", TINY_STEP: "tiny_step",
                EMPTY: "empty", FP64_ESCALATION_FAILED: "fp64_escalation_failed"}
EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT = -22, -12, -100, -101, -102
FILTER_CAP = 64


class ProblemDescC(ctypes.Structure):
    _fields_ = [("n_quads", ctypes.c_int), ("horizon", ctypes.c_int), ("dt", ctypes.c_double),
                ("n_spheres", ctypes.c_int), ("n_cylinders", ctypes.c_int),
                ("pair_dist", ctypes.c_double), ("n_moving", ctypes.c_int)]


def desc_c(desc):
    """The C record of a workloads.ProblemDesc (the 12-state model; any other model
    is rejected, the library has no kernel for it)."""
    model = getattr(desc, "model", "euler12")
    if model != "euler12":
        raise ValueError(f"problem model {model!r}: the library solves the 12-state quadrotor model only")
    return ProblemDescC(desc.nq, desc.horizon, desc.dt, desc.n_sph, desc.n_cyl, desc.pair_dist,
                        getattr(desc, "n_mov", 0))


class OptionsC(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mu_init", ctypes.c_double),
                ("precision", ctypes.c_int), ("schedule", ctypes.c_int),
                ("fp32_switch", ctypes.c_double), ("warm_mu_init", ctypes.c_double),
                ("warm_bound_push", ctypes.c_double), ("warm_max_iter", ctypes.c_int),
                ("time_limit_ms", ctypes.c_int), ("visit_cap", ctypes.c_int),
                ("warps_per_sm", ctypes.c_int), ("team_threads", ctypes.c_int),
                ("watchdog", ctypes.c_int), ("soft_resto", ctypes.c_int), ("mu_strategy", ctypes.c_int)]


class StatsC(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("resto_iters", ctypes.c_int),
                ("soc", ctypes.c_int), ("inertia_corr", ctypes.c_int), ("ir_steps", ctypes.c_int),
                ("fp64_escalations", ctypes.c_int), ("tiny_steps", ctypes.c_int),
                ("factorizations", ctypes.c_int), ("solves", ctypes.c_int),
                ("trials", ctypes.c_int), ("fact32", ctypes.c_int), ("solve32", ctypes.c_int),
                ("reserved", ctypes.c_int),
                ("obj", ctypes.c_double), ("kkt_err", ctypes.c_double),
                ("primal_inf", ctypes.c_double), ("mu", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class ResultC(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("factorizations", ctypes.c_int),
                ("solves", ctypes.c_int), ("trials", ctypes.c_int), ("ir_steps", ctypes.c_int),
                ("fp64_escalations", ctypes.c_int), ("resto_iters", ctypes.c_int),
                ("fact32", ctypes.c_int), ("solve32", ctypes.c_int), ("warm", ctypes.c_int),
                ("warm_iters", ctypes.c_int), ("obj", ctypes.c_double), ("kkt_err", ctypes.c_double)]


RESULT_DTYPE = np.dtype([(f, "<i4" if t is ctypes.c_int else "<f8") for f, t in ResultC._fields_])


def results_from_bytes(buf) -> dict:
    """Per-problem result fields from the raw bytes of a device results buffer."""
    arr = np.frombuffer(bytes(buf), dtype=RESULT_DTYPE)
    return {f: arr[f].copy() for f in RESULT_DTYPE.names}


class IterateC(ctypes.Structure):
    _fields_ = [("x", _DP), ("y", _DP), ("zl", _DP), ("zu", _DP), ("p", _DP), ("nn", _DP),
                ("zp", _DP), ("zn", _DP), ("x_ref", _DP), ("filter", _DP), ("filter_r", _DP),
                ("mode", ctypes.c_int), ("status", ctypes.c_int), ("iter", ctypes.c_int),
                ("need_init", ctypes.c_int), ("need_y_ls", ctypes.c_int), ("tiny", ctypes.c_int),
                ("tiny_r", ctypes.c_int), ("n_filter", ctypes.c_int), ("n_filter_r", ctypes.c_int),
                ("mu", ctypes.c_double), ("dw_last", ctypes.c_double),
                ("theta_max", ctypes.c_double), ("theta_min", ctypes.c_double),
                ("mu_r", ctypes.c_double), ("dw_last_r", ctypes.c_double),
                ("theta_max_r", ctypes.c_double), ("theta_min_r", ctypes.c_double),
                ("zeta", ctypes.c_double), ("theta_ref", ctypes.c_double),
                ("wd_x", _DP), ("wd_y", _DP), ("wd_zl", _DP), ("wd_zu", _DP), ("wd_dx", _DP), ("wd_dy", _DP),
                ("wd_short", ctypes.c_int), ("wd_active", ctypes.c_int), ("wd_trials", ctypes.c_int),
                ("soft_active", ctypes.c_int), ("soft_iters", ctypes.c_int), ("reserved_wd", ctypes.c_int),
                ("wd_theta", ctypes.c_double), ("wd_phi", ctypes.c_double), ("wd_gdx", ctypes.c_double),
                ("wd_amax", ctypes.c_double), ("wd_amin", ctypes.c_double),
                ("mu_free", ctypes.c_int), ("n_refs", ctypes.c_int), ("mu_refs", ctypes.c_double * 4),
                ("mu_max", ctypes.c_double)]


EXPORTS = ["bipm_create_batch", "bipm_dims", "bipm_set_problems", "bipm_set_initial_guess",
           "bipm_solve", "bipm_step", "bipm_get_solution", "bipm_get_stats", "bipm_get_iterate",
           "bipm_set_iterate", "bipm_get_phase_cycles", "bipm_solve_queue", "bipm_solve_queue_warm", "bipm_solve_mixed",
           "bipm_solve_static", "bipm_warm_features", "bipm_warm_encode", "bipm_warm_decode",
           "bipm_mlp_create", "bipm_mlp_param_count", "bipm_mlp_set_params", "bipm_mlp_get_params",
           "bipm_mlp_forward", "bipm_mlp_loss_grad", "bipm_mlp_train_step", "bipm_mlp_destroy",
           "bipm_check_rsqrt", "bipm_last_error", "bipm_destroy"]
PHASES = ["eval", "derivs", "factor", "solve", "line_search", "other", "lsq_mult", "total"]

_LIB = None


def load_library(build_if_missing: bool = True):
    """Load libbipm.so (building it first if needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libbipm.so not found at {path}; build it with "
                           "paper_2606_26341_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i = ctypes.c_int
    lib.bipm_create_batch.argtypes = [ctypes.POINTER(ProblemDescC), i, ctypes.POINTER(OptionsC), vp,
                                      ctypes.POINTER(vp)]
    lib.bipm_dims.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.bipm_set_problems.argtypes = [vp, vp, i, i, i]
    lib.bipm_set_initial_guess.argtypes = [vp, vp, vp, i, i, i]
    lib.bipm_solve.argtypes = [vp]
    lib.bipm_step.argtypes = [vp, i]
    lib.bipm_get_solution.argtypes = [vp, vp, vp, vp, vp, i, i, i]
    lib.bipm_get_stats.argtypes = [vp, ctypes.POINTER(StatsC), i, i]
    lib.bipm_get_iterate.argtypes = [vp, i, ctypes.POINTER(IterateC)]
    lib.bipm_set_iterate.argtypes = [vp, i, ctypes.POINTER(IterateC)]
    lib.bipm_get_phase_cycles.argtypes = [vp, vp, i, i]
    lib.bipm_solve_queue.argtypes = [vp, vp, i, vp, vp, i]
    lib.bipm_solve_static.argtypes = [ctypes.POINTER(ProblemDescC), ctypes.POINTER(OptionsC), vp, i,
                                      vp, vp, vp]
    lib.bipm_solve_queue_warm.argtypes = [vp, vp, vp, i, vp, vp, i]
    lib.bipm_solve_mixed.argtypes = [ctypes.POINTER(ProblemDescC), i, ctypes.POINTER(OptionsC), i, vp, vp, i,
                                     vp, vp, i, vp]
    pd = ctypes.POINTER(ProblemDescC)
    lib.bipm_warm_features.argtypes = [pd, vp, i, i, vp, vp]
    lib.bipm_warm_encode.argtypes = [pd, vp, vp, i, vp, vp]
    lib.bipm_warm_decode.argtypes = [pd, vp, vp, i, vp, vp]
    lib.bipm_mlp_create.argtypes = [vp, i, i, vp, ctypes.POINTER(vp)]
    lib.bipm_mlp_param_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    lib.bipm_mlp_set_params.argtypes = [vp, vp, i]
    lib.bipm_mlp_get_params.argtypes = [vp, vp, i]
    lib.bipm_mlp_forward.argtypes = [vp, vp, i, vp, i]
    lib.bipm_mlp_loss_grad.argtypes = [vp, vp, vp, i, vp, vp, i]
    lib.bipm_mlp_train_step.argtypes = [vp, vp, vp, i, vp, i, ctypes.c_float, vp]
    lib.bipm_mlp_destroy.argtypes = [vp]
    lib.bipm_mlp_destroy.restype = None
    lib.bipm_check_rsqrt.argtypes = [i, ctypes.POINTER(ctypes.c_double)]
    lib.bipm_last_error.restype = ctypes.c_char_p
    lib.bipm_destroy.argtypes = [vp]
    lib.bipm_destroy.restype = None
    for name in EXPORTS:
        if name not in ("bipm_last_error", "bipm_destroy", "bipm_mlp_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


class BipmError(RuntimeError):
    """A failed library call; `code` is the C return value (EINVAL, ETIMEOUT, ...)."""

    def __init__(self, msg, code=0):
        super().__init__(msg)
        self.code = code


def check_rsqrt(n: int) -> float:
    """Largest ulp distance of the factorisation's FP64 reciprocal square root
    from CUDA's 1.0 / sqrt(x) over n log-spaced x (bipm_check_rsqrt)."""
    out = ctypes.c_double()
    _check(load_library().bipm_check_rsqrt(int(n), ctypes.byref(out)))
    return out.value


def solve_static(desc, theta_dev, x_out=None, results=None, options: "Options | None" = None,
                 stream=None):
    """bipm_solve_static: solve the rows of theta_dev (CUDA float64 tensor) with the
    library's fixed static workspace (no device allocation by the library).

    x_out: optional CUDA float64 tensor (count x n); results: CUDA uint8 tensor of
    count * RESULT_DTYPE.itemsize bytes (read back with results_from_bytes)."""
    lib = load_library()
    d = desc_c(desc)
    o = options or Options()
    oc = o.to_c()
    sp = _stream_ptr(stream)
    pt, dev = _ptr(theta_dev)
    px, _ = _ptr(x_out)
    if not dev or results is None:
        raise ValueError("solve_static takes CUDA tensors (theta, results)")
    _check(lib.bipm_solve_static(ctypes.byref(d), ctypes.byref(oc), pt, theta_dev.shape[0], px,
                                 ctypes.c_void_p(results.data_ptr()), sp))


def _check(rc):
    if rc != 0:
        msg = load_library(False).bipm_last_error().decode()
        raise BipmError(f"bipm error {rc}: {msg}", rc)


def _ptr(arr):
    """(pointer, on_device) of a contiguous float64 numpy array or torch tensor."""
    if arr is None:
        return None, 0
    if hasattr(arr, "data_ptr"):  # torch tensor
        import torch
        if arr.dtype != torch.float64 or not arr.is_contiguous():
            raise ValueError("tensor must be contiguous float64")
        return ctypes.c_void_p(arr.data_ptr()), int(arr.is_cuda)
    if arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous float64")
    return arr.ctypes.data_as(ctypes.c_void_p), 0


@dataclasses.dataclass
class Options:
    tol: float = 1e-6
    max_iter: int = 500
    mu_init: float = 0.1
    precision: int = 0  # 0 FP64, 1 FP32 factorisation + FP64 refinement, 2 double-float factorisation
    schedule: int = 0   # 0 warp then block teams, 1 warp teams only, 2 block teams only
    fp32_switch: float = 0.0  # barrier scale above which precision 1 factorises in FP64
    warm_mu_init: float = 0.0     # mu_0 of a warm start (0: library default 1e-2)
    warm_bound_push: float = 0.0  # bound push of a warm start (0: library default 1e-3)
    warm_max_iter: int = 0        # iteration budget of a warm start (0: library default 60)
    time_limit_ms: int = 0        # device time budget of one call (0: none; BIPM_ETIMEOUT when spent)
    visit_cap: int = 0            # queue iterations before a straggler is parked (0: 96)
    warps_per_sm: int = 0         # resident warps per SM, 4..24 in steps of 4 (0: 24)
    team_threads: int = 0         # block-team threads, 128 or 256 (0: 256)
    watchdog: int = 0             # Table I row 3 on the original problem (0 off, 1 on)
    soft_resto: int = 0           # Table I row 5 on the original problem (0 off, 1 on)
    mu_strategy: int = 0          # Table I row 7: 0 monotone, 1 adaptive (free mode, monotone fallback)

    def to_c(self):
        return OptionsC(self.tol, self.max_iter, self.mu_init, self.precision, self.schedule,
                        self.fp32_switch, self.warm_mu_init, self.warm_bound_push, self.warm_max_iter,
                        self.time_limit_ms, self.visit_cap, self.warps_per_sm, self.team_threads,
                        self.watchdog, self.soft_resto, self.mu_strategy)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Batch:
    """A batch of `capacity` quadrotor NMPC problems sharing one structure."""

    def __init__(self, desc, capacity: int, options: Options | None = None, stream=None):
        self.lib = load_library()
        d = desc_c(desc)
        o = options or Options()
        oc = o.to_c()
        h = ctypes.c_void_p()
        sp = _stream_ptr(stream)
        _check(self.lib.bipm_create_batch(ctypes.byref(d), capacity, ctypes.byref(oc), sp,
                                          ctypes.byref(h)))
        self.h = h
        self.capacity = capacity
        self.desc = desc
        self.options = o
        n, m, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.bipm_dims(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nt)))
        self.n, self.m, self.n_theta = n.value, m.value, nt.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.bipm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------- inputs
    def set_problems(self, theta, first_slot: int = 0):
        count = theta.shape[0]
        p, dev = _ptr(theta)
        _check(self.lib.bipm_set_problems(self.h, p, first_slot, count, dev))

    def set_initial_guess(self, x, y=None, first_slot: int = 0):
        px, dev = _ptr(x)
        py, _ = _ptr(y)
        _check(self.lib.bipm_set_initial_guess(self.h, px, py, first_slot, x.shape[0], dev))

    # ---------------------------------------------------------- iterations
    def solve(self):
        _check(self.lib.bipm_solve(self.h))

    def solve_queue(self, theta_queue, x_out=None, results=None, x_guess=None):
        """Iteration-level batching over a queue of problems (rows of theta_queue).

        theta_queue / x_out / x_guess are numpy arrays (host) or CUDA tensors
        (device); with x_guess (n_queue x n) every problem is warm-started from
        its row (bipm_solve_queue_warm).  `results` (device mode) is a CUDA uint8
        tensor of n_queue * RESULT_DTYPE.itemsize bytes; read it back with
        results_from_bytes.  Returns a dict of numpy arrays in host mode.
        """
        nq = theta_queue.shape[0]
        pt, dev = _ptr(theta_queue)
        px, _ = _ptr(x_out)
        pg, _ = _ptr(x_guess)

        def call(res_ptr, on_dev):
            if x_guess is None:
                return self.lib.bipm_solve_queue(self.h, pt, nq, px, res_ptr, on_dev)
            return self.lib.bipm_solve_queue_warm(self.h, pt, pg, nq, px, res_ptr, on_dev)

        if dev:
            if results is None:
                raise ValueError("device mode needs a results buffer")
            _check(call(ctypes.c_void_p(results.data_ptr()), 1))
            return None
        arr = (ResultC * max(nq, 1))()
        rc = call(arr, 0)
        out = {f: np.array([getattr(arr[j], f) for j in range(nq)]) for f, _ in ResultC._fields_}
        try:
            _check(rc)
        except BipmError as e:
            if rc == ETIMEOUT:  # the records are valid: unfinished problems say RUNNING / EMPTY
                e.results = out
            raise
        return out

    def step(self, n_iterations: int = 1):
        _check(self.lib.bipm_step(self.h, n_iterations))

    # -------------------------------------------------------------- outputs
    def get_solution(self, first_slot: int = 0, count: int | None = None, out=None):
        """Returns (x, y, zl, zu) as numpy arrays (or fills the torch tensors in `out`)."""
        count = self.capacity - first_slot if count is None else count
        if out is None:
            x = np.empty((count, self.n))
            y = np.empty((count, self.m))
            zl = np.empty((count, self.n))
            zu = np.empty((count, self.n))
        else:
            x, y, zl, zu = out
        ptrs = [_ptr(a) for a in (x, y, zl, zu)]
        dev = max(pd for (_, pd) in ptrs)
        _check(self.lib.bipm_get_solution(self.h, *[p for (p, _) in ptrs], first_slot, count, dev))
        return x, y, zl, zu

    def get_stats(self, first_slot: int = 0, count: int | None = None):
        count = self.capacity - first_slot if count is None else count
        arr = (StatsC * max(count, 1))()
        _check(self.lib.bipm_get_stats(self.h, arr, first_slot, count))
        fields = [f for f, _ in StatsC._fields_]
        return {f: np.array([getattr(arr[i], f) for i in range(count)]) for f in fields}

    def get_phase_cycles(self, first_slot: int = 0, count: int | None = None):
        """Per-slot SM cycles per phase (columns: PHASES)."""
        count = self.capacity - first_slot if count is None else count
        out = np.zeros((max(count, 1), 8), dtype=np.int64)
        _check(self.lib.bipm_get_phase_cycles(self.h, out.ctypes.data_as(ctypes.c_void_p),
                                              first_slot, count))
        return out[:count]

    def get_iterate(self, slot: int) -> dict:
        n, m = self.n, self.m
        bufs = {k: np.zeros(n) for k in ("x", "zl", "zu", "x_ref", "wd_x", "wd_zl", "wd_zu", "wd_dx")}
        bufs.update({k: np.zeros(m) for k in ("y", "p", "nn", "zp", "zn", "wd_y", "wd_dy")})
        bufs["filter"] = np.zeros(2 * FILTER_CAP)
        bufs["filter_r"] = np.zeros(2 * FILTER_CAP)
        it = IterateC()
        for k, v in bufs.items():
            setattr(it, k, v.ctypes.data_as(_DP))
        _check(self.lib.bipm_get_iterate(self.h, slot, ctypes.byref(it)))
        out = dict(bufs)
        for f, _ in IterateC._fields_:
            if f not in bufs:
                out[f] = getattr(it, f)
        out["mu_refs"] = list(out["mu_refs"])[: out["n_refs"]]
        out["filter"] = out["filter"][: 2 * out["n_filter"]].reshape(-1, 2)
        out["filter_r"] = out["filter_r"][: 2 * out["n_filter_r"]].reshape(-1, 2)
        return out

    def set_iterate(self, slot: int, state: dict):
        it = IterateC()
        keep = []
        n, m = self.n, self.m
        sizes = {"x": n, "zl": n, "zu": n, "x_ref": n, "y": m, "p": m, "nn": m, "zp": m, "zn": m,
                 "wd_x": n, "wd_zl": n, "wd_zu": n, "wd_dx": n, "wd_y": m, "wd_dy": m}
        for k, ln in sizes.items():
            v = state.get(k)
            if v is None:
                v = np.zeros(ln)
            v = np.ascontiguousarray(v, dtype=np.float64)
            if v.shape != (ln,):
                raise ValueError(f"{k} must have length {ln}")
            keep.append(v)
            setattr(it, k, v.ctypes.data_as(_DP))
        for k, nk in (("filter", "n_filter"), ("filter_r", "n_filter_r")):
            f = np.zeros(2 * FILTER_CAP)
            src = np.asarray(state.get(k, np.zeros((0, 2))), dtype=np.float64).reshape(-1)
            f[: src.size] = src
            keep.append(f)
            setattr(it, k, f.ctypes.data_as(_DP))
            setattr(it, nk, int(src.size // 2))
        for f, _ in IterateC._fields_:
            if f in sizes or f in ("filter", "filter_r", "n_filter", "n_filter_r", "mu_refs", "n_refs"):
                continue
            setattr(it, f, state.get(f, 0))
        refs = list(state.get("mu_refs", []))
        it.n_refs = len(refs)
        it.mu_refs = (ctypes.c_double * 4)(*(refs + [0.0] * (4 - len(refs))))
        if "mu_free" not in state:
            it.mu_free = 1
        _check(self.lib.bipm_set_iterate(self.h, slot, ctypes.byref(it)))


# ------------------------------------------------------------------ warm start
def _desc_c(desc):
    return desc_c(desc)


def _dev_ptr(t, dtype_name):
    import torch
    if not (hasattr(t, "data_ptr") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if t.dtype != getattr(torch, dtype_name):
        raise ValueError(f"expected a {dtype_name} tensor")
    return ctypes.c_void_p(t.data_ptr())


def warm_features(desc, theta_dev, k_near, out, stream=None):
    """bipm_warm_features: out (count x (12 + 3 k_near), float32 CUDA tensor)."""
    lib = load_library()
    _check(lib.bipm_warm_features(ctypes.byref(_desc_c(desc)), _dev_ptr(theta_dev, "float64"),
                                  theta_dev.shape[0], k_near, _dev_ptr(out, "float32"), _stream_ptr(stream)))
    return out


def warm_encode(desc, theta_dev, x_dev, out, stream=None):
    """bipm_warm_encode: out (count x (12 (N+1) + 4 N), float32 CUDA tensor)."""
    lib = load_library()
    _check(lib.bipm_warm_encode(ctypes.byref(_desc_c(desc)), _dev_ptr(theta_dev, "float64"),
                                _dev_ptr(x_dev, "float64"), theta_dev.shape[0], _dev_ptr(out, "float32"),
                                _stream_ptr(stream)))
    return out


def warm_decode(desc, theta_dev, net_out, x_guess, stream=None):
    """bipm_warm_decode: x_guess (count x n, float64 CUDA tensor)."""
    lib = load_library()
    _check(lib.bipm_warm_decode(ctypes.byref(_desc_c(desc)), _dev_ptr(theta_dev, "float64"),
                                _dev_ptr(net_out, "float32"), theta_dev.shape[0], _dev_ptr(x_guess, "float64"),
                                _stream_ptr(stream)))
    return x_guess


def _fptr(arr):
    """(pointer, on_device) of a contiguous float32 numpy array or torch tensor."""
    if arr is None:
        return None, 0
    if hasattr(arr, "data_ptr"):
        import torch
        if arr.dtype != torch.float32 or not arr.is_contiguous():
            raise ValueError("tensor must be contiguous float32")
        return ctypes.c_void_p(arr.data_ptr()), int(arr.is_cuda)
    if arr.dtype != np.float32 or not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous float32")
    return arr.ctypes.data_as(ctypes.c_void_p), 0


class MLP:
    """The warm-start network (bipm_mlp_*): widths = (input, hidden..., output)."""

    def __init__(self, widths, max_rows: int, stream=None):
        self.lib = load_library()
        self.widths = tuple(int(w) for w in widths)
        arr = (ctypes.c_int * len(self.widths))(*self.widths)
        h = ctypes.c_void_p()
        _check(self.lib.bipm_mlp_create(arr, len(self.widths), max_rows, _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.max_rows = max_rows
        cnt = ctypes.c_longlong()
        _check(self.lib.bipm_mlp_param_count(h, ctypes.byref(cnt)))
        self.n_params = cnt.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.bipm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, flat):
        p, dev = _fptr(flat)
        if flat.shape[0] != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check(self.lib.bipm_mlp_set_params(self.h, p, dev))

    def get_params(self, out=None):
        out = np.empty(self.n_params, dtype=np.float32) if out is None else out
        p, dev = _fptr(out)
        _check(self.lib.bipm_mlp_get_params(self.h, p, dev))
        return out

    def forward(self, x, out=None):
        rows = x.shape[0]
        if out is None:
            out = np.empty((rows, self.widths[-1]), dtype=np.float32)
        px, dev = _fptr(x)
        po, _ = _fptr(out)
        _check(self.lib.bipm_mlp_forward(self.h, px, rows, po, dev))
        return out

    def loss_grad(self, x, t):
        """(loss, flat gradient) of one batch (host arrays)."""
        rows = x.shape[0]
        grad = np.empty(self.n_params, dtype=np.float32)
        loss = np.zeros(1)
        px, dev = _fptr(x)
        pt, _ = _fptr(t)
        if dev:
            raise ValueError("loss_grad takes host arrays")
        _check(self.lib.bipm_mlp_loss_grad(self.h, px, pt, rows, grad.ctypes.data_as(ctypes.c_void_p),
                                           loss.ctypes.data_as(ctypes.c_void_p), 0))
        return float(loss[0]), grad

    def train_step(self, x_dev, t_dev, idx_dev, rows: int, lr: float, want_loss=False):
        """One Adam step on rows idx_dev[:rows] of the CUDA tensors x_dev, t_dev."""
        import torch
        if idx_dev is not None and idx_dev.dtype != torch.int32:
            raise ValueError("idx must be int32")
        loss = np.zeros(1)
        pl = loss.ctypes.data_as(ctypes.c_void_p) if want_loss else None
        pi = ctypes.c_void_p(idx_dev.data_ptr()) if idx_dev is not None else None
        if t_dev.shape[0] != x_dev.shape[0]:
            raise ValueError("x and t must have the same number of rows")
        _check(self.lib.bipm_mlp_train_step(self.h, _dev_ptr(x_dev, "float32"), _dev_ptr(t_dev, "float32"),
                                            int(x_dev.shape[0]), pi, rows, ctypes.c_float(lr), pl))
        return float(loss[0]) if want_loss else None


def solve_mixed(classes, cls, theta, n_slots: int, options: "Options | None" = None, x_out=None,
                results=None, stream=None):
    """bipm_solve_mixed: problems of different structure classes in one queue.

    classes: list of ProblemDesc; cls: int array (class of each problem);
    theta: packed parameter rows (numpy float64, or a CUDA float64 tensor);
    x_out: packed solution rows or None.  Host mode returns the result records
    as a dict of arrays; device mode fills `results` (CUDA uint8 tensor)."""
    lib = load_library()
    arr = (ProblemDescC * len(classes))(*[desc_c(c) for c in classes])
    oc = (options or Options()).to_c()
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    nq = int(cls.shape[0])
    pt, dev = _ptr(theta)
    px, _ = _ptr(x_out)
    pc = cls.ctypes.data_as(ctypes.c_void_p)
    if dev:
        if results is None:
            raise ValueError("device mode needs a results buffer")
        _check(lib.bipm_solve_mixed(arr, len(classes), ctypes.byref(oc), n_slots, pc, pt, nq, px,
                                    ctypes.c_void_p(results.data_ptr()), 1, _stream_ptr(stream)))
        return None
    res = (ResultC * max(nq, 1))()
    _check(lib.bipm_solve_mixed(arr, len(classes), ctypes.byref(oc), n_slots, pc, pt, nq, px, res, 0,
                                _stream_ptr(stream)))
    return {f: np.array([getattr(res[j], f) for j in range(nq)]) for f, _ in ResultC._fields_}
