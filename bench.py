"""Benchmark: converged NLP solves/sec at KKT tolerance 1e-6 on one GB300.

Workload (default): reference tracking with three random spherical obstacles,
one quadrotor, RK4 horizon N = 30, 4096 problems per step ("track").  The K
steps' problems stream through the slots of one persistent queue launch
(iteration-level batching).  The headline `value` is the chosen form: the
autotuner's fastest precision form and schedule (its options are in
`config.options`, its arithmetic in `dtype`); the plain FP64 form is reported
beside it (`fp64`).  Each form's timed region is repeated (five times for the
chosen form, three for FP64) and the median
reported.  Further legs: the learned warm start (cluttered environment), four
quadrotors at N = 25 (`multi4`), the uneven queue against solve-level
batching (`uneven_queue`), and the CPU oracle on the host cores with each GPU
form's error against it (`cpu_baseline`).

python bench.py --gpus N --steps K --warmup W [--impl reference]
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workloads import make_batch  # noqa: E402

WORKLOAD = "track"
BATCH = 4096
METRIC = "converged NLP solves/sec at KKT tol 1e-6 on 1 GB300 (plain FP64 vs chosen form)"
UNIT = "solves/s"
FP64_PEAK_NOMINAL = 152 * 2 * 2 * 2.07e9  # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.07e9


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_first_id(rank, batch, steps, warmup):
    """First problem id of a rank's share (weak scaling): the timed problems
    (steps x batch), then its warm-up problems; ranks draw disjoint ranges."""
    return rank * batch * (steps + warmup + 1)


def reduce_scalar(v, op, world_size, device):
    """v combined over the ranks ("max" or "sum"); v itself for one rank."""
    if world_size == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return None


# ------------------------------------------------------------- flop model
# Operation counts of the model routines, from the host instantiation of the
# device templates with a counting scalar (tests/opcount.cpp;
# tests/test_flop_model.py recompiles it and checks these numbers).
RK4_VALUE_FLOPS = 152 + 200 + 4            # one RK4 step of one quadrotor, value only
RK4_ADJOINT_FLOPS = 403 + 620 + 4          # value + reverse sweep (gradient of lam^T F)
RK4_DUAL_FLOPS = 1122 + 1596 + 8           # forward-over-reverse, one direction

# DRAM traffic per problem-iteration of the queue kernel, measured by ncu on one
# timed launch of 4096 tracking problems (dram__bytes_read.sum +
# dram__bytes_write.sum = 41.35e9 + 33.20e9 B at 30.45 iterations each); scaled
# to a launch by its iterations.
TRAFFIC_PER_PROBLEM_ITER = (41.35e9 + 33.20e9) / (4096 * 30.45)


def unit_flops(desc):
    """Algorithmic FLOPs of the units the kernel counts, for one problem."""
    N, nq, ni = desc.horizon, desc.nq, desc.ni
    nx, nu = 12 * nq, 4 * nq
    n, m = desc.n, desc.m
    pos = 3 * nq
    # one Riccati factorisation: PA, Q^ (24 nx^2 each), PB, S^ (24 nx nu each),
    # R^ (24 nu^2), K (2 nx nu^2), P (2 nx^2 nu), Cholesky (nu^3/3), condensation
    fact_stage = 48 * nx * nx + 48 * nx * nu + 24 * nu * nu + 2 * nx * nu * nu \
        + 2 * nx * nx * nu + nu ** 3 / 3 + 4 * pos * pos * ni
    fact = N * fact_stage + 4 * pos * pos * ni
    # one solve: backward (P~d, B^T t, k, A^T t, K^T g) and forward (K dx, A dx + B du, P~ xi)
    solve_stage = 4 * nx * nx + 56 * nx + 4 * nx * nu + 24 * nu + 2 * nu * nu + 20 * ni
    solve = N * solve_stage
    # KKT mat-vec of one refinement step: dynamics blocks, Hessian, diagonal, inequality rows
    matvec = N * nq * (2 * 144 * 2 + 2 * 48 * 2 + 100 * 2) + 4 * n + N * ni * 12
    values = N * nq * RK4_VALUE_FLOPS + N * ni * 12 + 3 * n       # c(x), f(x)
    trial = values + 4 * n                                        # plus barrier objective
    derivs = N * nq * 10 * RK4_DUAL_FLOPS                         # A, B, lambda-Hessian
    jty = N * nq * RK4_ADJOINT_FLOPS + N * ni * pos * 4
    iter_fixed = values + jty + derivs + 30 * n                   # + vector updates/norms
    return {"fact": fact, "solve": solve, "matvec": matvec, "trial": trial,
            "derivs": derivs, "iter_fixed": iter_fixed, "values": values}


def step_flops(desc, stats, precision):
    """(FP64 flops, FP32 flops) of one batched solve from the per-problem counters."""
    u = unit_flops(desc)
    it = float(np.sum(stats["iters"]))
    fact = float(np.sum(stats["factorizations"]))
    solves = float(np.sum(stats["solves"]))
    trials = float(np.sum(stats["trials"]))
    ir = float(np.sum(stats["ir_steps"]))
    f32 = float(np.sum(stats["fact32"]))
    s32 = float(np.sum(stats["solve32"]))
    # derivative blocks run in the factor precision's block type (FP32 when precision = 1)
    derivs32 = it * u["derivs"] if precision == 1 else 0.0
    lowp = derivs32 + f32 * u["fact"] + s32 * u["solve"]
    # everything else is FP64: evaluation, residuals, trials, FP64 factorisations and
    # solves, and one KKT mat-vec per refinement step and per refined FP32 solve
    f64 = it * u["iter_fixed"] - derivs32 + trials * u["trial"] + (fact - f32) * u["fact"] \
        + (solves - s32) * u["solve"] + (ir + s32) * u["matvec"]
    return f64, lowp


# ------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from paper_2606_26341_gb300 import autotune, bipm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    B, K, W = args.batch, args.steps, args.warmup
    # K steps of B problems each, distinct per step and per rank (weak scaling)
    first = rank_first_id(rank, B, K, W)
    desc, theta = make_batch(WORKLOAD, B * K, first_id=first)
    _, theta_w = make_batch(WORKLOAD, B, first_id=first + B * K)
    theta_dev = torch.as_tensor(theta, device=dev)
    theta_wdev = torch.as_tensor(theta_w, device=dev)
    n, m = desc.n, desc.m
    rsize = bipm.RESULT_DTYPE.itemsize

    # chosen form: the autotuner's pick of precision form and schedule (untimed)
    if args.only_mixed:
        best, slots = bipm.Options(precision=1, fp32_switch=args.fp32_switch), B
        tune_table = []
    else:
        # the sample runs in the timed regime: a queue of twice the slot count
        _, theta_t = make_batch(WORKLOAD, 2 * B, first_id=10_000_000 + rank * 2 * B)
        pick, tune_table = autotune.autotune(desc, torch.as_tensor(theta_t, device=dev), B, stream=stream,
                                             schedule=not args.no_schedule_tune)
        best, slots = pick.options, pick.slots

    def timed_queue(options, capacity, repeats):
        """W untimed warm-up steps, then `repeats` timed regions of K steps each, every
        region one queue of the K steps' problems through `capacity` slots; the
        region with the median time is returned (time, records, clocks, all times)."""
        b = bipm.Batch(desc, capacity, options, stream=stream)
        res = torch.empty(B * K * rsize, dtype=torch.uint8, device=dev)
        for _ in range(W):
            b.solve_queue(theta_wdev, None, res[: B * rsize])
        torch.cuda.synchronize()
        runs = []
        for _ in range(repeats):
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            clocks = ClockSampler(local)
            clocks.start()
            torch.cuda.synchronize()
            e0.record(stream)
            b.solve_queue(theta_dev, None, res)
            e1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            barrier()
            runs.append((e0.elapsed_time(e1), bipm.results_from_bytes(res.cpu().numpy()), clk))
        b.close()
        order = sorted(range(repeats), key=lambda i: runs[i][0])
        ms, rec, clk = runs[order[repeats // 2]]
        return ms, rec, clk, [r[0] for r in runs]

    ms_mixed, r_mixed, clk, ms_all = timed_queue(best, slots, args.repeats)
    # the plain FP64 form with the chosen barrier update (the pair isolates the precision form)
    opt64 = bipm.Options(precision=0, mu_strategy=best.mu_strategy)
    if args.only_mixed:
        ms_fp64, r_fp64, ms_all64 = ms_mixed, r_mixed, ms_all
    else:
        ms_fp64, r_fp64, _, ms_all64 = timed_queue(opt64, B, min(args.repeats, 3))
    conv_mixed = int(np.sum(r_mixed["status"] == bipm.CONVERGED))
    conv_fp64 = int(np.sum(r_fp64["status"] == bipm.CONVERGED))

    # end to end through the public API: host parameters in, host solutions and
    # result records out, every copy inside the timed region
    theta_host = np.ascontiguousarray(theta)
    x_host = np.empty((B * K, n))
    b = bipm.Batch(desc, slots, best, stream=stream)
    b.solve_queue(np.ascontiguousarray(theta_w), None)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    r_e2e = b.solve_queue(theta_host, x_host)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    b.close()
    e2e_conv = int(np.sum(r_e2e["status"] == bipm.CONVERGED))

    def reduce(v, op):
        return reduce_scalar(v, op, ws, dev)

    MAX, SUM = "max", "sum"
    t_mixed = reduce(ms_mixed / 1e3, MAX)
    t_fp64 = reduce(ms_fp64 / 1e3, MAX)
    t_e2e_max = reduce(t_e2e, MAX)
    tot_mixed = reduce(conv_mixed, SUM)
    tot_fp64 = reduce(conv_fp64, SUM)
    tot_e2e = reduce(e2e_conv, SUM)

    # roofline of the queue kernel (the step is one launch of it)
    f64_m, f32_m = step_flops(desc, r_mixed, best.precision)
    f64_d, _ = step_flops(desc, r_fp64, 0)
    k_mixed = ms_mixed / 1e3
    k_fp64 = ms_fp64 / 1e3
    t_bound = f64_m / FP64_PEAK_NOMINAL + f32_m / FP32_PEAK_NOMINAL
    roof = {
        "bound": "alu", "unit": "TFLOP/s",
        "achieved": (f64_m + f32_m) / k_mixed / 1e12,
        "peak": (f64_m + f32_m) / t_bound / 1e12,
        "frac": t_bound / k_mixed,
        "traffic": TRAFFIC_PER_PROBLEM_ITER * float(np.sum(r_mixed["iters"])),
        "traffic_unit": "bytes per launch (ncu capture of one 4096-problem launch, scaled by iterations)",
        "kernel": "queue launch sequence of the chosen form (queue_kernel, then block teams for parked "
                  "stragglers); achieved = counted work of the sequence / its event time",
        "flops_fp64_per_launch": f64_m, "flops_fp32_per_launch": f32_m,
        "peak_source": "derived from unit counts and clocks (no FP64/FP32 ALU figure in "
                       "MEASURED_PEAKS.json): FP64 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = "
                       "1.26 TFLOP/s, FP32 152 x 128 FMA/clk x 2 x 2.07 GHz = 80.5 TFLOP/s; "
                       "mixed peak = flops / (f64/peak64 + f32/peak32)",
        "fp64_form": {"achieved": f64_d / k_fp64 / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
                      "frac": f64_d / k_fp64 / FP64_PEAK_NOMINAL},
    }

    warm = None if args.no_warm else warm_leg(args, dev, stream, rank, barrier, reduce, MAX, SUM)
    mixed = mixed_leg(args, dev, stream, barrier, reduce, MAX, SUM) if args.mixed > 0 else None
    multi = multi_leg(args, dev, stream, barrier, reduce, MAX, SUM) if args.multi > 0 else None

    if rank == 0:
        opt_desc = {"precision": best.precision, "fp32_switch": best.fp32_switch,
                    "mu_strategy": "adaptive" if best.mu_strategy else "monotone",
                    "visit_cap": best.visit_cap or 96, "warps_per_sm": best.warps_per_sm or 24,
                    "team_threads": best.team_threads or 256, "slots": slots}
        line = {
            "metric": METRIC, "value": tot_mixed / t_mixed, "unit": UNIT, "n_gpus": ws,
            "steps": K, "warmup": W, "ms_per_step": t_mixed * 1e3 / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": form_dtype(best),
            "data": "synthetic (seeded SplitMix64 tracking problems; no public dataset exists)",
            "config": {"workload": f"{WORKLOAD}: 1 quadrotor, RK4 N=30, 3 spheres, {B} problems per step",
                       "global_batch": B * ws, "parallelism": f"replicas x{ws}",
                       "mode": f"iteration-level batching: the {K} steps' problems stream through "
                               f"{slots} slots in one persistent launch",
                       "options": opt_desc,
                       "repeats": f"median of {args.repeats} timed regions of {K} steps each "
                                   f"(FP64 form: {min(args.repeats, 3)})",
                       "l2": "slot workspaces (~1.4 GB) exceed the 129 MB L2"},
            "repeats_ms": ms_all,
            "fp64": {"value": tot_fp64 / t_fp64, "unit": UNIT, "ms_per_step": t_fp64 * 1e3 / K,
                     "dtype": "f64", "repeats_ms": ms_all64},
            "autotune": tune_table,
            "converged_frac": conv_mixed / (B * K),
            "iters_mean": float(np.mean(r_mixed["iters"])),
            "iterations": iteration_summary(r_mixed),
            "e2e": {"value": tot_e2e / t_e2e_max, "unit": UNIT,
                    "h2d_bytes_per_step": B * desc_theta_len(desc) * 8,
                    "d2h_bytes_per_step": B * (n * 8 + rsize)},
            "roofline": roof,
            "clocks": clk,
            "gpu_launches": queue_launches(slots, best.warps_per_sm or 24),
        }
        if warm is not None:
            line["warm_start"] = warm
        if multi is not None:
            line["multi4"] = multi
        if mixed is not None:
            line["uneven_queue"] = mixed
        if ws == 1 and not args.no_cpu_baseline:
            forms = {"chosen": best, "fp64": opt64}
            line["cpu_baseline"] = cpu_baseline(desc, theta, forms, stream, budget_s=args.cpu_budget,
                                                mu_strategy=best.mu_strategy)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------- learned warm start leg
WARM_WORKLOAD = "cyl"


def warm_leg(args, dev, stream, rank, barrier, reduce, MAX, SUM):
    """Cluttered environment (1 quadrotor, N = 40, 20-50 cylinders, 16384 problems):
    plain FP64 cold start vs the chosen form cold and warm-started by the proposer
    network, which is first trained (untimed) on this solver's solutions of a
    disjoint set of problems.  The proposal (features, network, decoding) is
    inside the warm run's timed region; cold start is its fallback."""
    import torch

    from paper_2606_26341_gb300 import bipm, warmstart
    from workloads import mlp_init

    B = args.warm_batch
    chosen = bipm.Options(precision=1, fp32_switch=1e2)
    desc, th_train = make_batch(WARM_WORKLOAD, args.warm_train, first_id=1_000_000 + rank * args.warm_train)
    _, th_test = make_batch(WARM_WORKLOAD, B, first_id=rank * B)
    tr = torch.as_tensor(th_train, device=dev)
    te = torch.as_tensor(th_test, device=dev)
    t0 = time.perf_counter()
    data = warmstart.make_dataset(desc, tr, chosen, capacity=min(8192, args.warm_train), stream=stream)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    widths = warmstart.widths(desc)
    net = bipm.MLP(widths, max_rows=1024, stream=stream)
    net.set_params(mlp_init(widths, 5))
    t0 = time.perf_counter()
    hist = warmstart.train(net, data, epochs=args.warm_epochs, batch=512, lr=2e-3, lr_final=5e-5, seed=6)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    rsize = bipm.RESULT_DTYPE.itemsize
    res = torch.empty(B * rsize, dtype=torch.uint8, device=dev)

    def timed(options, warm_start):
        with bipm.Batch(desc, B, options, stream=stream) as b:
            g = warmstart.propose(net, desc, te[:256], stream=stream) if warm_start else None
            b.solve_queue(te[:256], None, res[: 256 * rsize], x_guess=g)  # warm-up
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g = warmstart.propose(net, desc, te, stream=stream) if warm_start else None
            b.solve_queue(te, None, res, x_guess=g)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        r = bipm.results_from_bytes(res.cpu().numpy())
        conv = int(np.sum(r["status"] == bipm.CONVERGED))
        t = reduce(e0.elapsed_time(e1) / 1e3, MAX)
        out = {"value": reduce(conv, SUM) / t, "unit": UNIT, "converged_frac": conv / B,
               "iters_mean": float(np.mean(r["iters"] + r["warm_iters"])),
               "max_kkt_err_converged": float(np.max(r["kkt_err"][r["status"] == bipm.CONVERGED]))}
        if warm_start:
            out["fallback_frac"] = float(np.mean(r["warm"] == 2))
        return out

    cold64 = timed(bipm.Options(precision=0), False)
    cold_mixed = timed(chosen, False)
    warm_mixed = timed(chosen, True)
    net.close()
    return {"workload": f"{WARM_WORKLOAD}: 1 quadrotor, RK4 N=40, 20-50 cylinders (padded to 50), "
                        f"{B} problems",
            "cold_fp64": cold64, "cold_chosen": cold_mixed, "warm_chosen": warm_mixed,
            "warm_vs_cold_fp64": warm_mixed["value"] / cold64["value"],
            "network": {"widths": list(widths), "dtype": "bf16 operands, f32 accumulation",
                        "train_problems": args.warm_train, "usable": int(len(data.usable)),
                        "epochs": args.warm_epochs, "loss_first_last": [hist[0], hist[-1]],
                        "dataset_s": t_data, "train_s": t_train}}


# ------------------------------------------------------- uneven queue leg
def mixed_leg(args, dev, stream, barrier, reduce, MAX, SUM):
    """Problems of 1-8 quadrotors and horizons 10/20/30/50 (32 structure
    classes, drawn uniformly), chosen form.  Iteration-level batching: all
    args.mixed problems in one persistent launch of the mixed queue through
    args.mixed_slots slots, a finished problem's slot refilled at once.
    Solve-level batching on the same problems: consecutive batches of
    args.mixed_slots problems, each launched with exactly its own slots, the
    next starting when the slowest of the previous batch has finished.  The
    slot count is below the resident warps, so no problem is parked in either
    arm.  Inputs are device-resident; each call sizes its workspace, so the
    rates are taken from the host clock around the calls."""
    import torch

    from paper_2606_26341_gb300 import bipm
    from workloads import make_mixed, n_theta

    ws, rank, _ = dist_env()
    Q, S = args.mixed, args.mixed_slots
    classes, cls, theta = make_mixed(Q, max_quads=args.mixed_max_quads, first_id=rank * Q)
    th = torch.as_tensor(theta, device=dev)
    rsize = bipm.RESULT_DTYPE.itemsize
    opts = bipm.Options(precision=1, fp32_switch=-1.0)
    off = np.concatenate([[0], np.cumsum([n_theta(classes[k]) for k in cls])]).astype(np.int64)

    def run(batches):
        res = torch.empty(Q * rsize, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for lo in range(0, Q, batches):
            hi = min(Q, lo + batches)
            bipm.solve_mixed(classes, cls[lo:hi], th[off[lo]:off[hi]], n_slots=min(S, hi - lo), options=opts,
                             results=res[lo * rsize:hi * rsize], stream=stream)
        torch.cuda.synchronize()
        dt = reduce(time.perf_counter() - t0, MAX)
        barrier()
        return bipm.results_from_bytes(res.cpu().numpy()), dt

    r, dt = run(Q)
    r_sl, dt_sl = run(S)
    conv = r["status"] == bipm.CONVERGED
    per_nq = {}
    for nq in range(1, args.mixed_max_quads + 1):
        sel = np.array([classes[k].nq == nq for k in cls])
        if not sel.any():
            continue
        per_nq[str(nq)] = {"problems": int(sel.sum()), "converged_frac": float(conv[sel].mean()),
                           "iters_mean": float(r["iters"][sel].mean())}
    ilb = reduce(float(conv.sum()), SUM) / dt
    slb = reduce(float(np.sum(r_sl["status"] == bipm.CONVERGED)), SUM) / dt_sl
    return {"workload": f"uneven queue: {Q} problems, 1-{args.mixed_max_quads} quadrotors (pairwise distance "
                        f"0.4; one sphere for a single quadrotor), N in 10/20/30/50, {S} slots",
            "value": ilb, "unit": UNIT, "seconds": dt,
            "solve_level_batching": {"value": slb, "unit": UNIT, "seconds": dt_sl,
                                     "batches": int(math.ceil(Q / S))},
            "ilb_gain": ilb / slb if slb > 0 else None,
            "converged_frac": float(conv.mean()), "iters_mean": float(r["iters"].mean()),
            "per_quad_count": per_nq}


# ------------------------------------------------ four-quadrotor leg
def multi_leg(args, dev, stream, barrier, reduce, MAX, SUM):
    """Configuration 3 at its size: 4 quadrotors (48 states, 16 inputs), pairwise
    separation 0.4, N = 25, args.multi problems solved as one batch through as
    many slots (every problem starts at once), FP32 factorisation with FP64
    refinement and plain FP64.  Device-timed (CUDA events on the stream)."""
    import torch

    from paper_2606_26341_gb300 import bipm
    from workloads import ProblemDesc

    ws, rank, _ = dist_env()
    desc = ProblemDesc(nq=4, horizon=25, dt=0.05, pair_dist=0.4)
    _, theta = make_batch("multi4", args.multi, desc=desc, first_id=rank * args.multi)
    th = torch.as_tensor(theta, device=dev)
    rsize = bipm.RESULT_DTYPE.itemsize
    out = {"workload": f"multi4: 4 quadrotors, RK4 N=25, pairwise distance 0.4, {args.multi} problems",
           "n": desc.n, "m": desc.m}
    for name, opt in (("fp32_refined", bipm.Options(precision=1)), ("fp64", bipm.Options(precision=0))):
        res = torch.empty(args.multi * rsize, dtype=torch.uint8, device=dev)
        with bipm.Batch(desc, args.multi, opt, stream=stream) as b:
            b.solve_queue(th[:8], None, res[:8 * rsize])  # warm-up
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.solve_queue(th, None, res)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        r = bipm.results_from_bytes(res.cpu().numpy())
        conv = r["status"] == bipm.CONVERGED
        t = reduce(e0.elapsed_time(e1) / 1e3, MAX)
        out[name] = {"value": reduce(float(conv.sum()), SUM) / t, "unit": UNIT, "seconds": t,
                     "converged_frac": float(conv.mean()),
                     "status_counts": {bipm.STATUS_NAMES[k]: int(np.sum(r["status"] == k))
                                       for k in np.unique(r["status"])},
                     "iters_mean": float(r["iters"].mean()),
                     "max_kkt_err_converged": float(np.max(r["kkt_err"][conv])) if conv.any() else None}
    return out


def iteration_summary(results, converged_status=1):
    """Iteration counts (mean, percentiles, max), histogram over fixed bins and
    the mean objective of the converged problems, from a result-record dict."""
    it = np.asarray(results["iters"])
    conv = np.asarray(results["status"]) == converged_status
    edges = [0, 10, 20, 30, 50, 100, 200, 500, 10 ** 9]
    hist, _ = np.histogram(it, bins=edges)
    return {"mean": float(it.mean()) if it.size else 0.0,
            "p50": float(np.percentile(it, 50)) if it.size else 0.0,
            "p90": float(np.percentile(it, 90)) if it.size else 0.0,
            "p99": float(np.percentile(it, 99)) if it.size else 0.0,
            "max": int(it.max()) if it.size else 0,
            "histogram": {f"{edges[i]}-{edges[i + 1] - 1}" if i < len(edges) - 2 else f">={edges[i]}": int(h)
                          for i, h in enumerate(hist)},
            "objective_mean_converged": float(np.mean(np.asarray(results["obj"])[conv])) if conv.any() else None}


def queue_launches(slots, warps_per_sm=24):
    """Kernels of one timed queue solve: the queue kernel alone when every slot
    has a resident warp; with spare slots also the slot reset, the block teams
    for parked stragglers and their write-out."""
    import torch
    resident = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * warps_per_sm
    return 4 if slots > resident else 1


def form_dtype(o):
    """The arithmetic of a precision form, for the JSON line's dtype."""
    if o.precision == 0:
        return "f64"
    if o.precision == 2:
        return "f32 derivative blocks + double-float (2 x f32) factorisation, f64 residuals and tests"
    if o.fp32_switch < 0:
        return "f32 derivative blocks + f64 factorisation, f64 residuals and tests"
    return "f32 derivative blocks + f32 factorisation with f64 refinement, f64 residuals and tests"


def stats_record_bytes():
    import ctypes

    from paper_2606_26341_gb300 import bipm
    return ctypes.sizeof(bipm.StatsC)


def desc_theta_len(desc):
    from workloads import n_theta
    return n_theta(desc)


# ------------------------------------------------------------ CPU oracle
def _oracle_one(args):
    desc, theta = args[0], args[1]
    mu_strategy = args[2] if len(args) > 2 else 0
    sys.path.insert(0, ROOT)
    import torch

    torch.set_num_threads(1)
    from oracle import ipm
    from oracle.quadrotor import QuadNLP
    t0 = time.perf_counter()
    opt = ipm.Options(mu_strategy="adaptive" if mu_strategy else "monotone")
    st, _ = ipm.solve(QuadNLP(desc, theta), opt=opt)
    return {"ok": st.status == ipm.CONVERGED, "s": time.perf_counter() - t0, "status": int(st.status),
            "iters": int(st.iter), "x": st.normal.x}


def single_thread_env():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"  # one thread per worker process: cores = processes


def oracle_rate(desc, theta, n_problems, processes, mu_strategy=0):
    """Converged count, wall time and per-problem records of the oracle on the
    first n_problems rows, one problem per process."""
    single_thread_env()
    ctx = mp.get_context("spawn")
    jobs = [(desc, theta[j], mu_strategy) for j in range(n_problems)]
    with ctx.Pool(processes=processes) as pool:
        pool.map(_oracle_one, jobs[:processes])  # warm the workers (imports)
        t0 = time.perf_counter()
        res = pool.map(_oracle_one, jobs)
        wall = time.perf_counter() - t0
    conv = sum(1 for r in res if r["ok"])
    return conv, wall, res


def _kkt_one(args):
    """The oracle's scaled optimality error E_0 at a GPU point (oracle arithmetic)."""
    desc, theta, x, y, zl, zu = args
    sys.path.insert(0, ROOT)
    import torch

    torch.set_num_threads(1)
    from oracle import ipm
    from oracle.quadrotor import QuadNLP
    nlp = QuadNLP(desc, theta)
    return ipm.opt_error(nlp, x, y, zl, zu, nlp.grad_f(x), nlp.jac_c(x), nlp.c(x), 0.0, ipm.Options())


def gpu_error_vs_oracle(desc, theta, oracle_res, options, stream, processes):
    """Each GPU form's result on the oracle's sample problems, against the oracle:
    the distance e_v of the solution (Eq. 8) where both converged, the oracle's own
    KKT error at every GPU-converged point, and the agreement of statuses and
    iteration counts."""
    from paper_2606_26341_gb300 import bipm

    cnt = len(oracle_res)
    with bipm.Batch(desc, cnt, options, stream=stream) as b:
        b.set_problems(np.ascontiguousarray(theta[:cnt]))
        b.solve()
        st = b.get_stats()
        x, y, zl, zu = b.get_solution()
    conv = st["status"] == bipm.CONVERGED
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=processes) as pool:
        kkt = pool.map(_kkt_one, [(desc, theta[j], x[j], y[j], zl[j], zu[j]) for j in np.nonzero(conv)[0]])
    ev = [float(np.max(np.abs(x[j] - o["x"]) / (1.0 + np.abs(o["x"])))) for j, o in enumerate(oracle_res)
          if o["ok"] and conv[j]]
    return {"problems": cnt,
            "e_v_x": {"max": max(ev) if ev else None, "median": float(np.median(ev)) if ev else None,
                      "per_problem": ev},
            "oracle_kkt_err_max": float(max(kkt)) if kkt else None,
            "oracle_kkt_pass": int(sum(k <= 1e-6 for k in kkt)), "gpu_converged": int(conv.sum()),
            "same_status": int(sum(st["status"][j] == o["status"] for j, o in enumerate(oracle_res))),
            "same_iters": int(sum(st["iters"][j] == o["iters"] for j, o in enumerate(oracle_res)))}


def cpu_baseline(desc, theta, forms, stream, budget_s=20.0, mu_strategy=0):
    """The oracle as it stands on the host cores, with the chosen form's barrier
    update: all cores (one problem per process, two problems per core) and one core
    (two problems); then each GPU form's error against the oracle's solutions of
    the same problems."""
    cores = os.cpu_count() or 1
    n_prob = 2 * cores
    conv, wall, res = oracle_rate(desc, theta, n_prob, cores, mu_strategy)
    conv1, wall1, _ = oracle_rate(desc, theta, 2, 1, mu_strategy)
    errors = {name: gpu_error_vs_oracle(desc, theta, res, opt, stream, cores) for name, opt in forms.items()}
    return {"value": conv / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_prob} problems of the {WORKLOAD} workload (the first of the timed set), one per "
                      f"process on {cores} cores, {wall:.1f} s wall, "
                      f"{'adaptive' if mu_strategy else 'monotone'} barrier update",
            "single_core": {"value": conv1 / wall1, "unit": UNIT, "cores": 1,
                            "sample": f"2 problems, {wall1:.1f} s"},
            "oracle_iters_mean": float(np.mean([r["iters"] for r in res])),
            "gpu_error_vs_oracle": errors}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    desc, theta = make_batch(WORKLOAD, 64)
    cores = os.cpu_count() or 1
    single_thread_env()
    ctx = mp.get_context("spawn")
    per_step = cores
    times, convs = [], []
    with ctx.Pool(processes=cores) as pool:
        for s in range(args.warmup + args.steps):
            jobs = [(desc, theta[(s * per_step + j) % theta.shape[0]]) for j in range(per_step)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_one, jobs)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
                convs.append(sum(1 for r in res if r["ok"]))
    total = sum(times)
    val = sum(convs) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": f"{WORKLOAD}: 1 quadrotor, RK4 N=30, 3 spheres",
                                        "per_step_sample": per_step},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} problems per step, one per process"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--batch", type=int, default=BATCH, help="problems per GPU (profiling runs only)")
    ap.add_argument("--only-mixed", action="store_true", help="skip the FP64 form (profiling runs only)")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--fp32-switch", type=float, default=1e2,
                    help="fp32_switch of the form --only-mixed runs (profiling runs only)")
    ap.add_argument("--warm-train", type=int, default=16384, help="training problems of the warm-start leg")
    ap.add_argument("--warm-epochs", type=int, default=30)
    ap.add_argument("--warm-batch", type=int, default=16384, help="problems of the warm-start leg")
    ap.add_argument("--mixed", type=int, default=192, help="problems of the uneven-queue leg (0: skip)")
    ap.add_argument("--mixed-slots", type=int, default=96, help="slots of the uneven-queue leg")
    ap.add_argument("--mixed-max-quads", type=int, default=4,
                    help="largest quadrotor count of the uneven-queue leg (the workload's own range is 1-8)")
    ap.add_argument("--multi", type=int, default=256, help="problems of the four-quadrotor leg (0: skip)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of the chosen form (median reported); the FP64 form takes at most 3")
    ap.add_argument("--no-schedule-tune", action="store_true", help="autotune the precision form only")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
