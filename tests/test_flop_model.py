"""The roofline's per-unit operation counts equal the counts of the device
templates instantiated on the host with a counting scalar (no GPU needed)."""

import os
import subprocess
import tempfile

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_26341_gb300", "csrc")


def test_model_operation_counts_match_device_templates():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "opcount")
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "opcount.cpp"),
                        "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    counts = {}
    for line in out.strip().splitlines():
        name, add, mul, div, sc = line.split()
        counts[name] = (int(add), int(mul), int(div), int(sc))
    # divisions by the constant step-size fractions (dt/6, dt/3, dt/2) are
    # folded at compile time on the device; the remaining divisions are the
    # 1/cos(theta) of each model evaluation (one per f evaluation, two per dual one)
    add, mul, div, _ = counts["rk4_value"]
    assert bench.RK4_VALUE_FLOPS == add + mul + 4
    add, mul, div, _ = counts["rk4_adjoint"]
    assert bench.RK4_ADJOINT_FLOPS == add + mul + 4
    add, mul, div, _ = counts["rk4_dual_adjoint"]
    assert bench.RK4_DUAL_FLOPS == add + mul + 8


def test_unit_flops_are_positive_and_scale_with_the_horizon():
    from workloads import ProblemDesc

    a = bench.unit_flops(ProblemDesc(nq=1, horizon=10, n_sph=1))
    b = bench.unit_flops(ProblemDesc(nq=1, horizon=20, n_sph=1))
    for k in a:
        assert a[k] > 0
        assert 1.8 < b[k] / a[k] < 2.2


def test_lower_triangle_index_arithmetic_covers_every_entry_once():
    """The factorisation's lower-triangle index helpers (csrc/tri_index.cuh, the
    same source the kernels compile), built for the host and checked exhaustively
    for 1..8 quadrotors."""
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tri_index_check")
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "tri_index_check.cpp"),
                        "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
