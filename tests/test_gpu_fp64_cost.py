"""The GB300 cost model the kernels are designed against (GPU test).

A probe kernel (tests/probes/fp64_issue_cost.cu) measures how many SM cycles
one warp instruction occupies: FP64 FMA, min/max, FP64<->FP32 conversion,
division and square root, each with 32, 12, 4 and 1 active lanes, and FP32 FMA.
The design relies on two facts it checks: an FP64 warp instruction costs the
same whatever the number of active lanes (so FP64 work is counted in warp
instructions, not lane operations), and it costs tens of FP32 FMAs.
"""

import os
import re
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_cost_is_per_warp_instruction(tmp_path):
    exe = str(tmp_path / "fp64_issue_cost")
    src = os.path.join(HERE, "probes", "fp64_issue_cost.cu")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    print(out)
    cost = {}
    for line in out.splitlines():
        m = re.match(r"(.+?)\s+active\s+(\d+):\s+[\d.]+ ms, ([\d.]+) SM-cycles", line)
        if m:
            cost[(m.group(1).strip(), int(m.group(2)))] = float(m.group(3))
    assert "status: no error" in out
    for kind in ("dfma x2", "dmin/dmax", "f64<->f32 cvt", "ddiv", "dsqrt"):
        assert cost[(kind, 1)] >= 0.8 * cost[(kind, 32)], kind
    assert cost[("dfma x2", 32)] >= 20 * cost[("ffma", 32)]
