"""Writes multi4_n<N>_oracle.json: the CPU oracle's outcome for the first
problems of the four-quadrotor workload (pairwise distance 0.4) at horizon N,
for the GPU outcome tests.  Calls only the oracle.

    python tests/golden/make_multi4.py 12 8     # N = 12, problems 0-7 (~10 min, 8 cores)
    python tests/golden/make_multi4.py 25 8     # N = 25, configuration 3's horizon
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ[_v] = "1"


def main():
    from oracle_bridge import oracle_solve_batch
    from workloads import ProblemDesc, make_batch

    horizon = int(sys.argv[1]) if len(sys.argv) > 1 else 12
    count = int(sys.argv[2]) if len(sys.argv) > 2 else 8
    desc = ProblemDesc(nq=4, horizon=horizon, dt=0.05, pair_dist=0.4)
    _, theta = make_batch("multi4", count, desc=desc)
    res = oracle_solve_batch(desc, theta, processes=min(count, os.cpu_count() or 1))
    out = {
        "workload": f"multi4 problems 0-{count - 1} at horizon {horizon} (4 quadrotors, pairwise distance 0.4)",
        "source": "oracle.ipm.solve from the default start, written by tests/golden/make_multi4.py",
        "status": [int(r["status"]) for r in res],
        "iters": [int(r["iter"]) for r in res],
        "resto_iters": [int(r["resto"]) for r in res],
        "obj": [float(r["metrics"]["obj"]) if r["metrics"] else None for r in res],
        "x": [[float(v) for v in r["x"]] for r in res],
    }
    with open(os.path.join(HERE, f"multi4_n{horizon}_oracle.json"), "w") as fh:
        json.dump(out, fh)
    print(out["status"], out["iters"])


if __name__ == "__main__":
    main()
