"""Writes multi4_n12_oracle.json: the CPU oracle's outcome for the first eight
problems of the four-quadrotor workload at horizon N = 12 (pairwise distance
0.4), for the GPU outcome test.  Calls only the oracle; about ten minutes on
eight host cores.

    python tests/golden/make_multi4_n12.py
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

    desc = ProblemDesc(nq=4, horizon=12, dt=0.05, pair_dist=0.4)
    _, theta = make_batch("multi4", 8, desc=desc)
    res = oracle_solve_batch(desc, theta, processes=8)
    out = {
        "workload": "multi4 problems 0-7 at horizon 12 (4 quadrotors, pairwise distance 0.4)",
        "source": "oracle.ipm.solve from the default start, written by tests/golden/make_multi4_n12.py",
        "status": [int(r["status"]) for r in res],
        "iters": [int(r["iter"]) for r in res],
        "obj": [float(r["metrics"]["obj"]) if r["metrics"] else None for r in res],
        "x": [[float(v) for v in r["x"]] for r in res],
    }
    with open(os.path.join(HERE, "multi4_n12_oracle.json"), "w") as fh:
        json.dump(out, fh)
    print(out["status"], out["iters"])


if __name__ == "__main__":
    main()
