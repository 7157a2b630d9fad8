"""Writes track_quat_oracle.json: the CPU oracle's outcome for the first
problems of the tracking workload on the 13-state quaternion model (dt = 0.1,
N = 30, three spheres), the paper's own model and step.  Calls only the oracle.

    python tests/golden/make_track_quat.py 8     # problems 0-7 (about a minute on 8 cores)
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
    from workloads import make_batch

    count = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    desc, theta = make_batch("track_quat", count)
    res = oracle_solve_batch(desc, theta, processes=min(count, os.cpu_count() or 1))
    out = {
        "workload": f"track_quat problems 0-{count - 1} (13-state quaternion model, dt 0.1, N 30, 3 spheres)",
        "source": "oracle.ipm.solve from the default start, written by tests/golden/make_track_quat.py",
        "status": [int(r["status"]) for r in res],
        "iters": [int(r["iter"]) for r in res],
        "resto_iters": [int(r["resto"]) for r in res],
        "obj": [float(r["metrics"]["obj"]) if r["metrics"] else None for r in res],
        "kkt": [float(r["metrics"]["kkt"]) if r["metrics"] else None for r in res],
        "x": [[float(v) for v in r["x"]] for r in res],
    }
    with open(os.path.join(HERE, "track_quat_oracle.json"), "w") as fh:
        json.dump(out, fh)
    print(out["status"], out["iters"])


if __name__ == "__main__":
    main()
