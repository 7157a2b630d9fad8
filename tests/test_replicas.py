"""Replicas (weak scaling, no collective on the data path): bench.py's
multi-rank host logic with world size 2 over gloo on CPU.  Each rank draws a
disjoint range of problems; time is the maximum over ranks, converged
problems the sum."""

import json
import os
import socket

import torch.multiprocessing as mp

import replica_worker


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_draw_disjoint_problems_and_reduce(tmp_path):
    mp.spawn(replica_worker.run, args=(_free_port(), str(tmp_path)), nprocs=2, join=True)
    r0 = json.load(open(os.path.join(tmp_path, "rank0.json")))
    r1 = json.load(open(os.path.join(tmp_path, "rank1.json")))
    assert r0["ws"] == r1["ws"] == 2
    # rank 1 starts after rank 0's timed and warm-up problems (8 x 3 + 8 + 8)
    assert r1["first"] - r0["first"] >= 8 * 3 + 8
    assert r0["theta0"] != r1["theta0"]
    assert r0["t"] == r1["t"] == 2.5
    assert r0["conv"] == r1["conv"] == 201
