"""Uneven queue (problems of different quadrotor counts and horizons in one
launch) against the homogeneous queue and the oracle (GPU tests, C ABI).

A mixed queue runs the same iteration per problem as a queue of its class
alone, so with no stragglers handed to block teams the two must agree bit for
bit; with hand-off the outcomes agree and converged points pass the KKT test.
A few small problems are checked against the oracle one by one.
"""

import numpy as np
import pytest

from oracle import ipm
from oracle_bridge import e_v, oracle_solve_batch
from workloads import make_mixed, n_theta

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bipm():
    import torch

    assert torch.cuda.is_available()
    from paper_2606_26341_gb300 import bipm as b

    b.load_library()
    return b


def _offsets(classes, cls, attr):
    sizes = [n_theta(classes[k]) if attr == "theta" else classes[k].n for k in cls]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _per_class(bipm, classes, cls, theta, options, capacity):
    """Each class's problems through a homogeneous queue of that class."""
    th_off = _offsets(classes, cls, "theta")
    x_off = _offsets(classes, cls, "x")
    x = np.zeros(x_off[-1])
    out = {}
    for k in np.unique(cls):
        ids = np.nonzero(cls == k)[0]
        rows = np.stack([theta[th_off[j]:th_off[j + 1]] for j in ids])
        xk = np.empty((len(ids), classes[k].n))
        with bipm.Batch(classes[k], min(capacity, len(ids)), options) as b:
            r = b.solve_queue(np.ascontiguousarray(rows), xk)
        for t, j in enumerate(ids):
            x[x_off[j]:x_off[j + 1]] = xk[t]
            out[j] = {f: r[f][t] for f in r}
    res = {f: np.array([out[j][f] for j in range(len(cls))]) for f in out[0]}
    return res, x


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_queue_equals_per_class_queues(bipm, precision):
    classes, cls, theta = make_mixed(160, max_quads=3, horizons=(6, 10))
    opts = bipm.Options(precision=precision, fp32_switch=-1.0 if precision else 0.0)
    x_off = _offsets(classes, cls, "x")
    x = np.zeros(x_off[-1])
    r = bipm.solve_mixed(classes, cls, theta, n_slots=48, options=opts, x_out=x)
    ref, xr = _per_class(bipm, classes, cls, theta, opts, capacity=48)
    np.testing.assert_array_equal(r["status"], ref["status"])
    np.testing.assert_array_equal(r["iters"], ref["iters"])
    for j in range(len(cls)):
        assert e_v(x[x_off[j]:x_off[j + 1]], xr[x_off[j]:x_off[j + 1]]) <= 1e-12, j
    conv = r["status"] == bipm.CONVERGED
    assert conv.mean() >= 0.6
    assert np.all(r["kkt_err"][conv] <= 1e-6)


def test_mixed_queue_hands_stragglers_to_block_teams(bipm):
    """More slots than resident warps: problems past the warp visit are parked
    and finished by block teams; outcomes match the per-class queues."""
    classes, cls, theta = make_mixed(3000, max_quads=3, horizons=(8,), first_id=5000)
    opts = bipm.Options(precision=1, fp32_switch=-1.0)
    r = bipm.solve_mixed(classes, cls, theta, n_slots=3000, options=opts)
    assert np.all(r["status"] != bipm.RUNNING) and np.all(r["status"] != bipm.EMPTY)
    assert np.sum(r["iters"] > 96) >= 20
    ref, _ = _per_class(bipm, classes, cls, theta, opts, capacity=3000)
    assert np.mean(r["status"] == ref["status"]) >= 0.97
    conv = r["status"] == bipm.CONVERGED
    assert np.all(r["kkt_err"][conv] <= 1e-6)


def test_mixed_queue_against_oracle(bipm):
    classes, cls, theta = make_mixed(24, max_quads=2, horizons=(6,), first_id=900)
    th_off = _offsets(classes, cls, "theta")
    x_off = _offsets(classes, cls, "x")
    x = np.zeros(x_off[-1])
    r = bipm.solve_mixed(classes, cls, theta, n_slots=24, options=bipm.Options(precision=0), x_out=x)
    for k in np.unique(cls):
        ids = np.nonzero(cls == k)[0][:3]
        rows = np.stack([theta[th_off[j]:th_off[j + 1]] for j in ids])
        res = oracle_solve_batch(classes[k], rows)
        for o, j in zip(res, ids):
            if o["status"] == ipm.CONVERGED:
                assert r["status"][j] == bipm.CONVERGED, (j, r["status"][j])
                if r["iters"][j] == o["iter"]:
                    assert e_v(x[x_off[j]:x_off[j + 1]], o["x"]) <= 1e-6
                else:
                    assert r["kkt_err"][j] <= 1e-6


def test_mixed_queue_rejects_bad_classes(bipm):
    classes, cls, theta = make_mixed(4, max_quads=2, horizons=(6,))
    bad = cls.copy()
    bad[2] = len(classes)
    with pytest.raises(bipm.BipmError, match="is not a class"):
        bipm.solve_mixed(classes, bad, theta, n_slots=4)
    with pytest.raises(bipm.BipmError, match="precision 0 and 1"):
        bipm.solve_mixed(classes, cls, theta, n_slots=4, options=bipm.Options(precision=2))
