"""The uneven-queue workload generator (CPU): per-problem streams, class
coverage and packed parameter rows."""

import numpy as np

from workloads import make_batch, make_mixed, mixed_classes, n_theta


def test_classes_cover_quads_and_horizons():
    cl = mixed_classes()
    assert len(cl) == 32
    assert {(c.nq, c.horizon) for c in cl} == {(q, N) for q in range(1, 9) for N in (10, 20, 30, 50)}
    for c in cl:
        assert c.ni == (1 if c.nq == 1 else c.nq * (c.nq - 1) // 2)


def test_problems_regenerate_alone_and_pack():
    classes, cls, theta = make_mixed(300)
    assert theta.size == sum(n_theta(classes[k]) for k in cls)
    assert np.all(np.bincount(cls, minlength=32) > 0)
    off = np.concatenate([[0], np.cumsum([n_theta(classes[k]) for k in cls])])
    for j in (0, 17, 299):
        _, cj, tj = make_mixed(1, first_id=j)
        assert cj[0] == cls[j]
        np.testing.assert_array_equal(tj, theta[off[j]:off[j + 1]])


def test_single_class_matches_the_multi_quadrotor_drawing_rules():
    classes, cls, theta = make_mixed(50, max_quads=1, horizons=(25,))
    assert np.all(cls == 0) and classes[0].n_sph == 1
    rows = theta.reshape(50, n_theta(classes[0]))
    # starts and goals in the 10 m cube, one sphere of radius 0.5
    assert np.all((rows[:, 0:3] >= 0) & (rows[:, 0:3] <= 10))
    assert np.all(rows[:, -1] == 0.5)
    _, ref = make_batch("multi4", 1)
    assert ref.shape[1] > 0
