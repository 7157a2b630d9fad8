"""Learned warm start on the GPU against the CPU oracle (GPU tests, through the C ABI).

* the proposer network: forward pass, loss gradient and one Adam step of the
  bfloat16 tensor-core kernels against the FP64 network of oracle.mlp, both at
  the kernels' rounding points (tight) and in plain FP64 (the bfloat16 bound);
* the encodings: features and targets bit for bit, decoded starting points;
* the warm-started iteration from the same starting point as the oracle's;
* cold fallback when the KKT test rejects a warm-started run;
* what a network trained on this solver's own solutions gains over cold start.
"""

import numpy as np
import pytest
import torch

from oracle import ipm, mlp, warm
from oracle_bridge import oracle_warm_case
from oracle.quadrotor import QuadNLP
from workloads import ProblemDesc, make_batch, mlp_init

pytestmark = pytest.mark.gpu

WIDTHS = (162, 256, 256, 256, 652)


@pytest.fixture(scope="module")
def bipm():
    assert torch.cuda.is_available()
    from paper_2606_26341_gb300 import bipm as b

    b.load_library()
    return b


def _net_inputs(seed, rows, widths=WIDTHS):
    rng = np.random.default_rng(seed)
    flat = mlp_init(widths, seed)
    # non-zero biases so that the bias paths are exercised
    flat = flat.copy()
    pos = 0
    for i in range(len(widths) - 1):
        pos += widths[i + 1] * widths[i]
        flat[pos:pos + widths[i + 1]] = rng.uniform(-0.2, 0.2, widths[i + 1])
        pos += widths[i + 1]
    x = rng.standard_normal((rows, widths[0])).astype(np.float32)
    t = (0.5 * rng.standard_normal((rows, widths[-1]))).astype(np.float32)
    return flat, x, t


def _layer_slices(widths):
    out, pos = [], 0
    for i in range(len(widths) - 1):
        nw = widths[i + 1] * widths[i]
        out.append(slice(pos, pos + nw))
        out.append(slice(pos + nw, pos + nw + widths[i + 1]))
        pos += nw + widths[i + 1]
    return out


@pytest.mark.parametrize("rows", [1, 300])
def test_forward_matches_oracle(bipm, rows):
    flat, x, _ = _net_inputs(11, rows)
    with bipm.MLP(WIDTHS, max_rows=128) as net:   # 300 rows: three chunks of max_rows
        net.set_params(flat)
        got = net.forward(x).astype(np.float64)
    ref_em, _ = mlp.forward(WIDTHS, flat.astype(np.float64), x.astype(np.float64), emulate_bf16=True)
    ref, _ = mlp.forward(WIDTHS, flat.astype(np.float64), x.astype(np.float64))
    scale = 1.0 + np.max(np.abs(ref))
    # same rounding points: FP32 accumulation order and tanhf are the only differences
    assert np.max(np.abs(got - ref_em)) <= 2e-3 * scale
    # against exact FP64 arithmetic: the bfloat16 operand bound (2^-8 per rounding)
    assert np.linalg.norm(got - ref) <= 3e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("rows", [7, 200, 1100])
def test_gradient_matches_oracle(bipm, rows):
    """Loss and parameter gradient; 1100 rows take the split-K weight-gradient path."""
    flat, x, t = _net_inputs(12 + rows, rows)
    with bipm.MLP(WIDTHS, max_rows=1100) as net:
        net.set_params(flat)
        loss, g = net.loss_grad(x, t)
    f64 = flat.astype(np.float64)
    l_em, g_em = mlp.loss_and_grad(WIDTHS, f64, x.astype(np.float64), t.astype(np.float64), emulate_bf16=True)
    l_ex, g_ex = mlp.loss_and_grad(WIDTHS, f64, x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(l_em, rel=1e-4)
    assert loss == pytest.approx(l_ex, rel=3e-2)
    g = g.astype(np.float64)
    for sl in _layer_slices(WIDTHS):
        assert np.linalg.norm(g[sl] - g_em[sl]) <= 2e-3 * np.linalg.norm(g_em[sl]), sl
        assert np.linalg.norm(g[sl] - g_ex[sl]) <= 5e-2 * np.linalg.norm(g_ex[sl]), sl
    # element by element: each gradient entry is a sum of products (dz_i a_j over
    # the rows, or dz_i alone for a bias); its magnitude bound M sums the products'
    # absolute values.  With the same bfloat16 rounding points on both sides the
    # kernels differ from the emulation by FP32 accumulation and by operands whose
    # bfloat16 rounding flips between neighbours (one unit 2^-8 of a factor of a
    # term: two per product, and as many again through the back-propagated
    # error the term's dz inherits), so |g - g_em| <= 4 * 2^-8 * M entry by entry.
    M = _grad_magnitude(WIDTHS, f64, x.astype(np.float64), t.astype(np.float64))
    ratio = np.abs(g - g_em) / (2.0 ** -8 * M + 1e-30)
    print(f"rows {rows}: max |g - g_em| / (2^-8 M) = {ratio.max():.3f}")
    assert np.all(np.abs(g - g_em) <= 4.0 * 2.0 ** -8 * M + 1e-12)


def _grad_magnitude(widths, flat, x, t):
    """Entry-wise magnitude of the loss gradient's sums: |dz_l|^T |a_{l-1}| for the
    weights and sum |dz_l| for the biases, with |dz| propagated through |W| and
    |tanh'| (the chain rule of oracle.mlp.loss_and_grad with absolute values)."""
    layers = mlp.unpack(widths, flat)
    out, acts = mlp.forward(widths, flat, x)
    dz = (out - t) / out.shape[0]
    dza = np.abs(dz)
    res = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        res[l] = (dza.T @ np.abs(acts[l]), dza.sum(axis=0))
        if l > 0:
            d = 1.0 - acts[l] * acts[l]
            dz, dza = (dz @ W) * d, (dza @ np.abs(W)) * np.abs(d)
    return mlp.pack(res)


def test_adam_step_matches_oracle(bipm):
    rows = 256
    flat, x, t = _net_inputs(21, 2 * rows)
    rng = np.random.default_rng(22)
    sel = np.sort(rng.choice(2 * rows, rows, replace=False)).astype(np.int32)
    lr = 1e-3
    with bipm.MLP(WIDTHS, max_rows=rows) as net:
        net.set_params(flat)
        xd = torch.as_tensor(x, device="cuda")
        td = torch.as_tensor(t, device="cuda")
        loss = net.train_step(xd, td, torch.as_tensor(sel, device="cuda"), rows, lr, want_loss=True)
        after = net.get_params().astype(np.float64)
    f64 = flat.astype(np.float64)
    l_em, g_em = mlp.loss_and_grad(WIDTHS, f64, x[sel].astype(np.float64), t[sel].astype(np.float64),
                                   emulate_bf16=True)
    assert loss == pytest.approx(l_em, rel=1e-4)
    ref = mlp.Adam(f64.size).step(f64, g_em, lr)
    step, ref_step = after - f64, ref - f64
    # Adam's first step is lr * g / (|g| + eps): components with a clear gradient
    # move by lr in the gradient's direction on both sides; every component moves
    # by at most lr
    clear = np.abs(g_em) > 1e-2 * np.sqrt(np.mean(g_em ** 2))
    assert np.max(np.abs(step[clear] - ref_step[clear])) <= 1e-6 + 1e-3 * lr
    assert np.max(np.abs(step)) <= lr * (1 + 1e-5)
    assert clear.mean() > 0.9


def test_training_on_the_gpu_reduces_the_loss(bipm):
    widths = (12, 64, 64, 24)
    rng = np.random.default_rng(31)
    n = 4096
    x = rng.uniform(-1, 1, (n, 12)).astype(np.float32)
    basis = rng.standard_normal((12, 24))
    t = np.tanh(x @ basis / 2.0).astype(np.float32)
    flat = mlp_init(widths, 32)
    with bipm.MLP(widths, max_rows=256) as net:
        net.set_params(flat)
        xd = torch.as_tensor(x, device="cuda")
        td = torch.as_tensor(t, device="cuda")
        first = None
        for s in range(600):
            idx = torch.as_tensor(rng.choice(n, 256, replace=False).astype(np.int32), device="cuda")
            l = net.train_step(xd, td, idx, 256, 3e-3, want_loss=(s == 0 or s == 599))
            if s == 0:
                first = l
        last = l
        trained = net.get_params().astype(np.float64)
    assert last < 0.1 * first
    # the trained parameters give the oracle's network the same small loss
    l_oracle, _ = mlp.loss_and_grad(widths, trained, x.astype(np.float64), t.astype(np.float64))
    assert l_oracle < 0.15 * first


# ----------------------------------------------------------------- encodings

def _cyl(count, horizon=40, first_id=0):
    return make_batch("cyl", count, first_id=first_id,
                      desc=ProblemDesc(nq=1, horizon=horizon, dt=0.05, n_cyl=50))


def test_features_and_targets_bit_exact(bipm):
    desc, theta = _cyl(64)
    td = torch.as_tensor(theta, device="cuda")
    f = torch.empty((64, 162), dtype=torch.float32, device="cuda")
    bipm.warm_features(desc, td, 50, f)
    ref = np.stack([warm.features(desc, th, 50) for th in theta]).astype(np.float32)
    np.testing.assert_array_equal(f.cpu().numpy(), ref)
    # fewer kept cylinders than the problem has, and more
    for k in (7, 60):
        fk = torch.empty((64, 12 + 3 * k), dtype=torch.float32, device="cuda")
        bipm.warm_features(desc, td, k, fk)
        refk = np.stack([warm.features(desc, th, k) for th in theta]).astype(np.float32)
        np.testing.assert_array_equal(fk.cpu().numpy(), refk)
    rng = np.random.default_rng(41)
    x = np.stack([QuadNLP(desc, th).default_start() for th in theta]) + rng.standard_normal((64, desc.n))
    tg = torch.empty((64, warm.output_dim(desc)), dtype=torch.float32, device="cuda")
    bipm.warm_encode(desc, td, torch.as_tensor(x, device="cuda"), tg)
    reft = np.stack([warm.encode(desc, theta[j], x[j]) for j in range(64)]).astype(np.float32)
    np.testing.assert_array_equal(tg.cpu().numpy(), reft)


def test_decode_matches_oracle(bipm):
    desc, theta = _cyl(32, horizon=12)
    rng = np.random.default_rng(42)
    out = (0.3 * rng.standard_normal((32, warm.output_dim(desc)))).astype(np.float32)
    xg = torch.empty((32, desc.n), dtype=torch.float64, device="cuda")
    bipm.warm_decode(desc, torch.as_tensor(theta, device="cuda"), torch.as_tensor(out, device="cuda"), xg)
    got = xg.cpu().numpy()
    for j in range(32):
        nlp = QuadNLP(desc, theta[j])
        ref = warm.decode(desc, theta[j], out[j].astype(np.float64),
                          lambda s: nlp.ineq(torch.as_tensor(s)).numpy())
        np.testing.assert_allclose(got[j], ref, rtol=1e-15, atol=1e-13)


def test_warm_encodings_reject_other_families(bipm):
    desc, theta = make_batch("track", 2)
    f = torch.empty((2, 162), dtype=torch.float32, device="cuda")
    with pytest.raises(bipm.BipmError, match="one quadrotor among cylinders"):
        bipm.warm_features(desc, torch.as_tensor(theta, device="cuda"), 50, f)


# ------------------------------------------------------------ warm-started solves

def test_warm_queue_matches_oracle_from_the_same_start(bipm):
    import multiprocessing as mp
    import os

    desc, theta = _cyl(8, horizon=12)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    with mp.get_context("spawn").Pool(8) as pool:
        cases = pool.map(oracle_warm_case, [(desc, theta[j], j) for j in range(8)])
    guess = np.ascontiguousarray(np.stack([c[0] for c in cases]))
    x = np.empty((8, desc.n))
    with bipm.Batch(desc, 8, bipm.Options(precision=0)) as b:
        r = b.solve_queue(np.ascontiguousarray(theta), x, x_guess=guess)
    same = 0
    for j, (_, ost, oit, ox, _) in enumerate(cases):
        if ost == ipm.CONVERGED:
            assert r["status"][j] == bipm.CONVERGED
            assert r["warm"][j] == 1
            err = np.max(np.abs(x[j] - ox) / (1.0 + np.abs(ox)))
            assert err <= 1e-5, (j, err)
            same += r["iters"][j] == oit
    assert same >= 6, [(r["iters"][j], cases[j][2]) for j in range(8)]


def test_rejected_warm_start_falls_back_to_cold(bipm):
    desc, theta = _cyl(4, horizon=12)
    guess = np.stack([QuadNLP(desc, th).default_start() for th in theta])
    with bipm.Batch(desc, 4, bipm.Options(precision=0, max_iter=2)) as b:
        r = b.solve_queue(np.ascontiguousarray(theta), None, x_guess=np.ascontiguousarray(guess))
    assert np.all(r["warm"] == 2)
    assert np.all(r["warm_iters"] == 2)
    assert np.all(r["status"] == bipm.MAX_ITER)
    with bipm.Batch(desc, 4, bipm.Options(precision=0)) as b:
        r = b.solve_queue(np.ascontiguousarray(theta), None)
    assert np.all(r["warm"] == 0)


def test_trained_warm_start_beats_cold_start(bipm):
    """Train the proposer on this solver's solutions of one set of cluttered
    problems, then solve a disjoint set warm and cold: the warm start must need
    fewer iterations in total (fallback runs included) at the same accuracy."""
    from paper_2606_26341_gb300 import warmstart

    desc, theta_train = _cyl(6144, first_id=10_000)
    _, theta_test = _cyl(1024, first_id=0)
    opts = bipm.Options(precision=1, fp32_switch=1e2)
    tr = torch.as_tensor(theta_train, device="cuda")
    data = warmstart.make_dataset(desc, tr, opts, capacity=4096)
    assert len(data.usable) > 0.95 * 6144
    with bipm.MLP(warmstart.widths(desc), max_rows=512) as net:
        net.set_params(mlp_init(warmstart.widths(desc), 5))
        hist = warmstart.train(net, data, epochs=30, batch=256, lr=2e-3, lr_final=1e-4, seed=6)
        te = torch.as_tensor(theta_test, device="cuda")
        guess = warmstart.propose(net, desc, te)
    assert hist[-1] < 0.3 * hist[0]
    with bipm.Batch(desc, 1024, opts) as b:
        r_cold = b.solve_queue(theta_test, None)
        r_warm = b.solve_queue(theta_test, None, x_guess=guess.cpu().numpy())
    conv_c = r_cold["status"] == bipm.CONVERGED
    conv_w = r_warm["status"] == bipm.CONVERGED
    it_c = r_cold["iters"].sum()
    it_w = (r_warm["iters"] + r_warm["warm_iters"]).sum()
    print(f"cold: {conv_c.mean():.4f} converged, {r_cold['iters'].mean():.1f} iterations; warm: "
          f"{conv_w.mean():.4f} converged, {(it_w / 1024):.1f} iterations incl. fallback "
          f"({np.mean(r_warm['warm'] == 2):.3f} fell back); loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    assert conv_w.mean() >= conv_c.mean() - 0.005
    assert np.max(r_warm["kkt_err"][conv_w]) <= 1e-6
    assert it_w < 0.9 * it_c


def test_training_rejects_indices_outside_the_data(bipm):
    widths = (12, 16, 8)
    rng = np.random.default_rng(51)
    x = torch.as_tensor(rng.standard_normal((64, 12)).astype(np.float32), device="cuda")
    t = torch.as_tensor(rng.standard_normal((64, 8)).astype(np.float32), device="cuda")
    with bipm.MLP(widths, max_rows=32) as net:
        net.set_params(mlp_init(widths, 52))
        ok = torch.arange(32, dtype=torch.int32, device="cuda")
        net.train_step(x, t, ok, 32, 1e-3, want_loss=True)
        bad = ok.clone()
        bad[5] = 64  # one past the last row
        with pytest.raises(bipm.BipmError, match="outside"):
            net.train_step(x, t, bad, 32, 1e-3, want_loss=True)
        # the flag is cleared: the next valid step succeeds
        net.train_step(x, t, ok, 32, 1e-3, want_loss=True)
