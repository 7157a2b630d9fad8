"""Learned warm start: dataset from this solver's own solutions, training of the
proposer network on the GPU, and warm-started solves with cold fallback.

Orchestration only: features, targets, the network's forward and backward
passes, Adam, the decoding of a proposal and the solves all run in the CUDA
library (bipm_warm_*, bipm_mlp_*, bipm_solve_queue[_warm]).  PyTorch provides
device buffers; index permutations are drawn on the host.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import bipm

HIDDEN = (256, 256, 256)
K_NEAR = 50


def widths(desc, k_near=K_NEAR, hidden=HIDDEN):
    """Layer widths (input, hidden..., output) of the proposer for this family."""
    return (12 + 3 * k_near, *hidden, 12 * (desc.horizon + 1) + 4 * desc.horizon)


@dataclasses.dataclass
class Dataset:
    features: object   # CUDA float32 (count x n_in)
    targets: object    # CUDA float32 (count x n_out)
    usable: np.ndarray  # row indices of converged solves
    results: dict       # per-problem solver results of the cold solves


def solve_cold(desc, theta_dev, options, capacity, stream=None):
    """Cold queue solve of every row; returns (x (CUDA float64), results dict)."""
    import torch

    n = theta_dev.shape[0]
    x = torch.empty((n, desc.n), dtype=torch.float64, device=theta_dev.device)
    res = torch.empty(n * bipm.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=theta_dev.device)
    with bipm.Batch(desc, capacity, options, stream=stream) as b:
        b.solve_queue(theta_dev, x, res)
    return x, bipm.results_from_bytes(res.cpu().numpy())


def make_dataset(desc, theta_dev, options, capacity, k_near=K_NEAR, stream=None):
    """Solve every problem cold and encode (features, targets) of the solutions."""
    import torch

    x, r = solve_cold(desc, theta_dev, options, capacity, stream)
    n = theta_dev.shape[0]
    w = widths(desc, k_near)
    feats = torch.empty((n, w[0]), dtype=torch.float32, device=theta_dev.device)
    targ = torch.empty((n, w[-1]), dtype=torch.float32, device=theta_dev.device)
    bipm.warm_features(desc, theta_dev, k_near, feats, stream)
    bipm.warm_encode(desc, theta_dev, x, targ, stream)
    usable = np.nonzero(r["status"] == bipm.CONVERGED)[0].astype(np.int32)
    return Dataset(feats, targ, usable, r)


def train(net: "bipm.MLP", data: Dataset, epochs: int, batch: int, lr: float, seed: int = 0,
          lr_final: float | None = None, log_every: int = 0):
    """Adam on minibatches of the usable rows; returns the per-epoch mean loss."""
    import torch

    rng = np.random.default_rng(seed)
    rows = data.usable
    dev = data.features.device
    steps_per_epoch = max(1, len(rows) // batch)
    total = epochs * steps_per_epoch
    lr_final = lr if lr_final is None else lr_final
    history = []
    step = 0
    for ep in range(epochs):
        perm = rows[rng.permutation(len(rows))][: steps_per_epoch * batch]
        idx = torch.as_tensor(perm.astype(np.int32), device=dev)
        losses = []
        for s in range(steps_per_epoch):
            # cosine decay from lr to lr_final
            frac = step / max(1, total - 1)
            cur = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * frac))
            want = s == steps_per_epoch - 1 or (log_every and s % log_every == 0)
            l = net.train_step(data.features, data.targets, idx[s * batch:(s + 1) * batch], batch, cur,
                               want_loss=want)
            if want:
                losses.append(l)
            step += 1
        history.append(float(np.mean(losses)))
    return history


def propose(net: "bipm.MLP", desc, theta_dev, k_near=K_NEAR, stream=None):
    """Warm starting points (CUDA float64, count x n) for the rows of theta_dev."""
    import torch

    n = theta_dev.shape[0]
    w = net.widths
    feats = torch.empty((n, w[0]), dtype=torch.float32, device=theta_dev.device)
    out = torch.empty((n, w[-1]), dtype=torch.float32, device=theta_dev.device)
    bipm.warm_features(desc, theta_dev, k_near, feats, stream)
    net.forward(feats, out)
    xg = torch.empty((n, desc.n), dtype=torch.float64, device=theta_dev.device)
    bipm.warm_decode(desc, theta_dev, out, xg, stream)
    return xg
