"""Seeded random initial weights for the warm-start network.

Draws numbers only (Glorot-uniform weights, zero biases) in the flat layout
both sides use: for every layer W (width_out x width_in, row-major), then b.
"""

from __future__ import annotations

import numpy as np


def mlp_init(dims, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
