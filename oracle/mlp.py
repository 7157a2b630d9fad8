"""Warm-start network on the CPU in FP64: forward pass, loss gradient, Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The method's learned warm start (the MLP proposer of primal initial guesses
for the interior-point iteration of Sec. IV) is a plain multilayer
perceptron:

    a_0 = x
    z_l = a_{l-1} W_l^T + b_l,   a_l = tanh(z_l)    (hidden layers l < L)
    out = z_L                                        (linear output layer)

with W_l of shape (width_l, width_{l-1}) and loss

    loss = 1 / (2 B) * sum_b |out_b - t_b|^2         (B rows in the batch).

The gradient is the chain rule written out layer by layer (backpropagation),
and the optimiser is Adam (Kingma & Ba, 2015: first and second moment
estimates with bias correction).

`emulate_bf16` reproduces the CUDA kernels' precision contract: the
operands of every matrix product (inputs, weights, activations and the
back-propagated errors) are rounded to bfloat16 before the product, whose
sum and everything else stays in wide precision.  With it off, the network
is evaluated in FP64 at the given parameters.

Parameters travel as one flat float vector: for every layer W_l (row-major,
width_l x width_{l-1}) followed by b_l.
"""

from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to the nearest bfloat16 value (8 significant bits, ties to even).

    Finite values in the normal FP32 range only (the network's values are
    far from both ends of it)."""
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                       # a = m * 2**e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def n_params(dims):
    return sum(dims[i + 1] * dims[i] + dims[i + 1] for i in range(len(dims) - 1))


def unpack(dims, flat):
    """Flat parameter vector -> [(W_l, b_l)]."""
    flat = np.asarray(flat, dtype=np.float64)
    out, pos = [], 0
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        W = flat[pos:pos + fan_out * fan_in].reshape(fan_out, fan_in)
        pos += fan_out * fan_in
        b = flat[pos:pos + fan_out]
        pos += fan_out
        out.append((W, b))
    assert pos == flat.size, "parameter vector does not match the layer widths"
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(dims, flat, x, emulate_bf16=False):
    """Network output and the activations the gradient needs."""
    rnd = bf16 if emulate_bf16 else (lambda v: v)
    layers = unpack(dims, flat)
    a = np.asarray(x, dtype=np.float64)
    acts = [a]
    for l, (W, b) in enumerate(layers):
        z = rnd(a) @ rnd(W).T + b
        if l < len(layers) - 1:
            a = np.tanh(z)
            acts.append(a)
        else:
            a = z
    return a, acts


def loss_and_grad(dims, flat, x, t, emulate_bf16=False):
    """Loss 1/(2B) |out - t|^2 and its gradient with respect to the flat parameters."""
    rnd = bf16 if emulate_bf16 else (lambda v: v)
    layers = unpack(dims, flat)
    out, acts = forward(dims, flat, x, emulate_bf16)
    t = np.asarray(t, dtype=np.float64)
    B = out.shape[0]
    err = out - t
    loss = 0.5 * float(np.sum(err * err)) / B
    dz = err / B                                  # d loss / d z_L
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_prev = acts[l]
        grads[l] = (rnd(dz).T @ rnd(a_prev), dz.sum(axis=0))
        if l > 0:
            da = rnd(dz) @ rnd(W)                 # d loss / d a_{l-1}
            dz = da * (1.0 - a_prev * a_prev)     # tanh'(z) = 1 - tanh(z)^2
    return loss, pack(grads)


class Adam:
    """Adam with bias-corrected moments; state is FP64 here."""

    def __init__(self, size, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(size)
        self.v = np.zeros(size)
        self.t = 0
        self.beta1, self.beta2, self.eps = beta1, beta2, eps

    def step(self, flat, grad, lr):
        self.t += 1
        b1, b2 = self.beta1, self.beta2
        self.m = b1 * self.m + (1.0 - b1) * grad
        self.v = b2 * self.v + (1.0 - b2) * grad * grad
        m_hat = self.m / (1.0 - b1 ** self.t)
        v_hat = self.v / (1.0 - b2 ** self.t)
        return flat - lr * m_hat / (np.sqrt(v_hat) + self.eps)
