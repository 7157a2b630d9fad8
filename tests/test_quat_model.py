"""The CUDA side's 13-state model routines (csrc/quat_model.cuh), built for the
host from the same source the kernels would compile, against the oracle's
13-state model (oracle/quat13.py): the RK4 step, the gradient of lam^T F from
the hand-derived adjoint, and the forward-over-reverse Jacobian- and
Hessian-vector products, all against PyTorch autograd of the oracle's RK4 step.
The routines are not used by the iteration kernels yet."""

import os
import subprocess
import tempfile

import numpy as np
import torch

from oracle.quadrotor import rk4
from oracle.quat13 import OMEGA_H, quat13_rhs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2606_26341_gb300", "csrc")
F64 = torch.float64


def _cases(rng, count):
    out = []
    for j in range(count):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        if j % 3 == 0:
            q *= 1.0 + 0.01 * rng.standard_normal()  # off the unit sphere as RK4 drifts
        x = np.concatenate([rng.uniform(-3, 3, 3), q, rng.uniform(-2, 2, 3), rng.uniform(-2, 2, 3)])
        u = OMEGA_H * rng.uniform(0.2, 1.4, 4)
        lam = rng.standard_normal(13)
        d = rng.standard_normal(17)
        d[13:] *= 50.0  # rotor-speed directions on their own scale
        out.append((0.1 if j % 2 else 0.05, x, u, lam, d))
    return out


def test_device_model_routines_match_the_oracle():
    rng = np.random.default_rng(13)
    cases = _cases(rng, 40)
    text = "\n".join(" ".join(f"{v:.17g}" for v in [dt, *x, *u, *lam, *d]) for dt, x, u, lam, d in cases)
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "quat_model_check")
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "quat_model_check.cpp"),
                        "-o", exe], check=True)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    rows = [np.array(line.split(), dtype=np.float64) for line in out.strip().splitlines()]
    assert len(rows) == len(cases)
    for (dt, x, u, lam, d), r in zip(cases, rows):
        F, F2, gx, gu = r[0:13], r[13:26], r[26:39], r[39:43]
        Fd, gxd, gud = r[43:56], r[56:69], r[69:73]
        lam_t = torch.as_tensor(lam)

        def step(z):
            return rk4(z[:13], z[13:], dt, quat13_rhs)

        def grad(z):
            return torch.func.vjp(step, z)[1](lam_t)[0]

        z = torch.as_tensor(np.concatenate([x, u]))
        dz = torch.as_tensor(d)
        F_ref = step(z).numpy()
        g_ref = grad(z).numpy()
        _, jvp = torch.func.jvp(step, (z,), (dz,))
        _, hvp = torch.func.jvp(grad, (z,), (dz,))
        scale = lambda a: 1e-12 * max(1.0, np.abs(a).max())  # noqa: E731
        assert np.abs(F - F_ref).max() <= scale(F_ref)
        assert np.abs(F2 - F_ref).max() <= scale(F_ref)
        assert np.abs(np.concatenate([gx, gu]) - g_ref).max() <= scale(g_ref)
        assert np.abs(Fd - jvp.numpy()).max() <= scale(jvp.numpy())
        assert np.abs(np.concatenate([gxd, gud]) - hvp.numpy()).max() <= scale(hvp.numpy())
