"""Small NLPs given as plain PyTorch callables (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Wraps f(x) and c(x) written with torch operations into the NLP interface the
oracle's interior-point iteration uses (Eq. 1: min f s.t. c = 0, bounds);
derivatives come from PyTorch autograd.  Used to pin the oracle on problems
with closed-form or brute-force solutions.
"""

from __future__ import annotations

import numpy as np
import torch

F64 = torch.float64


class TorchNLP:
    def __init__(self, f, c, n, m, xl=None, xu=None, x0=None):
        self._f = f
        self._c = c
        self.n, self.m = n, m
        self.xl = np.full(n, -np.inf) if xl is None else np.asarray(xl, dtype=np.float64)
        self.xu = np.full(n, np.inf) if xu is None else np.asarray(xu, dtype=np.float64)
        self._x0 = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64)

    def _ct(self, w):
        if self.m == 0:
            return torch.zeros(0, dtype=F64)
        return self._c(w)

    def f(self, w):
        return float(self._f(torch.as_tensor(w, dtype=F64)))

    def c(self, w):
        return self._ct(torch.as_tensor(w, dtype=F64)).detach().numpy()

    def grad_f(self, w):
        return torch.func.grad(self._f)(torch.as_tensor(w, dtype=F64)).numpy()

    def jac_c(self, w):
        if self.m == 0:
            return np.zeros((0, self.n))
        return torch.func.jacfwd(self._ct)(torch.as_tensor(w, dtype=F64)).numpy()

    def hess_lag(self, w, y, obj_factor=1.0):
        yt = torch.as_tensor(y, dtype=F64)

        def lag(wt):
            val = obj_factor * self._f(wt)
            if self.m:
                val = val + (yt * self._ct(wt)).sum()
            return val

        return torch.func.hessian(lag)(torch.as_tensor(w, dtype=F64)).numpy()

    def default_start(self):
        return self._x0.copy()
