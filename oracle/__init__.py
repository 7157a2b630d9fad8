"""CPU reference ("oracle") for the batched interior-point method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute this package: only the tests, the package smoke check and the CPU
baseline leg of the benchmark use it.  It shares no code with the CUDA path.

It is a plain, slow, FP64 restatement of what the paper's method computes for
one problem at a time:

* ``quadrotor``  - the multiple-shooting NMPC transcription of the quadrotor
  problems (problem form of Eq. 1, inequalities through slacks), written as
  plain PyTorch CPU functions; derivatives come from PyTorch autograd (a library
  primitive) of the stage functions, assembled into the full Jacobian and
  Lagrangian Hessian, never from hand-written code.
* ``ipm``        - the primal-dual interior-point iteration the paper reviews
  in Sec. IV (barrier Eq. 3, Lagrangian Eq. 4, optimality conditions Eq. 5,
  Newton system Eq. 6 reduced to the augmented system Eq. 7, inertia
  correction, and the branches of Table I: backtracking filter line search,
  second-order correction, watchdog and soft feasibility restoration (both
  optional, off by default), tiny step, hard feasibility restoration, and the
  monotone or the adaptive barrier update).  The details the paper defers to the IPOPT paper
  (Wachter & Biegler 2006) follow that paper's algorithm as read in the design
  notes.  Linear algebra is the dense full-space augmented matrix factorised
  by LAPACK's Bunch-Kaufman LDL^T (scipy.linalg.ldl); inertia is read off D.

* ``quat13``     - the 13-state quaternion quadrotor of Sec. VI (position,
  attitude quaternion, body velocities; rotor speeds as inputs) on the same
  NLP transcription; it has no CUDA counterpart yet (parity unpinned).
* ``mlp``        - the learned warm start's network in FP64 (forward pass,
  chain-rule gradient, Adam), optionally rounding product operands to
  bfloat16 at the CUDA kernels' rounding points.
* ``warm``       - the warm start's encodings (network input features,
  training targets, decoding of a network output into a starting point) and
  the warm starting options of the iteration.
* ``generic``    - small NLPs from PyTorch callables, for the closed-form and
  brute-force pins.

Parity unpinned: none of the functions here is left without a pin; the pins
live in tests/test_oracle_*.py.
"""
