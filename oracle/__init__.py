"""CPU FP64 oracle for the rational-function log-determinant estimator.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the paper "Fast Approximate Determinants Using Rational
Functions" (Colthurst, Vasudevan, Lottes, Patton; arXiv 2405.03474) computes.
It exists to check the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  The product path (``paper_2405_03474_gb300``) never imports it, and the two
share no code: the only thing both sides use is the seeded input generator
module ``paper_2405_03474_gb300/inputs.py``, which holds none of the method's
arithmetic.

Everything here is numpy float64.  Library primitives (matmul, ``eigh``,
``cholesky``, ``qr``, ``roots``) serve as single steps; there is no blocking,
fusion or reordering beyond what the paper's definitions state.

Modules
-------
coeffs     Eq. 1 rational approximations r_1, r_3, r_5 and their Table 1
           partial-fraction forms.
splitmix   SplitMix64 counter-based generator (Steele, Lea & Flood 2014), used
           for Rademacher probes that the device draws itself.
kernels    Matern-5/2 and RBF covariance functions (Section 3, citing
           Rasmussen & Williams) and dense / row-sampled kernel products.
precond    Randomized truncated SVD preconditioner P = D + A A^T (Section 2,
           Halko et al. Algorithms 4.1/4.4/5.3; Appendix list), its symmetric
           factor L and log det P.
estimator  Algorithm 1 (literal: Lanczos + Thomas) and its converged form
           (exact shifted solves), the multi-shift CG recurrence the device
           runs (Section 2, after Jegerlehner), plus exact Cholesky log det.
gradient   Gradient of the estimator with P frozen, and the exact gradient
           tr(M^-1 dM/dtheta).
mlp        FP64 forward/backward of the 4-128-128-128-1 GELU surrogate MLP.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
fact the paper or the mathematics fixes (see the test files).  The paper prints
no numeric results for its experiments (all are figures), so the absolute
accuracy of the estimator against the paper's own plots is "parity unpinned".
"""
