"""FP64 CPU oracle for the Myrtle / FC NNGP kernels and the kernel-ridge solve.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA product path (``paper_2303_05420_gb300``) never imports, calls or links
anything here, and nothing here imports the product path.

What it computes, and where each definition comes from
-------------------------------------------------------
The paper (Adlam et al., arXiv 2303.05420) specifies its kernels only as Neural
Tangents ``stax`` architecture listings (Appendix A: the FC3, CV8 and Myrtle
listings) and solves the ridge system with preconditioned conjugate gradients
(Section 2, "Iterative solvers").  It prints no kernel formula, so the oracle
follows the *definition* of the NNGP: the covariance of the scalar output of the
listed random network as every hidden width goes to infinity, weights
N(0, sigma_w^2 / fan_in) with fan_in = C_in * k^2, biases N(0, sigma_b^2).

* ``kernels.py``: ReLU arc-cosine map, Myrtle pixel-pair recursion (full
  (H*W) x (H'*W') tensors, no band or plane tricks), per-pixel self-variances
  taken from the full self tensor, FC3 kernel.  Written with plain torch
  float64 CPU ops so that autograd gives the exact adjoint of the written-out
  definition (the only custom derivative is J'(c) = pi - arccos(c), which is
  the closed-form derivative of the arc-cosine map).
* ``solve.py``: Cholesky ridge solve and textbook Jacobi-preconditioned CG.
* ``krr.py``: the kernel-ridge support-set loss and its gradient.

Parity status: every function here is pinned by a test in ``tests/`` that does
not re-type its formula (quadrature, Monte Carlo finite networks, closed forms,
a loop-by-loop brute force, special-case reductions, Cholesky, central
differences).  None is "parity unpinned".
"""

from .kernels import (  # noqa: F401
    Arch,
    relu_map,
    arccos_J,
    myrtle_self_q,
    myrtle_pair,
    myrtle_block,
    myrtle_layers_pair,
    myrtle_ntk_pair,
    myrtle_ntk_block,
    relu_derivative_map,
    erf_map,
    erf_derivative_map,
    cv_pair,
    cv_block,
    fc_nngp,
)
from .solve import cholesky_solve, pcg, pivchol_apply, pivoted_cholesky  # noqa: F401
from .krr import krr_loss, krr_loss_and_grads  # noqa: F401
