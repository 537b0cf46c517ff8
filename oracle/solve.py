"""Oracle ridge solvers: direct Cholesky and textbook preconditioned CG.

Test infrastructure only.  Section 2 ("Iterative solvers") of the paper solves
(K + lambda I) A = Y with conjugate gradients, one CG per label column run in
lock-step (Appendix B.3: "the CG routine is fully vectorized over tasks"); it
cites Shewchuk's tutorial for CG.  The Jacobi preconditioner M = diag(K) +
lambda is the one the benchmark configurations fix.
"""

from __future__ import annotations

import numpy as np


def cholesky_solve(K, Y, lam: float) -> np.ndarray:
    """A* = (K + lam I)^{-1} Y by float64 Cholesky and two triangular solves."""
    import scipy.linalg as sla

    K = np.asarray(K, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = K.shape[0]
    L = np.linalg.cholesky(K + lam * np.eye(n))
    Z = sla.solve_triangular(L, Y, lower=True)
    return sla.solve_triangular(L.T, Z, lower=False)


def pcg(K, Y, lam: float, precond: str = "jacobi", tol: float = 1e-6,
        maxit: int = 10000):
    """Column-wise preconditioned CG for (K + lam I) X = Y, float64.

    Per column: x = 0, r = y, z = M^{-1} r, p = z; each iteration
    alpha = r.z / p.Ap, x += alpha p, r -= alpha Ap, z = M^{-1} r,
    beta = r_new.z_new / r.z, p = z + beta p.  A column stops (is frozen) once
    ||r|| / ||y|| <= tol, and the stop is confirmed on the recomputed true
    residual y - (K + lam I) x.  Returns (X, iters, relres) with iters the
    largest iteration count over columns and relres the per-column true
    relative residuals.
    """
    K = np.asarray(K, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    n, R = Y.shape
    A = K + lam * np.eye(n)
    if precond == "jacobi":
        minv = 1.0 / np.diag(A)
    elif precond == "none":
        minv = np.ones(n)
    else:
        raise ValueError(precond)
    X = np.zeros((n, R))
    ynorm = np.linalg.norm(Y, axis=0)
    ynorm[ynorm == 0] = 1.0
    iters = np.zeros(R, dtype=np.int64)
    for col in range(R):
        x = np.zeros(n)
        r = Y[:, col].copy()
        z = minv * r
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit:
            if np.linalg.norm(r) / ynorm[col] <= tol:
                true_r = Y[:, col] - A @ x
                if np.linalg.norm(true_r) / ynorm[col] <= tol:
                    break
                r = true_r  # residual replacement, then keep iterating
                z = minv * r
                p = z.copy()
                rz = r @ z
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x = x + alpha * p
            r = r - alpha * Ap
            z = minv * r
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            it += 1
        X[:, col] = x
        iters[col] = it
    relres = np.linalg.norm(Y - A @ X, axis=0) / ynorm
    return X, int(iters.max()), relres
