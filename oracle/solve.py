"""Oracle ridge solvers: direct Cholesky and textbook preconditioned CG.

Test infrastructure only.  Section 2 ("Iterative solvers") of the paper solves
(K + lambda I) A = Y with conjugate gradients, one CG per label column run in
lock-step (Appendix B.3 vectorises its CG routine over the tasks); it
cites Shewchuk's tutorial for CG.  The Jacobi preconditioner M = diag(K) +
lambda is the one the benchmark configurations fix; the paper's own is the
partial pivoted Cholesky preconditioner (Section 2, after Wang et al. 2019):
K is approximated by L^T L from `rank` greedy pivots and M = L^T L + lambda I
is inverted through the Woodbury identity.
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


def pivoted_cholesky(K, rank: int):
    """Partial pivoted Cholesky of a symmetric positive semi-definite K:
    step k takes the pivot i with the largest remaining diagonal d (the
    diagonal of the Schur complement of the pivots so far; the lowest index
    on ties), forms the row l_k = (K[i, :] - sum_{m<k} L[m, i] L[m, :]) /
    sqrt(d[i]) and updates d -= l_k^2.  Stops early when the largest d is at
    most 1e-12 of the largest diagonal of K (numerically exhausted rank).
    Returns (L [k][n], pivots [k]) with K ~ L^T L."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    rank = min(int(rank), n)
    d = np.diag(K).copy()
    floor = 1e-12 * d.max() if n else 0.0
    L = np.zeros((rank, n))
    piv = []
    for k in range(rank):
        i = int(np.argmax(d))
        if not d[i] > floor:
            break
        row = K[i, :] - L[:k, i] @ L[:k, :]
        L[k] = row / np.sqrt(d[i])
        d = d - L[k] ** 2
        piv.append(i)
    return L[:len(piv)], piv


def pivchol_apply(L, lam: float, V):
    """(L^T L + lam I)^{-1} V by the Woodbury identity:
    (V - L^T (lam I + L L^T)^{-1} L V) / lam."""
    import scipy.linalg as sla

    V = np.asarray(V, dtype=np.float64)
    r = L.shape[0]
    if r == 0:
        return V / lam
    G = lam * np.eye(r) + L @ L.T
    C = np.linalg.cholesky(G)
    T = L @ V
    U = sla.solve_triangular(C.T, sla.solve_triangular(C, T, lower=True), lower=False)
    return (V - L.T @ U) / lam


def pcg(K, Y, lam: float, precond: str = "jacobi", tol: float = 1e-6,
        maxit: int = 10000, rank: int = 0):
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
        dinv = 1.0 / np.diag(A)
        minv = lambda v: dinv * v  # noqa: E731
    elif precond == "none":
        minv = lambda v: v  # noqa: E731
    elif precond == "pivchol":
        Lp, _ = pivoted_cholesky(K, rank)
        minv = lambda v: pivchol_apply(Lp, lam, v)  # noqa: E731
    else:
        raise ValueError(precond)
    X = np.zeros((n, R))
    ynorm = np.linalg.norm(Y, axis=0)
    ynorm[ynorm == 0] = 1.0
    iters = np.zeros(R, dtype=np.int64)
    for col in range(R):
        x = np.zeros(n)
        r = Y[:, col].copy()
        z = minv(r)
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit:
            if np.linalg.norm(r) / ynorm[col] <= tol:
                true_r = Y[:, col] - A @ x
                if np.linalg.norm(true_r) / ynorm[col] <= tol:
                    break
                r = true_r  # residual replacement, then keep iterating
                z = minv(r)
                p = z.copy()
                rz = r @ z
            Ap = A @ p
            alpha = rz / (p @ Ap)
            x = x + alpha * p
            r = r - alpha * Ap
            z = minv(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
            it += 1
        X[:, col] = x
        iters[col] = it
    relres = np.linalg.norm(Y - A @ X, axis=0) / ynorm
    return X, int(iters.max()), relres
