"""Pins for the oracle ridge solvers and the oracle gradients.

* PCG (Section 2, "Iterative solvers") against a float64 Cholesky solve, for
  ridges drawn from the paper's grid (Appendix C); Jacobi PCG produces the
  same iterates as plain CG on the symmetrically diagonal-scaled system (the
  defining property of a preconditioner applied as M = D).
* The Myrtle kernel architecture is the paper's own (Appendix A listing),
  cross-checked against the golden constants file.
* Gradients of the kernel-ridge loss: autograd through the float64 definition
  against fourth-order central differences at h = 1e-3; Euler identities with sigma_b^2 = 0
  (K is degree-1 homogeneous in each image and degree-L in sigma_w^2).
"""

import json
import os

import numpy as np
import pytest
import torch

from oracle import Arch, cholesky_solve, krr_loss, krr_loss_and_grads, myrtle_block, pcg
from oracle.kernels import myrtle_layers_pair, myrtle_self_q
import nkdata

F64 = torch.float64
GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_golden_constants_match_configs():
    g = json.load(open(GOLD))
    assert g["myrtle_listing"]["stage_convs"] == [3, 3, 3]
    layers = g["myrtle_listing"]["layers"]
    assert layers.count("conv") == 9 and layers.count("avgpool2") == 2
    assert nkdata.WORKLOADS["myrtle10_32x32_grad"]["convs"] == tuple(g["myrtle_listing"]["stage_convs"])
    assert nkdata.WORKLOADS["myrtle5_32x32"]["sw2"] == g["myrtle_listing"]["W_std_squared"]
    grid = np.concatenate([[0.0], np.logspace(g["ridge_grid"]["logspace_start"],
                                              g["ridge_grid"]["logspace_stop"],
                                              g["ridge_grid"]["logspace_num"])])
    assert grid.shape == (50,) and grid[1] == 1e-10 and grid[-1] == 1e4


@pytest.fixture(scope="module")
def gram():
    p = nkdata.image_problem(40, 8, 8, n_classes=10, blur=True)
    K = myrtle_block(Arch((2, 1, 0)), 2.0, 0.0, p.x_train, p.x_train, symmetric=True).numpy()
    return K, p.y_train


@pytest.mark.parametrize("rel_lam", [1e-4, 1e-2, 1.0])
def test_pcg_matches_cholesky(gram, rel_lam):
    K, Y = gram
    n = K.shape[0]
    lam = rel_lam * np.trace(K) / n
    Astar = cholesky_solve(K, Y, lam)
    X, iters, relres = pcg(K, Y, lam, "jacobi", tol=1e-10, maxit=5000)
    assert relres.max() <= 1e-10
    kappa = np.linalg.cond(K + lam * np.eye(n))
    assert np.linalg.norm(X - Astar) / np.linalg.norm(Astar) <= kappa * 1e-10


@pytest.mark.parametrize("k", [1, 2, 4])  # before CG loses orthogonality
def test_jacobi_pcg_is_cg_on_scaled_system(gram, k):
    K, Y = gram
    n = K.shape[0]
    lam = 1e-3 * np.trace(K) / n
    A = K + lam * np.eye(n)
    d = np.sqrt(np.diag(A))
    Ahat = A / d[:, None] / d[None, :]
    X1, _, _ = pcg(K, Y, lam, "jacobi", tol=0.0, maxit=k)
    Xh, _, _ = pcg(Ahat, Y / d[:, None], 0.0, "none", tol=0.0, maxit=k)
    assert np.allclose(X1, Xh / d[:, None], rtol=1e-9, atol=1e-12 * np.abs(X1).max())


def test_cholesky_residual(gram):
    K, Y = gram
    lam = 1e-6 * np.trace(K) / K.shape[0]
    A = cholesky_solve(K, Y, lam)
    r = Y - (K + lam * np.eye(K.shape[0])) @ A
    assert np.linalg.norm(r) / np.linalg.norm(Y) < 1e-9


def test_krr_gradients_match_central_differences():
    arch = Arch((3, 3, 3))
    rng = np.random.default_rng(nkdata.SEED_SUPPORT)
    Xs = rng.standard_normal((3, 4, 4, 3))
    Xt = rng.standard_normal((4, 4, 4, 3))
    Ys = nkdata.labels(3, 10)
    Yt = nkdata.labels(4, 10, seed=9)
    sw2, sb2, lam = 2.0, 0.01, 0.05
    L, dsw2, dsb2, dX = krr_loss_and_grads(arch, sw2, sb2, Xs, Ys, Xt, Yt, lam)
    h = 1e-3

    def f(sw, sb, X):
        return float(krr_loss(arch, sw, sb, X, Ys, Xt, Yt, lam))

    def cd(g, h=h):  # fourth-order central difference at step h
        return (-g(2 * h) + 8 * g(h) - 8 * g(-h) + g(-2 * h)) / (12 * h)

    fd_sw = cd(lambda e: f(sw2 + e, sb2, Xs))
    # sigma_b^2 = 0.01 is itself of the order of the step: step 1e-3 relative to it
    fd_sb = cd(lambda e: f(sw2, sb2 + e, Xs), h=1e-3 * sb2)
    assert abs(dsw2 - fd_sw) <= 1e-5 * abs(fd_sw)
    assert abs(dsb2 - fd_sb) <= 1e-5 * abs(fd_sb)
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1), (2, 3, 0, 2), (0, 1, 1, 2)]:
        def shifted(e, idx=idx):
            Xe = Xs.copy()
            Xe[idx] += e
            return f(sw2, sb2, Xe)

        fd = cd(shifted)
        assert abs(float(dX[idx]) - fd) <= 1e-5 * max(abs(fd), 1e-3 * abs(dX).max().item()), (idx, float(dX[idx]), fd)


def test_euler_identities():
    arch = Arch((2, 1, 1))
    rng = np.random.default_rng(12)
    x = torch.tensor(rng.standard_normal((8, 8, 3)), requires_grad=True)
    xp = torch.tensor(rng.standard_normal((8, 8, 3)))
    sw2 = torch.tensor(1.6, dtype=F64, requires_grad=True)
    qx = myrtle_self_q(arch, sw2, 0.0, x)
    qxp = myrtle_self_q(arch, sw2, 0.0, xp)
    K, _, _ = myrtle_layers_pair(arch, sw2, 0.0, x, xp, qx, qxp)
    K.backward()
    # degree 1 in x (q(x) scales as x^2 and the map is 1-homogeneous)
    assert abs(float((x.detach() * x.grad).sum()) - float(K.detach())) <= 1e-12 * abs(float(K.detach()))
    # degree L = #weight layers in sigma_w^2
    L = arch.n_weight_layers
    assert abs(float(sw2.grad) - L * float(K.detach()) / 1.6) <= 1e-12 * abs(float(K.detach()))


# --------------------------------------------------------------------------
# Partial pivoted Cholesky preconditioner (Section 2: the paper's own)
# --------------------------------------------------------------------------

def test_pivoted_cholesky_full_rank_is_exact(gram):
    from oracle import pivoted_cholesky

    K, _ = gram
    n = K.shape[0]
    L, piv = pivoted_cholesky(K, n)
    assert len(set(piv)) == len(piv)
    # the greedy factor of an SPD matrix reproduces it (up to where the
    # remaining diagonal vanishes at rounding level)
    assert np.abs(L.T @ L - K).max() <= 1e-9 * np.abs(K).max()


def test_pivoted_cholesky_pivots_are_greedy_schur_maxima(gram):
    """Each pivot is the argmax of the diagonal of the Schur complement of
    the previous pivots, computed here independently with a dense solve; the
    residual K - L^T L vanishes on the pivot rows (interpolation)."""
    from oracle import pivoted_cholesky

    K, _ = gram
    L, piv = pivoted_cholesky(K, 12)
    assert len(piv) == 12 and len(set(piv)) == 12
    for k in range(len(piv)):
        P = piv[:k]
        if k == 0:
            S = np.diag(K).copy()
        else:
            KP = K[np.ix_(P, P)]
            S = np.diag(K) - np.einsum("ij,ji->i", K[:, P], np.linalg.solve(KP, K[P, :]))
        assert int(np.argmax(S)) == piv[k]
    E = K - L.T @ L
    assert np.abs(E[piv, :]).max() <= 1e-10 * np.abs(K).max()
    # the remaining trace decreases with the rank
    tr = [np.trace(K - pivoted_cholesky(K, r)[0].T @ pivoted_cholesky(K, r)[0]) for r in (1, 4, 12)]
    assert tr[0] > tr[1] > tr[2] > 0


def test_pivoted_cholesky_stops_at_the_rank_of_a_rank_deficient_gram():
    """K = V^T V of r < n vectors has rank r: after r exact pivots the Schur
    complement is zero, and in float64 its computed diagonal is rounding noise
    (about k u max diag K after k steps).  The factor must stop at exactly r
    pivots and reproduce K; a stop rule of d > 0 would pivot on that noise
    (rank above r, rows divided by the square root of a rounding error), and
    a floor far above rounding would stop before r on a matrix whose last
    real pivot is small (second case: smallest pivot about 1e-9 of the
    largest diagonal, which must still be taken)."""
    from oracle import pivoted_cholesky

    rng = np.random.default_rng(12)
    n = 40
    for r in (1, 7, 25):
        V = rng.standard_normal((r, n))
        K = V.T @ V
        L, piv = pivoted_cholesky(K, n)
        assert len(piv) == r, (r, len(piv))
        assert np.isfinite(L).all()
        assert np.abs(L.T @ L - K).max() <= 1e-12 * np.abs(K).max()
    # full rank with one small direction: every one of the n pivots is real
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.ones(n)
    ev[-1] = 1e-9
    K = (Q * ev) @ Q.T
    L, piv = pivoted_cholesky(K, n)
    assert len(piv) == n
    assert np.abs(L.T @ L - K).max() <= 1e-12 * np.abs(K).max()


def test_pivchol_apply_is_the_woodbury_inverse(gram):
    from oracle import pivchol_apply, pivoted_cholesky

    K, Y = gram
    lam = 1e-3 * np.trace(K) / K.shape[0]
    L, _ = pivoted_cholesky(K, 7)
    M = L.T @ L + lam * np.eye(K.shape[0])
    want = np.linalg.solve(M, Y)
    assert np.allclose(pivchol_apply(L, lam, Y), want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
    assert np.allclose(pivchol_apply(L[:0], lam, Y), Y / lam)


def test_pivchol_pcg_converges_and_beats_jacobi(gram):
    K, Y = gram
    n = K.shape[0]
    lam = 1e-4 * np.trace(K) / n
    Astar = cholesky_solve(K, Y, lam)
    X, it_pc, rel = pcg(K, Y, lam, "pivchol", tol=1e-10, maxit=5000, rank=10)
    assert rel.max() <= 1e-10
    kappa = np.linalg.cond(K + lam * np.eye(n))
    assert np.linalg.norm(X - Astar) / np.linalg.norm(Astar) <= kappa * 1e-10
    _, it_j, _ = pcg(K, Y, lam, "jacobi", tol=1e-10, maxit=5000)
    assert it_pc < it_j
    # full rank: M = K + lam I, so CG needs a single step
    _, it_full, rel_full = pcg(K, Y, lam, "pivchol", tol=1e-8, maxit=50, rank=n)
    assert it_full <= 2 and rel_full.max() <= 1e-8
