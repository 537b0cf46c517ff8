"""GPU parity: libnk (through the C ABI) against the float64 CPU oracle.

Tolerances: kernel entries within 1e-5 max-relative for the FP32 / MIXED paths
and 1e-12 for PLAIN_FP64; self-variances within 1e-12 relative (FP64 on both
sides); PCG to relative residual 1e-6 and against a Cholesky solve.  Inputs
are the same seeded float32 images on both sides (the oracle upcasts them).
"""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, hw, seed, blur=True):
    x = nkdata.images(n, hw, 3, seed, blur)
    x = nkdata.standardise(x)[0]
    return x.astype(np.float32)


def _dev(x):
    return torch.tensor(x, device="cuda")


def _oracle_block(convs, sw2, sb2, xa, xb, symmetric=False, pairs=None):
    return oracle.myrtle_block(oracle.Arch(convs), sw2, sb2, xa.astype(np.float64),
                               xb.astype(np.float64), symmetric=symmetric, pairs=pairs).numpy()


def _maxrel(got, want):
    mask = ~np.isnan(want)
    return float(np.max(np.abs(got[mask] - want[mask]) / np.abs(want[mask])))


@pytest.mark.parametrize("hw,convs", [(8, (2, 1, 0)), (8, (3, 3, 3)), (16, (2, 1, 1)), (32, (2, 1, 0))])
def test_self_diag_matches_oracle(h, hw, convs):
    x = _imgs(3, hw, 0)
    qd, qs = h.self_diag(_dev(x), convs, 2.0, 0.01)
    h.sync_status()
    qd = qd.cpu().numpy()
    qs = qs.cpu().numpy()
    for n in range(3):
        want = np.concatenate([q.numpy().reshape(-1) for q in
                               oracle.myrtle_self_q(oracle.Arch(convs), 2.0, 0.01,
                                                    torch.tensor(x[n].astype(np.float64)))])
        assert np.allclose(qd[n], want, rtol=1e-12, atol=0)
        assert np.allclose(qs[n, :, 1], np.sqrt(want), rtol=1e-6)
        assert np.allclose(qs[n, :, 0], 1 / np.sqrt(want), rtol=1e-6)


@pytest.mark.parametrize("hw,convs,sb2", [(8, (2, 1, 0), 0.0), (8, (3, 3, 3), 0.01), (8, (1,), 0.1),
                                          (16, (2, 1, 0), 0.0), (16, (2, 1, 1), 0.01),
                                          (8, (1, 1, 1), 0.05)])
@pytest.mark.parametrize("prec", ["mixed", "plain_fp32", "plain_fp64"])
def test_block_small_matches_oracle(h, hw, convs, sb2, prec):
    xa = _imgs(7, hw, 0)
    xb = _imgs(5, hw, 1)
    Xa, Xb = _dev(xa), _dev(xb)
    qa = h.self_diag(Xa, convs, 2.0, sb2)
    qb = h.self_diag(Xb, convs, 2.0, sb2)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec)
    Ks = h.block(Xa, qa, Xa, qa, convs, 2.0, sb2, prec=prec, symmetric=True)
    h.sync_status()
    want = _oracle_block(convs, 2.0, sb2, xa, xb)
    wants = _oracle_block(convs, 2.0, sb2, xa, xa, symmetric=True)
    tol = 1e-12 if prec == "plain_fp64" else TOL32
    assert _maxrel(K.double().cpu().numpy(), want) <= tol
    assert _maxrel(Ks.double().cpu().numpy(), wants) <= tol


def test_block_ragged_ranges_and_ldk(h):
    convs = (2, 1, 0)
    x = _imgs(11, 8, 2)
    X = _dev(x)
    q = h.self_diag(X, convs, 2.0, 0.0)
    out = torch.full((5, 9), float("nan"), device="cuda")
    h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", a_range=(3, 8), b_range=(2, 8), out=out[:, :6])
    sym = torch.full((7, 7), float("nan"), device="cuda")
    h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", a_range=(4, 11), b_range=(4, 11), symmetric=True,
            out=sym)
    h.sync_status()
    want = _oracle_block(convs, 2.0, 0.0, x[3:8], x[2:8])
    got = out.cpu().numpy()
    assert _maxrel(got[:, :6], want) <= TOL32
    assert np.isnan(got[:, 6:]).all()  # beyond the block: untouched
    wants = _oracle_block(convs, 2.0, 0.0, x[4:11], x[4:11], symmetric=True)
    assert _maxrel(sym.cpu().numpy(), wants) <= TOL32


def test_block_empty_and_invalid(h):
    from paper_2303_05420_gb300._lib import NkError

    convs = (2, 1, 0)
    X = _dev(_imgs(4, 8, 0))
    q = h.self_diag(X, convs, 2.0, 0.0)
    out = torch.zeros((1, 1), device="cuda")
    h.block(X, q, X, q, convs, 2.0, 0.0, a_range=(2, 2), b_range=(0, 1), out=out[:0])
    with pytest.raises(NkError):  # symmetric with different ranges
        h.block(X, q, X, q, convs, 2.0, 0.0, a_range=(0, 2), b_range=(1, 3), symmetric=True)
    with pytest.raises(NkError):  # unsupported fused shape (12x12)
        Y = _dev(_imgs(2, 12, 0))
        qy = h.self_diag(Y, convs, 2.0, 0.0)
        h.block(Y, qy, Y, qy, convs, 2.0, 0.0, prec="mixed")


@pytest.mark.parametrize("convs,sb2", [((2, 1, 0), 0.0), ((2, 1, 0), 0.01), ((3, 3, 3), 0.01), ((2, 1, 1), 0.0),
                                       ((1,), 0.1)])
def test_block_32x32_sampled_pairs(h, convs, sb2):
    """(2,1,0) and (1) run the tiled form at 32x32 by default ((1): its
    single-stage path, the global average taken in the stage-0 tasks), the
    others the cluster kernel; sb2 > 0 takes the kernels' bias branch."""
    xa = _imgs(6, 32, 0)
    xb = _imgs(4, 32, 1)
    Xa, Xb = _dev(xa), _dev(xb)
    qa = h.self_diag(Xa, convs, 2.0, sb2)
    qb = h.self_diag(Xb, convs, 2.0, sb2)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec="mixed")
    h.sync_status()
    pairs = [(0, 0), (1, 3), (5, 2), (3, 1)]
    want = _oracle_block(convs, 2.0, sb2, xa, xb, pairs=pairs)
    assert _maxrel(K.cpu().numpy().astype(np.float64), want) <= TOL32


def test_pcg_matches_cholesky(h):
    p = nkdata.image_problem(128, 32, 8, n_classes=10, blur=False)
    x = p.x_train.astype(np.float32)
    X = _dev(x)
    convs = (2, 1, 0)
    q = h.self_diag(X, convs, 2.0, 0.0)
    K = h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", symmetric=True)
    Kh = K.double().cpu().numpy()
    lam = 1e-4 * np.trace(Kh) / Kh.shape[0]
    Y = torch.tensor(p.y_train, device="cuda")
    Astar = oracle.cholesky_solve(Kh, p.y_train, lam)
    for prec in ["mixed", "plain_fp64"]:
        tol = 1e-6
        A, its, rel = h.pcg_solve(K, Y, lam, precond="jacobi", prec=prec, tol=tol, maxit=5000)
        assert max(rel) <= tol, (prec, rel)
        An = A.cpu().numpy()
        r = p.y_train - (Kh + lam * np.eye(len(Kh))) @ An
        assert np.linalg.norm(r, axis=0).max() / np.linalg.norm(p.y_train, axis=0).min() <= 2 * tol
        kappa = np.linalg.cond(Kh + lam * np.eye(len(Kh)))
        assert np.linalg.norm(An - Astar) / np.linalg.norm(Astar) <= kappa * tol
        assert its > 0
    # FP32 products alone stall well above 1e-6 on this ill-conditioned system
    # (Section 2: float32 degrades the solve); the solver must say so
    # rather than claim convergence, and its iterate is still a usable
    # ("anytime") approximation.
    A, its, rel = h.pcg_solve(K, Y, lam, precond="jacobi", prec="plain_fp32", tol=1e-6, maxit=400,
                              allow_not_converged=True)
    r_true = p.y_train - (Kh + lam * np.eye(len(Kh))) @ A.cpu().numpy()
    rel_true = np.linalg.norm(r_true, axis=0) / np.linalg.norm(p.y_train, axis=0)
    assert np.allclose(rel_true, rel, rtol=1e-3)
    assert max(rel) < 0.5


@pytest.mark.parametrize("n,R", [(300, 17), (1000, 10), (37, 1)])
def test_pcg_forms_many_columns(h, n, R):
    """Every precision form on a ragged size with R > 16 (two column groups of
    the matvec) and iteration counts that are not a multiple of the captured
    block; the mixed form's refinement sweeps cost at most a few times the
    FP64 form's iterations."""
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n + 5))
    Kh = (B @ B.T / n).astype(np.float32)
    Kd = Kh.astype(np.float64)
    lam = 1e-3 * np.trace(Kd) / n
    Yh = rng.standard_normal((n, R))
    K = torch.tensor(Kh, device="cuda")
    Y = torch.tensor(Yh, device="cuda")
    want = np.linalg.solve(Kd + lam * np.eye(n), Yh)
    its_by = {}
    for prec in ["plain_fp64", "mixed"]:
        A, its, rel = h.pcg_solve(K, Y, lam, precond="jacobi", prec=prec, tol=1e-8, maxit=5000)
        r = Yh - (Kd + lam * np.eye(n)) @ A.cpu().numpy()
        rel_true = np.linalg.norm(r, axis=0) / np.linalg.norm(Yh, axis=0)
        assert rel_true.max() <= 1e-8, (prec, rel_true.max())
        assert np.allclose(rel_true, rel, rtol=1e-3, atol=1e-12)
        kappa = np.linalg.cond(Kd + lam * np.eye(n))
        assert np.linalg.norm(A.cpu().numpy() - want) <= kappa * 1e-8 * np.linalg.norm(want)
        its_by[prec] = its
    assert its_by["mixed"] <= 4 * its_by["plain_fp64"] + 16, its_by


@pytest.mark.parametrize("rank", [10, 40, 128])
def test_pcg_pivchol_matches_cholesky_and_oracle(h, rank):
    """Section 2's partial pivoted Cholesky preconditioner: the solve reaches
    1e-6 against Cholesky in both precisions; the FP64 form takes the
    oracle's iteration count (same greedy pivots and Woodbury apply); at full
    rank M = K + lambda I and one or two steps suffice."""
    p = nkdata.image_problem(128, 32, 8, n_classes=10, blur=False)
    X = _dev(p.x_train.astype(np.float32))
    convs = (2, 1, 0)
    q = h.self_diag(X, convs, 2.0, 0.0)
    K = h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", symmetric=True)
    Kh = K.double().cpu().numpy()
    lam = 1e-4 * np.trace(Kh) / Kh.shape[0]
    Y = torch.tensor(p.y_train, device="cuda")
    Astar = oracle.cholesky_solve(Kh, p.y_train, lam)
    kappa = np.linalg.cond(Kh + lam * np.eye(len(Kh)))
    _, it_or, _ = oracle.pcg(Kh, p.y_train, lam, "pivchol", tol=1e-6, maxit=5000, rank=rank)
    h.pcg_set_rank(rank)
    try:
        for prec in ["plain_fp64", "mixed"]:
            A, its, rel = h.pcg_solve(K, Y, lam, precond="pivchol", prec=prec, tol=1e-6, maxit=5000)
            An = A.cpu().numpy()
            r = p.y_train - (Kh + lam * np.eye(len(Kh))) @ An
            rel_true = np.linalg.norm(r, axis=0) / np.linalg.norm(p.y_train, axis=0)
            assert rel_true.max() <= 1e-6, (prec, rel_true.max())
            # residuals far below tol are compared at the level of their own rounding
            assert np.allclose(rel_true, rel, rtol=1e-3, atol=1e-9)
            assert np.linalg.norm(An - Astar) / np.linalg.norm(Astar) <= kappa * 1e-6
            if prec == "plain_fp64":
                assert abs(its - it_or) <= 2 + it_or // 10, (its, it_or)
                if rank == 128:
                    assert its <= 2
    finally:
        h.pcg_set_rank(100)


def test_pcg_not_converged_and_edge(h):
    from paper_2303_05420_gb300._lib import NK_ERR_NOT_CONVERGED, NkError

    n = 64
    rng = np.random.default_rng(0)
    B = rng.standard_normal((n, n))
    Kh = (B @ B.T / n).astype(np.float32)
    K = torch.tensor(Kh, device="cuda")
    Y = torch.tensor(rng.standard_normal((n, 3)), device="cuda")
    with pytest.raises(NkError) as ei:
        h.pcg_solve(K, Y, 1e-8, prec="plain_fp64", tol=1e-12, maxit=2)
    assert ei.value.status == NK_ERR_NOT_CONVERGED
    A, its, rel = h.pcg_solve(K, Y, 1.0, prec="plain_fp64", tol=1e-10, maxit=500)
    want = np.linalg.solve(Kh.astype(np.float64) + np.eye(n), Y.cpu().numpy())
    assert np.allclose(A.cpu().numpy(), want, rtol=1e-8, atol=1e-10)


def test_autotune_variants_agree(h):
    """Every launch variant the autotuner may pick computes the same block."""
    from paper_2303_05420_gb300._lib import NkError

    x = _imgs(6, 32, 4)
    X = _dev(x)
    # (2,1,0) and (3,3,3) have the three cluster launches and the tiled form
    # (3); (1,1,1) the cluster launches only
    for convs, sb2, nvar in [((2, 1, 0), 0.0, 4), ((3, 3, 3), 0.01, 4), ((1, 1, 1), 0.0, 3)]:
        q = h.self_diag(X, convs, 2.0, sb2)
        chosen = h.autotune(convs, 2.0, sb2, 32, 32, 3)
        assert 0 <= chosen < nvar
        ref = _oracle_block(convs, 2.0, sb2, x[:3], x[3:])
        for v in range(nvar):
            h.autotune_set(convs, 2.0, sb2, 32, 32, v)
            K = h.block(X, q, X, q, convs, 2.0, sb2, prec="mixed", a_range=(0, 3), b_range=(3, 6))
            h.sync_status()
            assert _maxrel(K.double().cpu().numpy(), ref) <= TOL32, v
        h.autotune_set(convs, 2.0, sb2, 32, 32, chosen)
    with pytest.raises(NkError):
        h.autotune_set((2, 1, 0), 2.0, 0.0, 32, 32, 4)
    with pytest.raises(NkError):
        h.autotune_set((1, 1, 1), 2.0, 0.0, 32, 32, 3)


@pytest.mark.parametrize("precond", ["none", "jacobi", "pivchol"])
@pytest.mark.parametrize("prec", ["plain_fp64", "plain_fp32", "mixed"])
def test_pcg_degenerate_cases(h, precond, prec):
    """N = 1; a zero right-hand side next to a non-zero one; K with a leading
    dimension larger than N; maxit = 0."""
    from paper_2303_05420_gb300._lib import NK_ERR_NOT_CONVERGED, NkError

    K = torch.tensor([[2.0]], device="cuda")
    Y = torch.tensor([[4.0]], dtype=torch.float64, device="cuda")
    A, its, rel = h.pcg_solve(K, Y, 2.0, precond=precond, prec=prec, tol=1e-10, maxit=10)
    assert abs(float(A[0, 0]) - 1.0) <= 1e-6 and rel[0] <= 1e-10
    n = 37
    rng = np.random.default_rng(5)
    B = rng.standard_normal((n, n))
    Kh = (B @ B.T / n + np.eye(n)).astype(np.float32)
    Kbig = torch.zeros((n, n + 11), device="cuda")
    Kbig[:, :n] = torch.tensor(Kh, device="cuda")
    Kv = Kbig[:, :n]  # leading dimension n + 11
    Yh = np.stack([rng.standard_normal(n), np.zeros(n)], axis=1)
    Y2 = torch.tensor(Yh, device="cuda")
    tol = 1e-6 if prec == "plain_fp32" else 1e-9
    A, its, rel = h.pcg_solve(Kv, Y2, 0.5, precond=precond, prec=prec, tol=tol, maxit=500)
    want = np.linalg.solve(Kh.astype(np.float64) + 0.5 * np.eye(n), Yh)
    assert np.allclose(A.cpu().numpy(), want, rtol=0, atol=20 * tol * np.abs(want).max())
    assert rel[1] == 0.0 and float(A[:, 1].abs().max()) == 0.0
    with pytest.raises(NkError) as ei:
        h.pcg_solve(Kv, Y2, 0.5, precond=precond, prec=prec, tol=1e-9, maxit=0)
    assert ei.value.status == NK_ERR_NOT_CONVERGED


def test_pcg_rejects_bad_arguments(h):
    import ctypes

    from paper_2303_05420_gb300._lib import NK_ERR_INVALID_ARG, lib

    K = torch.eye(4, device="cuda")
    Y = torch.ones((4, 1), dtype=torch.float64, device="cuda")
    A = torch.empty_like(Y)
    its = ctypes.c_int(0)
    rel = (ctypes.c_double * 1)()

    def call(N=4, ldk=4, R=1, lam=1.0, precond=1, prec=2, tol=1e-6, maxit=10, refine=4):
        return lib().nk_pcg_solve(h._h, ctypes.c_void_p(K.data_ptr()), ldk, N, ctypes.c_void_p(Y.data_ptr()), R,
                                  lam, precond, prec, tol, maxit, refine, ctypes.c_void_p(A.data_ptr()),
                                  ctypes.byref(its), ctypes.cast(rel, ctypes.c_void_p), None)

    assert call() == 0
    for kw in [dict(N=-1), dict(ldk=3), dict(R=-2), dict(R=257), dict(lam=float("nan")), dict(precond=3),
               dict(prec=5), dict(tol=-1.0), dict(maxit=-1), dict(refine=-1)]:
        assert call(**kw) == NK_ERR_INVALID_ARG, kw
    assert call(N=0) == 0 and call(R=0) == 0
    from paper_2303_05420_gb300._lib import NkError

    with pytest.raises(NkError):
        h.pcg_set_rank(0)


def test_pcg_out_of_core_host_K(h):
    """K in pinned host memory, read by the kernels directly (out of core):
    the same solution as with K in HBM, for the Jacobi and pivoted Cholesky
    preconditioners.  The CG inner products accumulate with FP64 atomics, so
    two solves round differently; each stops at relative residual <= tol, so
    each lies within cond(K + lam I) * tol of the exact FP64 solution (per
    column, relative), and the two within twice that of each other."""
    n = 1536
    tol = 1e-8
    rng = np.random.default_rng(8)
    B = rng.standard_normal((n, n + 32)).astype(np.float32)
    Kh = (B @ B.T / n).astype(np.float32)
    Kdev = torch.tensor(Kh, device="cuda")
    Khost = torch.tensor(Kh).pin_memory()
    Yh = rng.standard_normal((n, 4))
    Y = torch.tensor(Yh, device="cuda")
    K64 = Kh.astype(np.float64)
    lam = 1e-3 * np.trace(K64) / n
    w = np.linalg.eigvalsh(K64)
    kappa = (w.max() + lam) / (w.min() + lam)
    Astar = np.linalg.solve(K64 + lam * np.eye(n), Yh)
    colrel = lambda A, Bm: np.linalg.norm(A - Bm, axis=0) / np.linalg.norm(Bm, axis=0)  # noqa: E731
    for pc in ["jacobi", "pivchol"]:
        Ad, itd, reld = h.pcg_solve(Kdev, Y, -1e-3, precond=pc, prec="mixed", tol=tol, maxit=5000)
        Ah, ith, relh = h.pcg_solve(Khost, Y, -1e-3, precond=pc, prec="mixed", tol=tol, maxit=5000)
        assert max(relh) <= tol and max(reld) <= tol
        # the rounding order also moves the refinement restarts by a few iterations
        assert abs(ith - itd) <= max(2, 0.02 * itd)
        Ad, Ah = Ad.cpu().numpy(), Ah.cpu().numpy()
        assert colrel(Ah, Astar).max() <= kappa * tol
        assert colrel(Ad, Astar).max() <= kappa * tol
        assert colrel(Ah, Ad).max() <= 2 * kappa * tol
