"""The block store and the resumable solve with the real kernels: a
symmetric 32x32 kernel matrix computed as tiles by nk_block, interrupted and
resumed from disk, equals the single-call block; a PCG solve stopped after a
few iterations and resumed from its saved iterate (nk_pcg_set_warm_start)
reaches the same solution as a cold solve, for MIXED and PLAIN_FP64."""

import numpy as np
import pytest
import torch

import nkdata

pytestmark = pytest.mark.gpu

CONVS = (2, 1, 0)


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def test_block_store_resume_matches_one_block(h, tmp_path):
    from paper_2303_05420_gb300.store import BlockStore, nngp_tiles

    x = nkdata.standardise(nkdata.images(20, 32, 3, 31, blur=True))[0].astype(np.float32)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, CONVS, 2.0, 0.01)
    full = h.block(X, q, X, q, CONVS, 2.0, 0.01, symmetric=True).double().cpu().numpy()
    compute = nngp_tiles(h, X, q, CONVS, 2.0, 0.01)
    path = str(tmp_path / "k")
    assert BlockStore(path, 20, 20, 8, symmetric=True).run(compute, limit=2) == 2
    st = BlockStore(path, 20, 20, 8, symmetric=True)  # as after a restart
    assert st.run(compute) == 4
    K = st.assemble().astype(np.float64)
    assert float(np.max(np.abs(K - full) / np.abs(full))) <= 1e-6
    assert np.array_equal(K, K.T)


def _spd_problem(h, n=600, r=4):
    x = nkdata.fc_rows(n, 256, seed=41).astype(np.float32)
    X = torch.tensor(x, device="cuda")
    K = h.fc_block(X, X, 2.0, 0.01, depth=3, symmetric=True)
    Y = torch.tensor(np.random.default_rng(42).standard_normal((n, r)), device="cuda")
    return K, Y


@pytest.mark.parametrize("prec", ["mixed", "plain_fp64"])
def test_pcg_warm_start_resumes_a_stopped_solve(h, prec):
    K, Y = _spd_problem(h)
    lam = 1e-3
    A_ref, its_ref, rel_ref = h.pcg_solve(K, Y, lam, prec=prec, tol=1e-8)
    assert max(rel_ref) <= 1e-8
    A0, its0, rel0 = h.pcg_solve(K, Y, lam, prec=prec, tol=1e-8, maxit=5, allow_not_converged=True)
    assert max(rel0) > 1e-8
    h.pcg_set_warm_start(True)
    try:
        A1, its1, rel1 = h.pcg_solve(K, Y, lam, prec=prec, tol=1e-8, A=A0.clone())
        # from the exact solution: nothing left to do
        A2, its2, rel2 = h.pcg_solve(K, Y, lam, prec=prec, tol=1e-8, A=A_ref.clone())
    finally:
        h.pcg_set_warm_start(False)
    assert max(rel1) <= 1e-8
    assert its2 == 0 and max(rel2) <= 1e-8
    # both solutions solve the system to 1e-8; their difference is bounded by
    # the condition number times that
    diff = float((A1 - A_ref).norm() / A_ref.norm())
    assert diff <= 1e-4, diff


def test_solve_resumable_in_pieces(h, tmp_path):
    from paper_2303_05420_gb300.store import solve_resumable

    K, Y = _spd_problem(h)
    path = str(tmp_path / "A.npy")
    A, pieces, ok = solve_resumable(h, K, Y, 1e-3, path, piece_iters=6, max_pieces=2, tol=1e-8)
    assert not ok and pieces == 2
    A, more, ok = solve_resumable(h, K, Y, 1e-3, path, piece_iters=40, tol=1e-8)
    assert ok
    A_ref, _, _ = h.pcg_solve(K, Y, 1e-3, tol=1e-8)
    assert float((A - A_ref).norm() / A_ref.norm()) <= 1e-4
