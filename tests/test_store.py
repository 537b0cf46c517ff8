"""Host logic of the preemption-safe block store (paper_2303_05420_gb300.store):
tiles written by rename and then marked done, a resume that computes only the
unmarked tiles, a process killed mid-run, and assembly of symmetric and
rectangular matrices.  A deterministic function stands in for the kernel
block, so no GPU is needed."""

import multiprocessing as mp
import os
import time

import numpy as np
import pytest

from paper_2303_05420_gb300.store import BlockStore


def _value(i, j):
    return np.sin(0.37 * i + 0.11) * np.cos(0.23 * j - 0.5) + 0.01 * (i + j)


def _want(n, m, symmetric):
    i, j = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    K = _value(i, j)
    if symmetric:
        K = np.triu(K) + np.triu(K, 1).T
    return K.astype(np.float32)


class Counter:
    def __init__(self, fail_after=None, delay=0.0):
        self.calls, self.fail_after, self.delay = [], fail_after, delay

    def __call__(self, r0, r1, c0, c1, diagonal):
        if self.fail_after is not None and len(self.calls) >= self.fail_after:
            raise RuntimeError("interrupted")
        self.calls.append((r0, c0))
        time.sleep(self.delay)
        i, j = np.meshgrid(np.arange(r0, r1), np.arange(c0, c1), indexing="ij")
        K = _value(i, j)
        if diagonal:
            K = np.where(i <= j, K, np.nan)  # a diagonal tile's lower triangle is not used
        return K


@pytest.mark.parametrize("n,m,block,sym", [(23, 23, 5, True), (17, 30, 8, False), (8, 8, 8, True),
                                           (1, 9, 4, False)])
def test_store_assembles_the_matrix(tmp_path, n, m, block, sym):
    st = BlockStore(str(tmp_path / "k"), n, m, block, symmetric=sym)
    c = Counter()
    assert st.run(c) == len(list(st.tiles()))
    np.testing.assert_array_equal(st.assemble(), _want(n, m, sym))


def test_store_resumes_only_missing_tiles(tmp_path):
    n, block = 40, 8  # 15 upper-triangle tiles
    path = str(tmp_path / "k")
    st = BlockStore(path, n, n, block, symmetric=True)
    with pytest.raises(RuntimeError):
        st.run(Counter(fail_after=6))
    assert int(BlockStore(path, n, n, block, symmetric=True).done.sum()) == 6
    # a fresh object on the same directory, as after a restart
    st2 = BlockStore(path, n, n, block, symmetric=True)
    c = Counter()
    assert st2.run(c) == 9
    done_first = {st.bounds(t)[0::2] for t in list(st.tiles())[:6]}
    assert not done_first & set(c.calls)
    np.testing.assert_array_equal(st2.assemble(), _want(n, n, True))
    # an unfinished temporary file from a kill is ignored
    open(os.path.join(path, "tile_0_0.npy.tmp.npy"), "wb").write(b"partial")
    np.testing.assert_array_equal(BlockStore(path, n, n, block, symmetric=True).assemble(), _want(n, n, True))


def _child(path):
    BlockStore(path, 48, 48, 8, symmetric=True).run(Counter(delay=0.2))


def test_store_survives_a_killed_process(tmp_path):
    path = str(tmp_path / "k")
    ctx = mp.get_context("spawn")
    p = ctx.Process(target=_child, args=(path,))
    p.start()
    done_path = os.path.join(path, "done.npy")
    t0 = time.time()
    while time.time() - t0 < 60:
        if os.path.exists(done_path) and np.load(done_path).sum() >= 3:
            break
        time.sleep(0.05)
    p.kill()
    p.join()
    st = BlockStore(path, 48, 48, 8, symmetric=True)
    done = int(st.done.sum())
    assert 3 <= done < 21
    c = Counter()
    assert st.run(c) == 21 - done
    np.testing.assert_array_equal(st.assemble(), _want(48, 48, True))


def test_store_refuses_another_shape(tmp_path):
    path = str(tmp_path / "k")
    BlockStore(path, 10, 10, 4, symmetric=True)
    with pytest.raises(ValueError):
        BlockStore(path, 10, 12, 4)
    with pytest.raises(RuntimeError):
        BlockStore(path, 10, 10, 4, symmetric=True).assemble()


class _RichardsonHandle:
    """Stands in for Handle's PCG calls: maxit Richardson steps on
    (K + lam I) A = Y from the A it is given when warm start is on (from zero
    otherwise), relres per column."""

    def __init__(self):
        self.warm, self.starts = False, []

    def pcg_set_warm_start(self, on):
        self.warm = bool(on)

    def pcg_solve(self, K, Y, lam, A=None, maxit=100, allow_not_converged=False, tol=1e-6):
        import torch

        M = K + lam * torch.eye(K.shape[0], dtype=K.dtype)
        w = 1.0 / float(torch.linalg.matrix_norm(M, 2))
        X = A.clone() if self.warm else torch.zeros_like(Y)
        self.starts.append(X.clone())
        its = 0
        for its in range(1, maxit + 1):
            X = X + w * (Y - M @ X)
            rel = ((Y - M @ X).norm(dim=0) / Y.norm(dim=0)).tolist()
            if max(rel) <= tol:
                break
        A.copy_(X)
        return A, its, rel


def test_solve_resumable_saves_each_piece_and_resumes(tmp_path):
    import torch

    from paper_2303_05420_gb300.store import solve_resumable

    rng = np.random.default_rng(3)
    G = rng.standard_normal((6, 6))
    K = torch.tensor(G @ G.T / 6 + 0.5 * np.eye(6))
    Y = torch.tensor(rng.standard_normal((6, 2)))
    lam, path = 0.1, str(tmp_path / "A.npy")
    h = _RichardsonHandle()
    A1, pieces, ok = solve_resumable(h, K, Y, lam, path, piece_iters=5, max_pieces=2, tol=1e-10)
    assert (pieces, ok) == (2, False) and not h.warm
    saved = np.load(path)
    assert np.array_equal(saved, A1.numpy())
    # each piece starts from the previous one's iterate
    assert torch.equal(h.starts[0], torch.zeros_like(Y)) and not torch.equal(h.starts[1], h.starts[0])
    h2 = _RichardsonHandle()
    A2, pieces2, ok2 = solve_resumable(h2, K, Y, lam, path, piece_iters=50, max_pieces=1000, tol=1e-10)
    assert ok2 and not h2.warm
    assert np.array_equal(h2.starts[0].numpy(), saved)  # a restart resumes from the saved iterate
    want = torch.linalg.solve(K + lam * torch.eye(6, dtype=K.dtype), Y)
    assert float((A2 - want).abs().max() / want.abs().max()) <= 1e-8
    assert np.array_equal(np.load(path), A2.numpy())
    with pytest.raises(ValueError):
        solve_resumable(h2, K, Y, lam, path, maxit=10)
