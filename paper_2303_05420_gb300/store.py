"""Preemption-safe computation of a kernel matrix and its ridge solve.

The paper computes the kernel matrix as independent blocks of its upper
triangle (Figure 1), stores them on disk, and notes that with so little
coordination the routines are easy to make preemption-safe (Section 2).
`BlockStore` keeps that contract on one machine: the matrix is cut into
tiles, each tile is computed by a caller-supplied function (normally a
kernel block through `Handle.block`), written to its own ``.npy`` file, and
only then marked in a done bitmap; both writes go to a temporary file that
is renamed into place, so a process killed at any point leaves a store in
which every tile marked done is complete.  `run` computes the tiles that are
not marked (a tile in flight at the kill is computed again), `assemble`
returns the matrix.  `solve_resumable` runs the PCG solve in bounded pieces,
saving the iterate after each and restarting from it (the solver's warm
start), so an interrupted solve resumes from its last saved iterate.
"""

import json
import os
from typing import Callable, Iterator, List, Optional, Tuple

import numpy as np

Tile = Tuple[int, int]


def _save_atomic(path: str, arr: np.ndarray) -> None:
    tmp = path + ".tmp.npy"
    np.save(tmp, arr)
    os.replace(tmp, path)


class BlockStore:
    """Tiles of an n_rows x n_cols kernel matrix under directory `path`.

    block: tile side.  symmetric: the matrix is K(X, X) (n_rows == n_cols);
    only tiles on or above the diagonal are computed and the lower triangle
    is mirrored in `assemble`.  Reopening a directory checks that its shape
    matches."""

    def __init__(self, path: str, n_rows: int, n_cols: int, block: int, symmetric: bool = False,
                 dtype=np.float32):
        if block < 1 or n_rows < 0 or n_cols < 0:
            raise ValueError("bad store shape")
        if symmetric and n_rows != n_cols:
            raise ValueError("a symmetric store is square")
        self.path, self.n_rows, self.n_cols, self.block = path, n_rows, n_cols, block
        self.symmetric, self.dtype = symmetric, np.dtype(dtype)
        self.nbi = -(-n_rows // block)
        self.nbj = -(-n_cols // block)
        os.makedirs(path, exist_ok=True)
        meta = {"n_rows": n_rows, "n_cols": n_cols, "block": block, "symmetric": bool(symmetric),
                "dtype": self.dtype.str}
        mpath = os.path.join(path, "meta.json")
        if os.path.exists(mpath):
            with open(mpath) as f:
                if json.load(f) != meta:
                    raise ValueError(f"{path} holds a store of another shape")
        else:
            tmp = mpath + ".tmp"
            with open(tmp, "w") as f:
                json.dump(meta, f)
            os.replace(tmp, mpath)
        self._done_path = os.path.join(path, "done.npy")
        if os.path.exists(self._done_path):
            self.done = np.load(self._done_path)
        else:
            self.done = np.zeros((self.nbi, self.nbj), dtype=np.uint8)

    def tiles(self) -> Iterator[Tile]:
        for bi in range(self.nbi):
            for bj in range(bi if self.symmetric else 0, self.nbj):
                yield bi, bj

    def bounds(self, t: Tile) -> Tuple[int, int, int, int]:
        bi, bj = t
        b = self.block
        return bi * b, min((bi + 1) * b, self.n_rows), bj * b, min((bj + 1) * b, self.n_cols)

    def missing(self) -> List[Tile]:
        return [t for t in self.tiles() if not self.done[t]]

    def _tile_path(self, t: Tile) -> str:
        return os.path.join(self.path, f"tile_{t[0]}_{t[1]}.npy")

    def run(self, compute: Callable[[int, int, int, int, bool], np.ndarray], limit: Optional[int] = None) -> int:
        """Computes the missing tiles in order (at most `limit`) and returns
        how many.  compute(r0, r1, c0, c1, diagonal) returns the tile
        K[r0:r1, c0:c1]; `diagonal` is true for a diagonal tile of a
        symmetric store (its lower triangle may be left unset)."""
        n = 0
        for t in self.missing():
            if limit is not None and n >= limit:
                break
            r0, r1, c0, c1 = self.bounds(t)
            diag = self.symmetric and t[0] == t[1]
            k = np.asarray(compute(r0, r1, c0, c1, diag), dtype=self.dtype)
            if k.shape != (r1 - r0, c1 - c0):
                raise ValueError(f"tile {t}: compute returned {k.shape}, expected {(r1 - r0, c1 - c0)}")
            _save_atomic(self._tile_path(t), k)
            self.done[t] = 1
            _save_atomic(self._done_path, self.done)
            n += 1
        return n

    def complete(self) -> bool:
        return not self.missing()

    def assemble(self) -> np.ndarray:
        if not self.complete():
            raise RuntimeError(f"{len(self.missing())} tiles missing")
        K = np.zeros((self.n_rows, self.n_cols), dtype=self.dtype)
        for t in self.tiles():
            r0, r1, c0, c1 = self.bounds(t)
            k = np.load(self._tile_path(t))
            if self.symmetric and t[0] == t[1]:
                iu = np.triu_indices(r1 - r0)
                K[r0:r1, c0:c1][iu] = k[iu]
            else:
                K[r0:r1, c0:c1] = k
        if self.symmetric:
            il = np.tril_indices(self.n_rows, -1)
            K[il] = K.T[il]
        return K


def nngp_tiles(handle, Xa, qa, convs, sw2: float, sb2: float, Xb=None, qb=None, **block_kw):
    """compute(r0, r1, c0, c1, diagonal) for BlockStore.run by nk_block
    (MIXED unless block_kw says otherwise): K(Xa[r0:r1], Xb[c0:c1]), or
    K(Xa, Xa) for a symmetric store (diagonal tiles as symmetric blocks)."""
    Xb = Xa if Xb is None else Xb
    qb = qa if qb is None else qb

    def compute(r0, r1, c0, c1, diagonal):
        if diagonal:
            K = handle.block(Xa, qa, Xa, qa, convs, sw2, sb2, a_range=(r0, r1), b_range=(c0, c1), symmetric=True,
                             **block_kw)
        else:
            K = handle.block(Xa, qa, Xb, qb, convs, sw2, sb2, a_range=(r0, r1), b_range=(c0, c1), **block_kw)
        handle.sync_status()
        return K.cpu().numpy()

    return compute


def solve_resumable(handle, K, Y, lam: float, path: str, piece_iters: int = 200, max_pieces: int = 100,
                    **solve_kw):
    """(K + lam I) A = Y by nk_pcg_solve in pieces of at most piece_iters
    iterations, saving A to `path` (.npy) after each piece and starting each
    piece, and a restarted call, from the saved A (nk_pcg_set_warm_start).
    Returns (A, pieces run by this call, converged)."""
    import torch

    if "maxit" in solve_kw:
        raise ValueError("solve_resumable bounds each piece by piece_iters; pass no maxit")
    A = torch.zeros_like(Y)
    if os.path.exists(path):
        A.copy_(torch.from_numpy(np.load(path)).to(Y.device))
    handle.pcg_set_warm_start(True)
    try:
        for piece in range(max_pieces):
            A, its, rel = handle.pcg_solve(K, Y, lam, A=A, maxit=piece_iters, allow_not_converged=True,
                                           **solve_kw)
            _save_atomic(path, A.cpu().numpy())
            tol = solve_kw.get("tol", 1e-6)
            if max(rel) <= tol:
                return A, piece + 1, True
        return A, max_pieces, False
    finally:
        handle.pcg_set_warm_start(False)
