"""Python API over libnk: torch tensors in, torch tensors out.

PyTorch supplies device memory and the current CUDA stream; the computation
is libnk's.  Names follow the C ABI (include/nk.h): ``self_diag``, ``block``,
``pcg_solve``.
"""

from __future__ import annotations

import ctypes
from ctypes import byref, c_int, c_void_p
from typing import Optional, Sequence, Tuple

import torch

from . import _lib
from ._lib import NkError, lib, make_arch, make_params


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ranges(Xa: torch.Tensor, Xb: torch.Tensor, a_range, b_range) -> Tuple[int, int, int, int]:
    """Index ranges of a block, checked against the image tensors (the C ABI
    takes plain pointers and cannot check them)."""
    a0, a1 = a_range if a_range is not None else (0, Xa.shape[0])
    b0, b1 = b_range if b_range is not None else (0, Xb.shape[0])
    if not (0 <= a0 <= a1 <= Xa.shape[0] and 0 <= b0 <= b1 <= Xb.shape[0]):
        raise ValueError(f"block ranges [{a0}, {a1}) x [{b0}, {b1}) outside {Xa.shape[0]} x {Xb.shape[0]} images")
    return int(a0), int(a1), int(b0), int(b1)


class Handle:
    """Owns an nk_handle (workspace, device status word)."""

    def __init__(self):
        self._h = c_void_p()
        st = lib().nk_create(byref(self._h))
        if st != 0:
            raise NkError(st, lib().nk_status_string(st).decode())

    def close(self):
        if self._h:
            lib().nk_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int, what: str):
        if st != 0:
            buf = ctypes.create_string_buffer(512)
            lib().nk_last_error(self._h, buf, 512)
            raise NkError(st, f"{what}: {buf.value.decode()}")

    def launch_count(self) -> int:
        return int(lib().nk_launch_count(self._h))

    def last_lambda(self) -> float:
        return float(lib().nk_last_lambda(self._h))

    def sync_status(self):
        self.check(lib().nk_sync_status(self._h, c_void_p(_stream())), "nk_sync_status")

    # ------------------------------------------------------------------
    def q_size(self, convs: Sequence[int], H: int, W: int, filt: int = 3) -> int:
        a = make_arch(convs, filt)
        return int(lib().nk_q_size(byref(a), H, W))

    def self_diag(self, X: torch.Tensor, convs: Sequence[int], sw2: float, sb2: float,
                  filt: int = 3, act: str = "relu", norm: str = "none") -> Tuple[torch.Tensor, torch.Tensor]:
        """X [n, H, W, C] float32 CUDA -> (qd [n, nq] float64, qs [n, nq, 2] float32)."""
        assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
        n, H, W, C = X.shape
        a = make_arch(convs, filt, act, norm)
        p = make_params(sw2, sb2)
        nq = int(lib().nk_q_size(byref(a), H, W))
        if nq < 0:
            raise NkError(_lib.NK_ERR_INVALID_ARG, "invalid architecture / size")
        qd = torch.empty((n, nq), dtype=torch.float64, device=X.device)
        qs = torch.empty((n, nq, 2), dtype=torch.float32, device=X.device)
        st = lib().nk_self_diag(self._h, byref(a), byref(p), c_void_p(_ptr(X)), n, H, W, C,
                                c_void_p(_ptr(qd)), c_void_p(_ptr(qs)), c_void_p(_stream()))
        self.check(st, "nk_self_diag")
        return qd, qs

    def autotune(self, convs: Sequence[int], sw2: float, sb2: float, H: int, W: int, C: int = 3,
                 filt: int = 3, act: str = "relu", norm: str = "none") -> int:
        """Times the fused-kernel launch variants for this shape; caches and
        returns the chosen variant."""
        a = make_arch(convs, filt, act, norm)
        p = make_params(sw2, sb2)
        v = c_int(0)
        st = lib().nk_autotune(self._h, byref(a), byref(p), H, W, C, byref(v), c_void_p(_stream()))
        self.check(st, "nk_autotune")
        return v.value

    def autotune_set(self, convs: Sequence[int], sw2: float, sb2: float, H: int, W: int, variant: int,
                     C: int = 3, filt: int = 3):
        a = make_arch(convs, filt)
        p = make_params(sw2, sb2)
        self.check(lib().nk_autotune_set(self._h, byref(a), byref(p), H, W, C, int(variant)),
                   "nk_autotune_set")

    def block(self, Xa: torch.Tensor, qa: Tuple[torch.Tensor, torch.Tensor], Xb: torch.Tensor,
              qb: Tuple[torch.Tensor, torch.Tensor], convs: Sequence[int], sw2: float, sb2: float,
              prec: str = "mixed", a_range=None, b_range=None, symmetric: bool = False,
              out: Optional[torch.Tensor] = None, filt: int = 3, act: str = "relu",
              norm: str = "none", readout: str = "gap") -> torch.Tensor:
        """K[i - a0, j - b0] = NNGP(Xa[i], Xb[j]) over the given index ranges."""
        assert Xa.is_cuda and Xb.is_cuda and Xa.dtype == torch.float32 and Xb.dtype == torch.float32
        _, H, W, C = Xa.shape
        a0, a1, b0, b1 = _ranges(Xa, Xb, a_range, b_range)
        dt = torch.float64 if prec == "plain_fp64" else torch.float32
        if out is None:
            out = torch.empty((a1 - a0, b1 - b0), dtype=dt, device=Xa.device)
        assert out.dtype == dt and out.stride(1) == 1
        a = make_arch(convs, filt, act, norm, readout)
        p = make_params(sw2, sb2)
        st = lib().nk_block(self._h, byref(a), byref(p), _lib.PREC[prec],
                            c_void_p(_ptr(Xa)), c_void_p(_ptr(qa[0])), c_void_p(_ptr(qa[1])), a0, a1,
                            c_void_p(_ptr(Xb)), c_void_p(_ptr(qb[0])), c_void_p(_ptr(qb[1])), b0, b1,
                            H, W, C, c_void_p(_ptr(out)), out.stride(0), int(symmetric),
                            c_void_p(_stream()))
        self.check(st, "nk_block")
        return out

    def block_ntk(self, Xa: torch.Tensor, qa, Xb: torch.Tensor, qb, convs: Sequence[int], sw2: float,
                  sb2: float, prec: str = "plain_fp32", a_range=None, b_range=None, symmetric: bool = False,
                  filt: int = 3, act: str = "relu"):
        """(K, Theta): NNGP and NTK blocks by the layer-wise forms (nk_block_ntk)."""
        _, H, W, C = Xa.shape
        a0, a1, b0, b1 = _ranges(Xa, Xb, a_range, b_range)
        dt = torch.float64 if prec == "plain_fp64" else torch.float32
        K = torch.empty((a1 - a0, b1 - b0), dtype=dt, device=Xa.device)
        T = torch.empty_like(K)
        a = make_arch(convs, filt, act)
        p = make_params(sw2, sb2)
        st = lib().nk_block_ntk(self._h, byref(a), byref(p), _lib.PREC[prec],
                                c_void_p(_ptr(Xa)), c_void_p(_ptr(qa[0])), c_void_p(_ptr(qa[1])), a0, a1,
                                c_void_p(_ptr(Xb)), c_void_p(_ptr(qb[0])), c_void_p(_ptr(qb[1])), b0, b1,
                                H, W, C, c_void_p(_ptr(K)), c_void_p(_ptr(T)), K.stride(0), int(symmetric),
                                c_void_p(_stream()))
        self.check(st, "nk_block_ntk")
        return K, T

    def block_queue(self, tasks: Sequence[dict], convs: Sequence[int], sw2: float, sb2: float,
                    filt: int = 3) -> list:
        """Several MIXED kernel blocks, of image sides 8, 16 or 32, or 64 and
        32 (the tiled form), in one persistent launch (nk_block_queue).  Each task is a dict with keys
        Xa, qa, Xb, qb (self_diag outputs), optional a_range, b_range,
        symmetric, out.  Returns the output tensors in task order."""
        if len(tasks) > _lib.NK_QUEUE_MAX:
            raise NkError(_lib.NK_ERR_INVALID_ARG, f"at most {_lib.NK_QUEUE_MAX} tasks")
        arr = (_lib.NkBlockTask * max(1, len(tasks)))()
        outs = []
        C = None
        for k, t in enumerate(tasks):
            Xa, Xb = t["Xa"], t["Xb"]
            assert Xa.is_cuda and Xa.dtype == torch.float32 and Xb.dtype == torch.float32
            _, H, W, Ck = Xa.shape
            C = Ck if C is None else C
            a0, a1, b0, b1 = _ranges(Xa, Xb, t.get("a_range"), t.get("b_range"))
            out = t.get("out")
            if out is None:
                out = torch.empty((a1 - a0, b1 - b0), dtype=torch.float32, device=Xa.device)
            assert out.dtype == torch.float32 and out.stride(1) == 1
            outs.append(out)
            arr[k] = _lib.NkBlockTask(_ptr(Xa), _ptr(t["qa"][1]), a0, a1, _ptr(Xb), _ptr(t["qb"][1]), b0, b1,
                                      H, W, _ptr(out), out.stride(0), int(bool(t.get("symmetric", False))))
        a = make_arch(convs, filt)
        p = make_params(sw2, sb2)
        st = lib().nk_block_queue(self._h, byref(a), byref(p), int(C or 3), arr, len(tasks),
                                  c_void_p(_stream()))
        self.check(st, "nk_block_queue")
        return outs

    def fc_block(self, Xa: torch.Tensor, Xb: torch.Tensor, sw2: float, sb2: float, depth: int = 3,
                 a_range=None, b_range=None, symmetric: bool = False,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """FC NNGP block (tensor-core Gram + fused arc-cosine recursion)."""
        assert Xa.dtype == torch.float32 and Xa.is_contiguous() and Xb.is_contiguous()
        d = Xa.shape[1]
        a0, a1, b0, b1 = _ranges(Xa, Xb, a_range, b_range)
        if out is None:
            out = torch.empty((a1 - a0, b1 - b0), dtype=torch.float32, device=Xa.device)
        p = make_params(sw2, sb2)
        st = lib().nk_fc_block(self._h, int(depth), byref(p), c_void_p(_ptr(Xa)), a0, a1, c_void_p(_ptr(Xb)),
                               b0, b1, d, c_void_p(_ptr(out)), out.stride(0), int(symmetric),
                               c_void_p(_stream()))
        self.check(st, "nk_fc_block")
        return out

    def block_backward(self, Xa, qa, Xb, qb, convs, sw2, sb2, dK, dXa, dXb, dsw2, dsb2,
                       prec: str = "plain_fp32", a_range=None, b_range=None, symmetric: bool = False,
                       filt: int = 3, act: str = "relu"):
        """Accumulates (+=) the adjoint of block(...) for upstream gradient dK
        into dXa, dXb (image-shaped, may be None), dsw2, dsb2 (1-element
        float64 CUDA tensors)."""
        _, H, W, C = Xa.shape
        a0, a1, b0, b1 = _ranges(Xa, Xb, a_range, b_range)
        a = make_arch(convs, filt, act)
        p = make_params(sw2, sb2)
        assert dK.stride(1) == 1
        st = lib().nk_block_backward(self._h, byref(a), byref(p), _lib.PREC[prec],
                                     c_void_p(_ptr(Xa)), c_void_p(_ptr(qa[0])), c_void_p(_ptr(qa[1])), a0, a1,
                                     c_void_p(_ptr(Xb)), c_void_p(_ptr(qb[0])), c_void_p(_ptr(qb[1])), b0, b1,
                                     H, W, C, c_void_p(_ptr(dK)), dK.stride(0), int(symmetric),
                                     c_void_p(_ptr(dXa)), c_void_p(_ptr(dXb)), c_void_p(_ptr(dsw2)),
                                     c_void_p(_ptr(dsb2)), c_void_p(_stream()))
        self.check(st, "nk_block_backward")

    def set_wait_limit(self, polls: int):
        """Bound of the device-side waits of later calls (polls; < 0: defaults)."""
        self.check(lib().nk_set_wait_limit(self._h, int(polls)), "nk_set_wait_limit")

    def pcg_set_rank(self, rank: int):
        """Rank of the pivoted Cholesky preconditioner (precond="pivchol")."""
        self.check(lib().nk_pcg_set_rank(self._h, int(rank)), "nk_pcg_set_rank")

    def pcg_set_warm_start(self, on: bool):
        """Later pcg_solve calls start from the A they are given (resume)."""
        self.check(lib().nk_pcg_set_warm_start(self._h, int(bool(on))), "nk_pcg_set_warm_start")

    def pcg_solve(self, K: torch.Tensor, Y: torch.Tensor, lam: float, precond: str = "jacobi",
                  prec: str = "mixed", tol: float = 1e-6, maxit: int = 10000, refine_max: int = 16,
                  A: Optional[torch.Tensor] = None, allow_not_converged: bool = False):
        """Solve (K + lam I) A = Y.  K [N, N] float32, Y [N, R] float64 (CUDA).
        Returns (A, iters, relres[R])."""
        assert K.dtype == torch.float32 and K.stride(1) == 1
        assert Y.dtype == torch.float64 and Y.is_contiguous()
        N, R = Y.shape
        if A is None:
            A = torch.empty_like(Y)
        its = c_int(0)
        rel = (ctypes.c_double * max(R, 1))()
        st = lib().nk_pcg_solve(self._h, c_void_p(_ptr(K)), K.stride(0), N, c_void_p(_ptr(Y)), R,
                                float(lam), _lib.PRECOND[precond], _lib.PREC[prec], float(tol), int(maxit),
                                int(refine_max), c_void_p(_ptr(A)), byref(its),
                                ctypes.cast(rel, c_void_p), c_void_p(_stream()))
        if st == _lib.NK_ERR_NOT_CONVERGED and allow_not_converged:
            pass
        else:
            self.check(st, "nk_pcg_solve")
        return A, its.value, [rel[i] for i in range(R)]


def probe(which: str, work: int = 0) -> Tuple[float, float]:
    """(rate per second, kernel ms) of a machine probe (nk_probe): "fp32_fma"
    and "fp64_fma" in lane-FMAs/s, "l2_read" and "hbm_read" in bytes/s."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().nk_probe(_lib.PROBE[which], int(work), byref(rate), byref(ms), c_void_p(_stream()))
    if st != 0:
        raise NkError(st, f"nk_probe {which}")
    return rate.value, ms.value


_DEFAULT: Optional[Handle] = None


def default_handle() -> Handle:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Handle()
    return _DEFAULT


class NNGPBlock(torch.autograd.Function):
    """K = NNGP(Xa, Xb) for the Myrtle-family architecture ``convs`` as a
    differentiable op: forward by nk_self_diag + nk_block, backward by
    nk_block_backward (gradients for Xa, Xb, sigma_w^2, sigma_b^2).

    apply(Xa, Xb, sw2, sb2, handle, convs, symmetric, prec, bprec): Xa, Xb
    float32 CUDA images [n, H, W, C]; sw2, sb2 0-dim float64 tensors.
    symmetric: Xb is Xa and only the upper triangle is computed.  prec is the
    forward precision ("mixed", "plain_fp32", "plain_fp64"), bprec the
    adjoint's ("plain_fp32" or "plain_fp64").
    """

    @staticmethod
    def forward(ctx, Xa, Xb, sw2, sb2, handle, convs, symmetric, prec, bprec):
        h = handle
        s, b = float(sw2), float(sb2)
        qa = h.self_diag(Xa, convs, s, b)
        qb = qa if symmetric else h.self_diag(Xb, convs, s, b)
        K = h.block(Xa, qa, Xb, qb, convs, s, b, prec=prec, symmetric=symmetric)
        ctx.h, ctx.convs, ctx.sym, ctx.bprec = h, convs, symmetric, bprec
        ctx.sw2, ctx.sb2 = s, b
        ctx.save_for_backward(Xa, Xb, qa[0], qa[1], qb[0], qb[1])
        return K

    @staticmethod
    def backward(ctx, dK):
        Xa, Xb, qda, qsa, qdb, qsb = ctx.saved_tensors
        fp64 = ctx.bprec == "plain_fp64"
        dt = torch.float64 if fp64 else torch.float32
        dK = dK.to(dt).contiguous()
        # image gradients only where autograd wants them (nk_block_backward
        # skips the input contraction for a NULL dX; the self-variance adjoint
        # still runs for both sets, since q depends on sigma_w^2 and sigma_b^2)
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if ctx.sym:
            need_a = need_b = need_a or need_b
        dXa = torch.zeros(Xa.shape, dtype=dt, device=Xa.device) if need_a else None
        dXb = dXa if ctx.sym else (torch.zeros(Xb.shape, dtype=dt, device=Xb.device) if need_b else None)
        dsw2 = torch.zeros(1, dtype=torch.float64, device=Xa.device)
        dsb2 = torch.zeros(1, dtype=torch.float64, device=Xa.device)
        ctx.h.block_backward(Xa, (qda, qsa), Xb, (qdb, qsb), ctx.convs, ctx.sw2, ctx.sb2, dK, dXa, dXb,
                             dsw2, dsb2, prec=ctx.bprec, symmetric=ctx.sym)
        gXa = dXa.to(Xa.dtype) if need_a else None
        gXb = None if (ctx.sym or not need_b) else dXb.to(Xb.dtype)
        return gXa, gXb, dsw2.reshape(()), dsb2.reshape(()), None, None, None, None, None


def nngp_block(Xa, Xb, sw2, sb2, convs, handle: Optional[Handle] = None, symmetric: bool = False,
               prec: str = "mixed", bprec: str = "plain_fp32"):
    """Differentiable Myrtle NNGP block (see NNGPBlock)."""
    h = handle or default_handle()
    return NNGPBlock.apply(Xa, Xb, sw2, sb2, h, tuple(convs), symmetric, prec, bprec)
