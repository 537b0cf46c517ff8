"""ctypes binding of libnk.so (the C ABI declared in include/nk.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Importing this module does not load the library;
``lib()`` does, and raises if ``libnk.so`` has not been built.  There is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnk.so")

NK_OK, NK_ERR_INVALID_ARG, NK_ERR_CUDA, NK_ERR_NUMERICAL = 0, 1, 2, 3
NK_ERR_NOT_CONVERGED, NK_ERR_TIMEOUT, NK_ERR_NO_MEMORY, NK_ERR_UNSUPPORTED = 4, 5, 6, 7
PREC = {"plain_fp64": 0, "plain_fp32": 1, "mixed": 2}
ACT = {"relu": 0, "identity": 1, "erf": 2}
NORM = {"none": 0, "layer": 1}
READOUT = {"gap": 0, "flatten": 1}
PRECOND = {"none": 0, "jacobi": 1, "pivchol": 2}

# Every symbol include/nk.h declares (checked by a CPU test).
EXPORTS = ["nk_create", "nk_destroy", "nk_status_string", "nk_last_error", "nk_sync_status",
           "nk_q_size", "nk_launch_count", "nk_last_lambda", "nk_self_diag", "nk_block", "nk_block_backward", "nk_fc_block",
           "nk_autotune",
           "nk_autotune_set", "nk_block_fused_noalloc", "nk_block_queue", "nk_block_ntk", "nk_set_wait_limit", "nk_pcg_set_rank", "nk_pcg_set_warm_start",
           "nk_pcg_solve", "nk_probe"]
PROBE = {"fp32_fma": 0, "fp64_fma": 1, "l2_read": 2, "hbm_read": 3}


class NkArch(ctypes.Structure):
    _fields_ = [("n_stages", c_int), ("convs", c_int * 4), ("filter", c_int), ("activation", c_int),
                ("norm", c_int), ("readout", c_int)]


class NkParams(ctypes.Structure):
    _fields_ = [("sigma_w2", c_double), ("sigma_b2", c_double)]


class NkBlockTask(ctypes.Structure):
    _fields_ = [("Xa", c_void_p), ("qsa", c_void_p), ("a0", c_int64), ("a1", c_int64),
                ("Xb", c_void_p), ("qsb", c_void_p), ("b0", c_int64), ("b1", c_int64),
                ("H", c_int), ("W", c_int), ("K", c_void_p), ("ldk", c_int64), ("symmetric", c_int)]


NK_QUEUE_MAX = 8


class NkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libnk status {status}: {msg}")
        self.status = status


_LIB = None


def lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    L.nk_create.argtypes = [POINTER(c_void_p)]
    L.nk_create.restype = c_int
    L.nk_destroy.argtypes = [c_void_p]
    L.nk_destroy.restype = None
    L.nk_status_string.argtypes = [c_int]
    L.nk_status_string.restype = c_char_p
    L.nk_last_error.argtypes = [c_void_p, c_char_p, c_size_t]
    L.nk_last_error.restype = c_int
    L.nk_sync_status.argtypes = [c_void_p, c_void_p]
    L.nk_sync_status.restype = c_int
    L.nk_q_size.argtypes = [POINTER(NkArch), c_int, c_int]
    L.nk_q_size.restype = c_int64
    L.nk_launch_count.argtypes = [c_void_p]
    L.nk_launch_count.restype = c_int64
    L.nk_last_lambda.argtypes = [c_void_p]
    L.nk_last_lambda.restype = c_double
    L.nk_self_diag.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_void_p, c_int64, c_int,
                               c_int, c_int, c_void_p, c_void_p, c_void_p]
    L.nk_self_diag.restype = c_int
    L.nk_block.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int,
                           c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                           c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                           c_int, c_int, c_int, c_void_p, c_int64, c_int, c_void_p]
    L.nk_block.restype = c_int
    L.nk_block_backward.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int,
                                    c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                                    c_void_p, c_void_p, c_void_p, c_int64, c_int64,
                                    c_int, c_int, c_int, c_void_p, c_int64, c_int,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.nk_block_backward.restype = c_int
    L.nk_fc_block.argtypes = [c_void_p, c_int, POINTER(NkParams), c_void_p, c_int64, c_int64, c_void_p, c_int64,
                              c_int64, c_int, c_void_p, c_int64, c_int, c_void_p]
    L.nk_fc_block.restype = c_int
    L.nk_autotune.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int, c_int, c_int,
                              POINTER(c_int), c_void_p]
    L.nk_autotune.restype = c_int
    L.nk_autotune_set.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int, c_int, c_int, c_int]
    L.nk_autotune_set.restype = c_int
    L.nk_block_fused_noalloc.argtypes = [POINTER(NkArch), POINTER(NkParams), c_void_p, c_void_p, c_int64,
                                         c_int64, c_void_p, c_void_p, c_int64, c_int64, c_int, c_int,
                                         c_int, c_void_p, c_int64, c_int, c_void_p, c_char_p, c_size_t]
    L.nk_block_fused_noalloc.restype = c_int
    L.nk_block_ntk.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int, c_void_p, c_void_p, c_void_p,
                               c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_int, c_int,
                               c_int, c_void_p, c_void_p, c_int64, c_int, c_void_p]
    L.nk_block_ntk.restype = c_int
    L.nk_block_queue.argtypes = [c_void_p, POINTER(NkArch), POINTER(NkParams), c_int, POINTER(NkBlockTask),
                                 c_int, c_void_p]
    L.nk_block_queue.restype = c_int
    L.nk_set_wait_limit.argtypes = [c_void_p, c_int64]
    L.nk_set_wait_limit.restype = c_int
    L.nk_pcg_set_rank.argtypes = [c_void_p, c_int]
    L.nk_pcg_set_rank.restype = c_int
    L.nk_pcg_set_warm_start.argtypes = [c_void_p, c_int]
    L.nk_pcg_set_warm_start.restype = c_int
    L.nk_pcg_solve.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_int, c_double, c_int,
                               c_int, c_double, c_int, c_int, c_void_p, POINTER(c_int),
                               c_void_p, c_void_p]
    L.nk_pcg_solve.restype = c_int
    L.nk_probe.argtypes = [c_int, c_int64, POINTER(c_double), POINTER(c_double), c_void_p]
    L.nk_probe.restype = c_int
    _LIB = L
    return L


def make_arch(convs, filt: int = 3, act: str = "relu", norm: str = "none", readout: str = "gap") -> NkArch:
    a = NkArch()
    a.n_stages = len(convs)
    for i in range(4):
        a.convs[i] = convs[i] if i < len(convs) else 0
    a.filter = filt
    a.activation = ACT[act]
    a.norm = NORM[norm]
    a.readout = READOUT[readout]
    return a


def make_params(sw2: float, sb2: float) -> NkParams:
    return NkParams(float(sw2), float(sb2))
