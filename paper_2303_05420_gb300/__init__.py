"""GB300-native neural-kernel regression (arXiv 2303.05420 hot path).

Myrtle CNN / FC NNGP kernel blocks and the kernel-ridge PCG solve, computed
by libnk.so (hand-written CUDA for sm_103a) behind a C ABI (include/nk.h).
"""

from ._lib import EXPORTS, LIB_PATH, NkError, lib  # noqa: F401

__all__ = ["EXPORTS", "LIB_PATH", "NkError", "lib", "Handle", "default_handle"]


def __getattr__(name):
    if name in ("Handle", "default_handle"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
