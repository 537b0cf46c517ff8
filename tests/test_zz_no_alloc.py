"""The allocation-free kernel-block entry point against nk_block.

nk_block_fused_noalloc serves callers that cannot allocate device memory when
they need a block (a process whose device memory is reserved up front by its
own allocator, a plugin whose host framework owns all device memory): it
takes no handle and keeps its scratch in a fixed device array.  This test
calls it through the C ABI twice in a row (the second call reuses the array
the first left behind) and checks both results against nk_block's fused path
at the kernel-entry tolerance.  It lives in a file collected last, and works
alone in a fresh process as well as after the other tests.
"""

import ctypes

import numpy as np
import pytest
import torch

import nkdata

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def _call(L, convs, sb2, X, qs, a, b, hw, out, sym):
    from paper_2303_05420_gb300._lib import make_arch, make_params

    arch = make_arch(convs)
    prm = make_params(2.0, sb2)
    err = ctypes.create_string_buffer(256)
    st = L.nk_block_fused_noalloc(ctypes.byref(arch), ctypes.byref(prm), X.data_ptr(), qs.data_ptr(),
                                  a[0], a[1], X.data_ptr(), qs.data_ptr(), b[0], b[1], hw, hw, 3,
                                  out.data_ptr(), out.stride(0), int(sym),
                                  torch.cuda.current_stream().cuda_stream, err, 256)
    return st, err.value.decode()


def test_noalloc_block_matches_nk_block_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300 import _lib
    from paper_2303_05420_gb300.api import Handle

    L = _lib.lib()
    h = Handle()
    cases = [((2, 1, 0), 0.0, 32, (0, 5), (5, 11), False),
             ((3, 3, 3), 0.01, 16, (2, 9), (2, 9), True),
             ((2, 1, 1), 0.01, 8, (0, 4), (3, 11), False)]
    for convs, sb2, hw, a, b, sym in cases:
        x = nkdata.standardise(nkdata.images(11, hw, 3, 5))[0].astype(np.float32)
        X = torch.tensor(x, device="cuda")
        qd, qs = h.self_diag(X, convs, 2.0, sb2)
        ref = h.block(X, (qd, qs), X, (qd, qs), convs, 2.0, sb2, prec="mixed", a_range=a, b_range=b,
                      symmetric=sym).double().cpu().numpy()
        for _ in range(2):
            out = torch.full((a[1] - a[0], b[1] - b[0]), float("nan"), device="cuda")
            st, msg = _call(L, convs, sb2, X, qs, a, b, hw, out, sym)
            assert st == 0, msg
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            assert np.isfinite(got).all()
            assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= TOL32


def test_noalloc_rejects_bad_arguments_with_a_message():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300 import _lib

    L = _lib.lib()
    X = torch.zeros((2, 12, 12, 3), device="cuda")
    qs = torch.zeros((2, 1000, 2), device="cuda")
    out = torch.zeros((2, 2), device="cuda")
    st, msg = _call(L, (2, 1, 0), 0.0, X, qs, (0, 2), (0, 2), 12, out, False)
    assert st == _lib.NK_ERR_UNSUPPORTED and "no fused kernel" in msg
    st, msg = _call(L, (2, 1, 0), 0.0, X, qs, (0, 2), (1, 2), 12, out, True)
    assert st == _lib.NK_ERR_INVALID_ARG and msg


def test_noalloc_rejects_64x64():
    """64x64 images need the tiled form, whose slot ring lives in a handle's
    workspace: the allocation-free entry point refuses them before any work."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300 import _lib

    L = _lib.lib()
    X = torch.zeros((2, 64, 64, 3), device="cuda")
    qs = torch.zeros((2, 2 * 64 * 64 + 32 * 32, 2), device="cuda")
    out = torch.zeros((2, 2), device="cuda")
    st, msg = _call(L, (2, 1, 0), 0.0, X, qs, (0, 2), (0, 2), 64, out, False)
    assert st == _lib.NK_ERR_UNSUPPORTED and "64x64" in msg
