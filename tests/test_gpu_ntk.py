"""GPU parity of the layer-wise NTK block (nk_block_ntk) against the oracle's
Myrtle NTK (itself pinned by the linear closed form and Monte Carlo
empirical NTKs): K and Theta within 1e-12 (FP64) and 1e-5 (FP32) relative."""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, hw, seed):
    return nkdata.standardise(nkdata.images(n, hw, 3, seed, blur=True))[0].astype(np.float32)


def _rel(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


@pytest.mark.parametrize("convs,sb2,act", [((2, 1, 0), 0.0, "relu"), ((3, 3, 3), 0.01, "relu"),
                                           ((1,), 0.1, "relu"), ((2, 1, 1), 0.0, "identity")])
@pytest.mark.parametrize("prec", ["plain_fp64", "plain_fp32"])
def test_ntk_matches_oracle(h, convs, sb2, act, prec):
    xa, xb = _imgs(3, 8, 0), _imgs(4, 8, 1)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2, act=act)
    qb = h.self_diag(Xb, convs, 2.0, sb2, act=act)
    K, T = h.block_ntk(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec, act=act)
    h.sync_status()
    arch = oracle.Arch(convs, act=act)
    Kw, Tw = oracle.myrtle_ntk_block(arch, 2.0, sb2, xa.astype(np.float64), xb.astype(np.float64))
    tol = 1e-12 if prec == "plain_fp64" else 1e-5
    assert _rel(K.double().cpu().numpy(), Kw.numpy()) <= tol
    assert _rel(T.double().cpu().numpy(), Tw.numpy()) <= tol


def test_ntk_symmetric_ranges_and_unsupported(h):
    from paper_2303_05420_gb300._lib import NK_ERR_UNSUPPORTED, NkError

    convs = (2, 1, 0)
    x = _imgs(5, 8, 2)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, 0.0)
    K, T = h.block_ntk(X, q, X, q, convs, 2.0, 0.0, prec="plain_fp64", symmetric=True)
    Kr, Tr = h.block_ntk(X, q, X, q, convs, 2.0, 0.0, prec="plain_fp64", a_range=(1, 4), b_range=(0, 5))
    h.sync_status()
    T, Tr = T.cpu().numpy(), Tr.cpu().numpy()
    assert np.array_equal(T, T.T)
    assert np.allclose(Tr, T[1:4, :], rtol=1e-13)
    # the fused NTK (prec "mixed") takes 32x32 and 64x64 images only
    with pytest.raises(NkError) as ei:
        h.block_ntk(X, q, X, q, convs, 2.0, 0.0, prec="mixed")
    assert ei.value.status == NK_ERR_UNSUPPORTED


def test_ntk_32x32_pair(h):
    convs = (2, 1, 0)
    x = _imgs(2, 32, 3)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, 0.0)
    K, T = h.block_ntk(X, q, X, q, convs, 2.0, 0.0, prec="plain_fp32", a_range=(0, 1), b_range=(1, 2))
    h.sync_status()
    arch = oracle.Arch(convs)
    x64 = torch.tensor(x.astype(np.float64))
    qx = [oracle.myrtle_self_q(arch, 2.0, 0.0, x64[i]) for i in range(2)]
    Kw, Tw = oracle.myrtle_ntk_pair(arch, 2.0, 0.0, x64[0], x64[1], qx[0], qx[1])
    assert abs(float(K[0, 0]) - float(Kw)) <= 1e-5 * abs(float(Kw))
    assert abs(float(T[0, 0]) - float(Tw)) <= 1e-5 * abs(float(Tw))
