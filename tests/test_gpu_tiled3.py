"""GPU parity of the tiled form for three-stage nets at 32x32 (Myrtle-10
(3,3,3) and (2,1,1)): the stage-1 task pools into an 8x8 stage-2 tile in
shared memory and runs stage 2 on the same CTA.  NNGP (nk_block MIXED with
the tiled launch variant pinned) and NTK (nk_block_ntk MIXED) against the
oracle element by element within 1e-5, on blocks with more pairs than the
launch's slot ring (78 slots for one CTA per SM), ragged ranges, and
against the cluster kernel on the same block."""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu

TILED = 3


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, seed):
    return nkdata.standardise(nkdata.images(n, 32, 3, seed, blur=True))[0].astype(np.float32)


def _rel(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


def test_tiled3_myrtle10_symmetric_block(h):
    convs, sb2 = (3, 3, 3), 0.01
    x = _imgs(13, 51)  # 91 pairs
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, sb2)
    h.autotune_set(convs, 2.0, sb2, 32, 32, TILED)
    try:
        K = h.block(X, q, X, q, convs, 2.0, sb2, symmetric=True).double().cpu().numpy()
    finally:
        h.autotune_set(convs, 2.0, sb2, 32, 32, 0)
    Kc = h.block(X, q, X, q, convs, 2.0, sb2, symmetric=True).double().cpu().numpy()  # cluster kernel
    h.sync_status()
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, sb2, x.astype(np.float64), x.astype(np.float64),
                               symmetric=True).numpy()
    assert _rel(K, want) <= 1e-5
    assert np.array_equal(K, K.T)
    assert _rel(K, Kc) <= 2e-6


@pytest.mark.parametrize("convs,sb2", [((3, 3, 3), 0.0), ((2, 1, 1), 0.05)])
def test_tiled3_ragged_block(h, convs, sb2):
    xa, xb = _imgs(6, 52), _imgs(7, 53)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa, qb = h.self_diag(Xa, convs, 2.0, sb2), h.self_diag(Xb, convs, 2.0, sb2)
    h.autotune_set(convs, 2.0, sb2, 32, 32, TILED)
    try:
        K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, a_range=(2, 6), b_range=(1, 4)).double().cpu().numpy()
    finally:
        h.autotune_set(convs, 2.0, sb2, 32, 32, 0)
    h.sync_status()
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, sb2, xa[2:6].astype(np.float64),
                               xb[1:4].astype(np.float64)).numpy()
    assert _rel(K, want) <= 1e-5


def test_tiled3_myrtle10_ntk(h):
    """The 10-layer Myrtle NTK fused: a symmetric 13-image block (91 pairs)
    against the oracle's NTK pair by pair, and a ragged block."""
    convs, sb2 = (3, 3, 3), 0.01
    x = _imgs(13, 54)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, sb2)
    K, T = h.block_ntk(X, q, X, q, convs, 2.0, sb2, prec="mixed", symmetric=True)
    Kr, Tr = h.block_ntk(X, q, X, q, convs, 2.0, sb2, prec="mixed", a_range=(0, 3), b_range=(5, 9))
    h.sync_status()
    K, T = K.double().cpu().numpy(), T.double().cpu().numpy()
    Kr, Tr = Kr.double().cpu().numpy(), Tr.double().cpu().numpy()
    assert np.array_equal(K, K.T) and np.array_equal(T, T.T)
    arch = oracle.Arch(convs)
    x64 = torch.tensor(x.astype(np.float64))
    qx = [oracle.myrtle_self_q(arch, 2.0, sb2, x64[i]) for i in range(13)]
    for i in range(13):
        for j in range(i, 13):
            kw, tw = oracle.myrtle_ntk_pair(arch, 2.0, sb2, x64[i], x64[j], qx[i], qx[j])
            assert abs(K[i, j] - float(kw)) <= 1e-5 * abs(float(kw)), (i, j)
            assert abs(T[i, j] - float(tw)) <= 1e-5 * abs(float(tw)), (i, j)
            if i < 3 and 5 <= j < 9:
                assert abs(Kr[i, j - 5] - float(kw)) <= 1e-5 * abs(float(kw))
                assert abs(Tr[i, j - 5] - float(tw)) <= 1e-5 * abs(float(tw))


def test_tiled3_refusals(h):
    from paper_2303_05420_gb300._lib import NK_ERR_UNSUPPORTED, NkError

    x64 = torch.tensor(nkdata.standardise(nkdata.images(2, 64, 3, 55, blur=True))[0].astype(np.float32),
                       device="cuda")
    q64 = h.self_diag(x64, (3, 3, 3), 2.0, 0.0)
    with pytest.raises(NkError) as ei:
        h.block_ntk(x64, q64, x64, q64, (3, 3, 3), 2.0, 0.0, prec="mixed")
    assert ei.value.status == NK_ERR_UNSUPPORTED
    x16 = torch.tensor(nkdata.standardise(nkdata.images(2, 16, 3, 56, blur=True))[0].astype(np.float32),
                       device="cuda")
    q16 = h.self_diag(x16, (3, 3, 3), 2.0, 0.0)
    with pytest.raises(NkError) as ei:
        h.block_ntk(x16, q16, x16, q16, (3, 3, 3), 2.0, 0.0, prec="mixed")
    assert ei.value.status == NK_ERR_UNSUPPORTED
