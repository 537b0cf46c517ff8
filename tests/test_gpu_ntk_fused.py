"""GPU parity of the fused Myrtle NTK (nk_block_ntk with NK_PREC_MIXED: the
tiled row stream carrying the tangent rows Theta beside the NNGP rows K)
against the oracle's Myrtle NTK (oracle.myrtle_ntk_block, itself pinned by
the linear closed form and Monte Carlo empirical NTKs), element by element
within 1e-5 relative for K and Theta."""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu

CONVS = (2, 1, 0)


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


def _oracle(xa, xb, sb2):
    K, T = oracle.myrtle_ntk_block(oracle.Arch(CONVS), 2.0, sb2, xa.astype(np.float64), xb.astype(np.float64))
    return K.numpy(), T.numpy()


@pytest.mark.parametrize("sb2", [0.0, 0.01])
def test_fused_ntk_32x32_symmetric_block_matches_oracle(h, sb2):
    # 18 images: 171 pairs, more than the 154 slots of the ring of a launch
    # of two CTAs per SM (LAG = 2 x 304 stage-0 tasks), so slots are reused
    x = _imgs(18, 32, 21)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, CONVS, 2.0, sb2)
    K, T = h.block_ntk(X, q, X, q, CONVS, 2.0, sb2, prec="mixed", symmetric=True)
    Kn = h.block(X, q, X, q, CONVS, 2.0, sb2, prec="mixed", symmetric=True)
    h.sync_status()
    K, T, Kn = K.double().cpu().numpy(), T.double().cpu().numpy(), Kn.double().cpu().numpy()
    Kw, Tw = _oracle(x, x, sb2)
    assert _rel(K, Kw) <= 1e-5
    assert _rel(T, Tw) <= 1e-5
    assert np.array_equal(K, K.T) and np.array_equal(T, T.T)
    # the NNGP half is the NNGP block's own arithmetic; the pooled stage-0
    # sums are atomic adds, whose order (and so the last bits) may differ
    assert _rel(K, Kn) <= 1e-6


def test_fused_ntk_32x32_ranges_and_ldk(h):
    xa, xb = _imgs(12, 32, 22), _imgs(9, 32, 23)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa, qb = h.self_diag(Xa, CONVS, 2.0, 0.01), h.self_diag(Xb, CONVS, 2.0, 0.01)
    K, T = h.block_ntk(Xa, qa, Xb, qb, CONVS, 2.0, 0.01, prec="mixed", a_range=(3, 10), b_range=(1, 8))
    h.sync_status()
    Kw, Tw = _oracle(xa[3:10], xb[1:8], 0.01)
    assert _rel(K.double().cpu().numpy(), Kw) <= 1e-5
    assert _rel(T.double().cpu().numpy(), Tw) <= 1e-5


def test_fused_ntk_64x64_matches_oracle(h):
    # 64 stage-0 tasks per pair (two row bands with their halos) and a 32x32
    # stage-1 task reading both pooled tensors from the slot
    xa, xb = _imgs(2, 64, 24), _imgs(3, 64, 25)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa, qb = h.self_diag(Xa, CONVS, 2.0, 0.0), h.self_diag(Xb, CONVS, 2.0, 0.0)
    K, T = h.block_ntk(Xa, qa, Xb, qb, CONVS, 2.0, 0.0, prec="mixed")
    h.sync_status()
    Kw, Tw = _oracle(xa, xb, 0.0)
    assert _rel(K.double().cpu().numpy(), Kw) <= 1e-5
    assert _rel(T.double().cpu().numpy(), Tw) <= 1e-5


def test_fused_ntk_zero_image_and_anticorrelated_pair(h):
    # a zero image has q = 0 at every pixel: the maps and the derivative
    # kernel are zero there (K and Theta reduce to bias terms); x' = -x puts
    # the first layer's correlations at c = -1
    x = _imgs(3, 32, 26)
    x = np.concatenate([x, np.zeros_like(x[:1]), -x[:1]], axis=0)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, CONVS, 2.0, 0.01)
    K, T = h.block_ntk(X, q, X, q, CONVS, 2.0, 0.01, prec="mixed", symmetric=True)
    h.sync_status()
    Kw, Tw = _oracle(x, x, 0.01)
    assert _rel(K.double().cpu().numpy(), Kw) <= 1e-5
    assert _rel(T.double().cpu().numpy(), Tw) <= 1e-5


def test_fused_ntk_refusals(h):
    from paper_2303_05420_gb300._lib import NK_ERR_UNSUPPORTED, NkError

    x16 = torch.tensor(_imgs(2, 16, 27), device="cuda")
    q16 = h.self_diag(x16, CONVS, 2.0, 0.0)
    x32 = torch.tensor(_imgs(2, 32, 28), device="cuda")
    # (3,3,3) and (2,1,1) at 32x32 have the fused NTK (test_gpu_tiled3.py)
    for X, convs in ((x16, CONVS), (x32, (1,)), (x32, (1, 1))):
        q = q16 if X is x16 else h.self_diag(X, convs, 2.0, 0.0)
        with pytest.raises(NkError) as ei:
            h.block_ntk(X, q, X, q, convs, 2.0, 0.0, prec="mixed")
        assert ei.value.status == NK_ERR_UNSUPPORTED


def test_fused_ntk_bench_block_sampled(h):
    """The bench's fused-NTK workload at full size (a symmetric block of 256
    32x32 images, 32,896 pairs: the slot ring turns over about 200 times):
    entries from the start, the middle and the end of the item order and a
    random sample, each against the oracle's NTK pair; K and Theta of the
    whole block exactly symmetric."""
    x = nkdata.standardise(nkdata.images(256, 32, 3, nkdata.SEED_TRAIN, blur=True))[0].astype(np.float32)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, CONVS, 2.0, 0.0)
    K, T = h.block_ntk(X, q, X, q, CONVS, 2.0, 0.0, prec="mixed", symmetric=True)
    h.sync_status()
    K, T = K.double().cpu().numpy(), T.double().cpu().numpy()
    assert np.array_equal(K, K.T) and np.array_equal(T, T.T)
    rng = np.random.default_rng(12)
    pairs = [(0, 0), (0, 1), (0, 255), (1, 1), (127, 128), (128, 200), (254, 255), (255, 255)]
    pairs += [tuple(sorted(p)) for p in rng.integers(0, 256, size=(8, 2))]
    arch = oracle.Arch(CONVS)
    x64 = torch.tensor(x.astype(np.float64))
    qx = {}
    for i, j in pairs:
        for k in (i, j):
            if k not in qx:
                qx[k] = oracle.myrtle_self_q(arch, 2.0, 0.0, x64[k])
        kw, tw = oracle.myrtle_ntk_pair(arch, 2.0, 0.0, x64[i], x64[j], qx[i], qx[j])
        assert abs(K[i, j] - float(kw)) <= 1e-5 * abs(float(kw)), (i, j)
        assert abs(T[i, j] - float(tw)) <= 1e-5 * abs(float(tw)), (i, j)
