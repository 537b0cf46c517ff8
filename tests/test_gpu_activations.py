"""GPU parity of the tuned-Myrtle options against the float64 oracle: the Erf
activation (one of the activations of the paper's architecture search,
Appendix on tuning the Myrtle architecture) and the LayerNorm between each
conv and its activation (the tuned Myrtle listing's norm layer), alone and
together.

The oracle is ``oracle.Arch(convs, act=..., norm=...)`` (pinned in
test_oracle_erf.py and test_oracle_layernorm.py).  Tolerances as for the
ReLU network: self-variances 1e-12 (FP64 on both sides), kernel entries
1e-12 for PLAIN_FP64 and 1e-5 max-relative for PLAIN_FP32 and MIXED.
"""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
ARCHS = [("erf", "none"), ("relu", "layer"), ("erf", "layer")]


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, hw, seed):
    return nkdata.standardise(nkdata.images(n, hw, 3, seed, blur=True))[0].astype(np.float32)


def _maxrel(got, want):
    mask = ~np.isnan(want)
    return float(np.max(np.abs(got[mask] - want[mask]) / np.abs(want[mask])))


@pytest.mark.parametrize("act,norm", ARCHS)
@pytest.mark.parametrize("hw,convs", [(8, (2, 1, 0)), (16, (3, 3, 3)), (32, (2, 1, 0))])
def test_self_diag_matches_oracle(h, act, norm, hw, convs):
    sb2 = 0.01
    x = _imgs(2, hw, 0)
    qd, qs = h.self_diag(torch.tensor(x, device="cuda"), convs, 2.0, sb2, act=act, norm=norm)
    h.sync_status()
    qd, qs = qd.cpu().numpy(), qs.cpu().numpy()
    arch = oracle.Arch(convs, act=act, norm=norm)
    nl = sum(convs)
    for n in range(2):
        qo = oracle.myrtle_self_q(arch, 2.0, sb2, torch.tensor(x[n].astype(np.float64)))
        q = np.concatenate([t.numpy().reshape(-1) for t in qo])
        nqb = q.size
        assert qd.shape[1] == nqb + (nl if norm == "layer" else 0)
        assert np.allclose(qd[n, :nqb], q, rtol=1e-12, atol=0)
        m = np.ones(nqb)
        if norm == "layer":
            ms = np.array([t.numpy().mean() for t in qo])
            assert np.allclose(qd[n, nqb:], ms, rtol=1e-12, atol=0)
            m = np.concatenate([np.full(t.numel(), t.numpy().mean()) for t in qo])
        if act == "erf":
            a, b = np.sqrt(2.0 / (m + 2.0 * q)), np.ones_like(q)
        else:
            a, b = 1.0 / np.sqrt(q), np.sqrt(q / m)
        assert np.allclose(qs[n, :nqb, 0], a, rtol=1e-6)
        assert np.allclose(qs[n, :nqb, 1], b, rtol=1e-6)


@pytest.mark.parametrize("act,norm", ARCHS)
@pytest.mark.parametrize("hw,convs,sb2", [(8, (2, 1, 0), 0.0), (8, (3, 3, 3), 0.01), (16, (2, 1, 1), 0.01)])
@pytest.mark.parametrize("prec", ["plain_fp64", "plain_fp32", "mixed"])
def test_block_small_matches_oracle(h, act, norm, hw, convs, sb2, prec):
    xa = _imgs(5, hw, 0)
    xb = _imgs(4, hw, 1)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2, act=act, norm=norm)
    qb = h.self_diag(Xb, convs, 2.0, sb2, act=act, norm=norm)
    if prec == "mixed" and act == "erf":
        # Erf runs in the tiled fused form only (32x32 and 64x64 images)
        from paper_2303_05420_gb300._lib import NK_ERR_UNSUPPORTED, NkError

        with pytest.raises(NkError) as ei:
            h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec, act=act, norm=norm)
        assert ei.value.status == NK_ERR_UNSUPPORTED
        return
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec, act=act, norm=norm)
    Ks = h.block(Xa, qa, Xa, qa, convs, 2.0, sb2, prec=prec, act=act, norm=norm, symmetric=True)
    h.sync_status()
    arch = oracle.Arch(convs, act=act, norm=norm)
    want = oracle.myrtle_block(arch, 2.0, sb2, xa.astype(np.float64), xb.astype(np.float64)).numpy()
    wants = oracle.myrtle_block(arch, 2.0, sb2, xa.astype(np.float64), xa.astype(np.float64),
                                symmetric=True).numpy()
    tol = 1e-12 if prec == "plain_fp64" else TOL32
    assert _maxrel(K.double().cpu().numpy(), want) <= tol
    assert _maxrel(Ks.double().cpu().numpy(), wants) <= tol


@pytest.mark.parametrize("act,norm", ARCHS)
@pytest.mark.parametrize("convs,sb2", [((2, 1, 0), 0.0), ((1,), 0.01), ((1, 1), 0.01)])
def test_block_32_tiled_matches_oracle(h, act, norm, convs, sb2):
    """The tiled fused form at 32x32 (ReLU + LayerNorm, Erf, Erf + LayerNorm)
    and the layer-wise FP32 form, pair by pair against the oracle; a symmetric
    block covers the mirrored stores."""
    xa = _imgs(4, 32, 2)
    xb = _imgs(3, 32, 3)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2, act=act, norm=norm)
    qb = h.self_diag(Xb, convs, 2.0, sb2, act=act, norm=norm)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec="mixed", act=act, norm=norm).double().cpu().numpy()
    Ks = h.block(Xa, qa, Xa, qa, convs, 2.0, sb2, prec="mixed", act=act, norm=norm,
                 symmetric=True).double().cpu().numpy()
    K32 = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec="plain_fp32", act=act, norm=norm).double().cpu().numpy()
    h.sync_status()
    arch = oracle.Arch(convs, act=act, norm=norm)
    pairs = [(0, 0), (1, 2), (3, 1), (2, 0)]
    want = oracle.myrtle_block(arch, 2.0, sb2, xa.astype(np.float64), xb.astype(np.float64), pairs=pairs).numpy()
    for i, j in pairs:
        assert abs(K[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, K[i, j], want[i, j])
        assert abs(K32[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, K32[i, j], want[i, j])
    spairs = [(0, 0), (0, 3), (1, 2)]
    wants = oracle.myrtle_block(arch, 2.0, sb2, xa.astype(np.float64), xa.astype(np.float64),
                                pairs=spairs).numpy()
    for i, j in spairs:
        assert abs(Ks[i, j] - wants[i, j]) <= TOL32 * abs(wants[i, j]), (i, j, Ks[i, j], wants[i, j])
        assert Ks[j, i] == Ks[i, j]


@pytest.mark.parametrize("act,norm", [("erf", "none"), ("erf", "layer")])
def test_block_64_tiled_erf_matches_oracle(h, act, norm):
    convs = (2, 1, 0)
    xa = _imgs(1, 64, 4)
    xb = _imgs(2, 64, 5)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, 0.0, act=act, norm=norm)
    qb = h.self_diag(Xb, convs, 2.0, 0.0, act=act, norm=norm)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, 0.0, prec="mixed", act=act, norm=norm).double().cpu().numpy()
    h.sync_status()
    want = oracle.myrtle_block(oracle.Arch(convs, act=act, norm=norm), 2.0, 0.0, xa.astype(np.float64),
                               xb.astype(np.float64)).numpy()
    assert _maxrel(K, want) <= TOL32


def test_unsupported_combinations_are_refused(h):
    from paper_2303_05420_gb300._lib import NK_ERR_INVALID_ARG, NK_ERR_UNSUPPORTED, NkError

    x = _imgs(2, 8, 6)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, (2, 1, 0), 2.0, 0.0, act="erf")
    h.sync_status()
    with pytest.raises(NkError) as ei:
        h.block_ntk(X, q, X, q, (2, 1, 0), 2.0, 0.0, act="erf")
    assert ei.value.status == NK_ERR_UNSUPPORTED
    dX = torch.zeros(X.shape, device="cuda")
    ds = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(NkError) as ei:
        h.block_backward(X, q, X, q, (2, 1, 0), 2.0, 0.0, torch.ones((2, 2), device="cuda"), dX, dX, ds, ds,
                         act="erf", symmetric=True)
    assert ei.value.status == NK_ERR_UNSUPPORTED
    with pytest.raises(NkError) as ei:
        h.self_diag(X, (2, 1, 0), 2.0, 0.0, act="identity", norm="layer")
    assert ei.value.status == NK_ERR_INVALID_ARG
