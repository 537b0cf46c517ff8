"""GPU parity of the CV8 network (Appendix A, CV8 listing: eight conv(3x3,
SAME) + ReLU layers, Flatten, Dense) against the float64 oracle
(``oracle.cv_block``, which carries the full pixel-pair tensor and is pinned
in test_oracle_cv.py by the offset-0 recursion, the 1x1 / FC reduction and
Monte Carlo).  nk_block with the Flatten readout: MIXED runs the diagonal
recursion (one warp per pair), PLAIN_FP32 / PLAIN_FP64 the layer-wise forms
with a diagonal readout.  Tolerances 1e-5 max-relative (FP32, MIXED) and
1e-12 (FP64)."""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, hw, seed, w=None):
    x = nkdata.standardise(nkdata.images(n, hw, 3, seed, blur=True))[0].astype(np.float32)
    return x if w is None else np.ascontiguousarray(x[:, :, :w])


def _run(h, xa, xb, depth, sb2, prec, act, symmetric=False):
    convs = (depth,)
    Xa = torch.tensor(xa, device="cuda")
    Xb = Xa if symmetric else torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2, act=act)
    qb = qa if symmetric else h.self_diag(Xb, convs, 2.0, sb2, act=act)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec, act=act, readout="flatten", symmetric=symmetric)
    h.sync_status()
    return K.double().cpu().numpy()


def _maxrel(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


@pytest.mark.parametrize("act", ["relu", "erf"])
@pytest.mark.parametrize("prec", ["mixed", "plain_fp32", "plain_fp64"])
@pytest.mark.parametrize("hw,depth,sb2", [(8, 8, 0.01), (16, 8, 0.0), (8, 3, 0.0)])
def test_cv_block_matches_oracle(h, act, prec, hw, depth, sb2):
    xa = _imgs(5, hw, 0)
    xb = _imgs(4, hw, 1)
    want = oracle.cv_block(xa.astype(np.float64), xb.astype(np.float64), 2.0, sb2, depth=depth, act=act).numpy()
    got = _run(h, xa, xb, depth, sb2, prec, act)
    tol = 1e-12 if prec == "plain_fp64" else TOL32
    assert _maxrel(got, want) <= tol
    wants = oracle.cv_block(xa.astype(np.float64), xa.astype(np.float64), 2.0, sb2, depth=depth, act=act).numpy()
    gots = _run(h, xa, xa, depth, sb2, prec, act, symmetric=True)
    assert _maxrel(gots, wants) <= tol
    assert np.array_equal(gots, gots.T)


@pytest.mark.parametrize("act", ["relu", "erf"])
def test_cv8_32x32_matches_oracle(h, act):
    """The CV8 listing on 32x32 images (sigma_w^2 = 2, sigma_b^2 = 0.01):
    MIXED over a 6 x 5 block, checked on sampled pairs; PLAIN_FP32 agrees."""
    xa = _imgs(6, 32, 2)
    xb = _imgs(5, 32, 3)
    got = _run(h, xa, xb, 8, 0.01, "mixed", act)
    pairs = [(0, 0), (5, 4), (2, 3)]
    for i, j in pairs:
        want = oracle.cv_pair(2.0, 0.01, xa[i].astype(np.float64), xb[j].astype(np.float64), 8, act=act).item()
        assert abs(got[i, j] - want) <= TOL32 * abs(want), (i, j, got[i, j], want)
    g32 = _run(h, xa[:2], xb[:2], 8, 0.01, "plain_fp32", act)
    assert _maxrel(g32, got[:2, :2]) <= 2 * TOL32


def test_cv_ragged_width_and_ranges(h):
    """A width below 32 (idle lanes), sub-ranges and a leading dimension wider
    than the block."""
    x = _imgs(7, 16, 4, w=12)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, (8,), 2.0, 0.0)
    out = torch.full((3, 6), float("nan"), device="cuda")
    h.block(X, q, X, q, (8,), 2.0, 0.0, prec="mixed", readout="flatten", a_range=(1, 4), b_range=(2, 6),
            out=out[:, :4])
    h.sync_status()
    want = oracle.cv_block(x[1:4].astype(np.float64), x[2:6].astype(np.float64), 2.0, 0.0, depth=8).numpy()
    got = out.double().cpu().numpy()
    assert _maxrel(got[:, :4], want) <= TOL32
    assert np.isnan(got[:, 4:]).all()


def test_cv_refusals(h):
    from paper_2303_05420_gb300._lib import NK_ERR_INVALID_ARG, NK_ERR_UNSUPPORTED, NkError

    x = torch.tensor(_imgs(2, 8, 5), device="cuda")
    q = h.self_diag(x, (2, 1), 2.0, 0.0)
    # pools mix pixel offsets: the diagonal recursion does not apply
    with pytest.raises(NkError) as ei:
        h.block(x, q, x, q, (2, 1), 2.0, 0.0, prec="mixed", readout="flatten")
    assert ei.value.status == NK_ERR_UNSUPPORTED
    # ... but the layer-wise forms take it (diagonal of the last tensor)
    h.block(x, q, x, q, (2, 1), 2.0, 0.0, prec="plain_fp32", readout="flatten")
    h.sync_status()
    with pytest.raises(NkError) as ei:
        h.block(x, q, x, q, (2, 1), 2.0, 0.0, prec="mixed", readout="flatten", norm="layer")
    assert ei.value.status == NK_ERR_INVALID_ARG
