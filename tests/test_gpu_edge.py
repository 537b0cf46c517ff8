"""GPU parity on the method's edge cases, through the C ABI, against the
float64 oracle (1e-5 max-relative for the FP32 / MIXED paths).

- Anticorrelated images (x' = -x, and -x plus a little noise): the first
  layer's correlations reach c = -1, where the arc-cosine map J(c) goes to
  zero like (1 + c)^{3/2}.
- Zero-variance inputs (a ReLU whose input has variance 0 outputs 0, the
  limit of the map as q -> 0; the paper is silent on it): images with
  all-zero regions and an all-zero image, with and without a bias variance.
- A NaN pixel: the self-variances become NaN and nk_sync_status reports
  NK_ERR_NUMERICAL; the handle stays usable.
- A device wait that runs out (Section 2: blocks are computed by
  independent, preemption-safe routines): the tiled kernel's dependency wait
  with a limit of 0 polls gives up, the launch returns, nk_sync_status
  reports NK_ERR_TIMEOUT, and the next call on the handle is correct.
"""

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


def _imgs(n, hw, seed):
    return nkdata.standardise(nkdata.images(n, hw, 3, seed, blur=True))[0].astype(np.float32)


def _relerr(got, want):
    """Element-wise |got - want| / |want|; entries whose oracle value is exactly
    zero must be exactly zero."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    zero = want == 0
    assert np.all(got[zero] == 0), got[zero]
    nz = ~zero & ~np.isnan(want)
    return float(np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz])))


def _block(h, xa, xb, convs, sb2, prec):
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2)
    qb = h.self_diag(Xb, convs, 2.0, sb2)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, sb2, prec=prec)
    h.sync_status()
    return K.double().cpu().numpy()


def _anti(x, noise, seed):
    z = np.random.default_rng(seed).standard_normal(x.shape).astype(np.float32)
    return (-x + noise * z).astype(np.float32)


@pytest.mark.parametrize("hw,convs,sb2", [(8, (2, 1, 0), 0.0), (8, (3, 3, 3), 0.01), (16, (2, 1, 1), 0.0)])
@pytest.mark.parametrize("prec", ["mixed", "plain_fp32"])
@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_anticorrelated_images_small(h, hw, convs, sb2, prec, noise):
    xa = _imgs(4, hw, 0)
    xb = np.concatenate([_anti(xa, noise, 3), _imgs(2, hw, 1)])
    got = _block(h, xa, xb, convs, sb2, prec)
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, sb2, xa.astype(np.float64), xb.astype(np.float64)).numpy()
    assert _relerr(got, want) <= TOL32


@pytest.mark.parametrize("variant", [3, 0])  # the tiled form (default) and the super-plane cluster kernel
@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_anticorrelated_images_32(variant, noise):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    h = Handle()
    convs = (2, 1, 0)
    h.autotune_set(convs, 2.0, 0.0, 32, 32, variant)
    xa = _imgs(3, 32, 0)
    xb = _anti(xa, noise, 4)
    got = _block(h, xa, xb, convs, 0.0, "mixed")
    pairs = [(0, 0), (1, 1), (2, 2), (0, 2)]
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, 0.0, xa.astype(np.float64), xb.astype(np.float64),
                               pairs=pairs).numpy()
    for i, j in pairs:
        assert abs(got[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, got[i, j], want[i, j])
    got32 = _block(h, xa, xb, convs, 0.0, "plain_fp32")
    for i, j in pairs:
        assert abs(got32[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, got32[i, j], want[i, j])


def _zero_region_images(hw):
    """Four images: the top half zeroed, the left 3 columns zeroed, an
    all-zero image, and an untouched one."""
    x = _imgs(4, hw, 2)
    x[0, : hw // 2] = 0.0
    x[1, :, :3] = 0.0
    x[2] = 0.0
    return x


@pytest.mark.parametrize("hw,convs", [(8, (2, 1, 0)), (16, (3, 3, 3))])
@pytest.mark.parametrize("sb2", [0.0, 0.01])
@pytest.mark.parametrize("prec", ["mixed", "plain_fp32", "plain_fp64"])
def test_zero_variance_inputs(h, hw, convs, sb2, prec):
    x = _zero_region_images(hw)
    xb = _imgs(3, hw, 5)
    xb[1] = 0.0
    got = _block(h, x, xb, convs, sb2, prec)
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, sb2, x.astype(np.float64), xb.astype(np.float64)).numpy()
    tol = 1e-12 if prec == "plain_fp64" else TOL32
    assert _relerr(got, want) <= tol
    if sb2 == 0.0:
        # the all-zero image gives an exactly zero row and column
        assert np.all(got[2] == 0) and np.all(got[:, 1] == 0)


def test_zero_variance_inputs_32(h):
    convs = (2, 1, 0)
    x = _zero_region_images(32)
    got = _block(h, x, x, convs, 0.0, "mixed")
    pairs = [(0, 0), (0, 1), (1, 3), (0, 3)]
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, 0.0, x.astype(np.float64), x.astype(np.float64),
                               pairs=pairs).numpy()
    for i, j in pairs:
        assert abs(got[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, got[i, j], want[i, j])
    assert np.all(got[2] == 0) and np.all(got[:, 2] == 0)


def test_nan_pixel_reports_numerical_and_the_handle_recovers(h):
    from paper_2303_05420_gb300._lib import NK_ERR_NUMERICAL, NkError

    convs = (2, 1, 0)
    x = _imgs(3, 8, 6)
    xn = x.copy()
    xn[1, 4, 5, 2] = np.nan
    Xn = torch.tensor(xn, device="cuda")
    h.self_diag(Xn, convs, 2.0, 0.0)
    with pytest.raises(NkError) as ei:
        h.sync_status()
    assert ei.value.status == NK_ERR_NUMERICAL
    # the status word was cleared: a clean call succeeds and is correct
    got = _block(h, x, x, convs, 0.0, "mixed")
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, 0.0, x.astype(np.float64), x.astype(np.float64)).numpy()
    assert _relerr(got, want) <= TOL32


@pytest.mark.parametrize("hw", [32, 64])
def test_tiled_wait_limit_runs_out_and_the_handle_recovers(h, hw):
    """In the tiled kernel a pair's stage-1 task waits for its stage-0 tasks.
    On a block this small every item is claimed in the first wave of CTAs
    (6 pairs x 9 items at 32x32 against 304 CTAs, 2 pairs x 65 items at
    64x64 against 152), so the stage-1 tasks find their pairs unfinished;
    with a limit of 0 polls they give up, raise the abort flag, and every CTA
    stops taking items."""
    from paper_2303_05420_gb300._lib import NK_ERR_TIMEOUT, NkError

    convs = (2, 1, 0)
    xa = _imgs(1 if hw == 64 else 2, hw, 7)
    xb = _imgs(2 if hw == 64 else 3, hw, 8)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, 0.0)
    qb = h.self_diag(Xb, convs, 2.0, 0.0)
    h.sync_status()
    h.set_wait_limit(0)
    try:
        h.block(Xa, qa, Xb, qb, convs, 2.0, 0.0, prec="mixed")
        with pytest.raises(NkError) as ei:
            h.sync_status()
        assert ei.value.status == NK_ERR_TIMEOUT
    finally:
        h.set_wait_limit(-1)
    K = h.block(Xa, qa, Xb, qb, convs, 2.0, 0.0, prec="mixed")
    h.sync_status()
    got = K.double().cpu().numpy()
    pairs = [(i, j) for i in range(xa.shape[0]) for j in range(xb.shape[0])]
    want = oracle.myrtle_block(oracle.Arch(convs), 2.0, 0.0, xa.astype(np.float64), xb.astype(np.float64),
                               pairs=pairs).numpy()
    for i, j in pairs:
        assert abs(got[i, j] - want[i, j]) <= TOL32 * abs(want[i, j]), (i, j, got[i, j], want[i, j])
