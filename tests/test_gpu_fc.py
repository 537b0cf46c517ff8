"""GPU parity of the FC NNGP block (Appendix A FC3 listing) computed on the
tensor cores (split-BF16 tcgen05 Gram, FP32 accumulation, fused arc-cosine
recursion) against the float64 oracle."""

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


def _maxrel(got, want):
    return float(np.max(np.abs(got - want) / np.abs(want)))


@pytest.mark.parametrize("na,nb,d,sym", [(300, 200, 3072, False), (300, 300, 3072, True), (1000, 777, 100, False),
                                         (129, 257, 64, False), (513, 513, 200, True)])
def test_fc3_matches_oracle(h, na, nb, d, sym):
    xa = nkdata.fc_rows(na, d, seed=0).astype(np.float32)
    xb = xa if sym else nkdata.fc_rows(nb, d, seed=1).astype(np.float32)
    Xa = torch.tensor(xa, device="cuda")
    Xb = Xa if sym else torch.tensor(xb, device="cuda")
    K = h.fc_block(Xa, Xb, 2.0, 0.01, depth=3, symmetric=sym)
    h.sync_status()
    want = oracle.fc_nngp(xa.astype(np.float64), xb.astype(np.float64), 2.0, 0.01, depth=3).numpy()
    got = K.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert _maxrel(got, want) <= 1e-5
    if sym:
        assert np.array_equal(got, got.T)


def test_fc_depth0_is_the_split_bf16_gram(h):
    # depth 0: K = sw2 x.x'/d + sb2 exposes the Gram's own accuracy
    rng = np.random.default_rng(3)
    xa = rng.standard_normal((260, 3072)).astype(np.float32)
    xb = rng.standard_normal((300, 3072)).astype(np.float32)
    K = h.fc_block(torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda"), 1.0, 0.0, depth=0)
    h.sync_status()
    want = xa.astype(np.float64) @ xb.astype(np.float64).T / 3072
    got = K.double().cpu().numpy()
    # split BF16 keeps ~16 bits of each operand: error ~ 2^-17 of sum |x x'|/d
    scale = np.abs(xa).astype(np.float64) @ np.abs(xb).astype(np.float64).T / 3072
    assert float(np.max(np.abs(got - want) / scale)) <= 2e-5


def test_fc_ranges_and_ldk(h):
    x = nkdata.fc_rows(400, 3072, seed=2).astype(np.float32)
    X = torch.tensor(x, device="cuda")
    out = torch.full((150, 300), float("nan"), device="cuda")
    h.fc_block(X, X, 2.0, 0.01, depth=3, a_range=(50, 200), b_range=(100, 350), out=out[:, :250])
    h.sync_status()
    want = oracle.fc_nngp(x[50:200].astype(np.float64), x[100:350].astype(np.float64), 2.0, 0.01).numpy()
    got = out.cpu().numpy()
    assert _maxrel(got[:, :250].astype(np.float64), want) <= 1e-5
    assert np.isnan(got[:, 250:]).all()
