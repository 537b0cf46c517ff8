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


# d = 20: one K stage (a single hi.hi' sum); d = 33: two stages, one per half;
# d = 200: an odd number of stages (7)
@pytest.mark.parametrize("na,nb,d,sym", [(300, 200, 3072, False), (300, 300, 3072, True), (1000, 777, 100, False),
                                         (129, 257, 64, False), (513, 513, 200, True), (200, 150, 20, False),
                                         (260, 260, 33, True)])
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


@pytest.fixture(scope="module")
def fc_full(h):
    """The benchmark's FC workload: 50000 train + 10000 test rows of dimension
    3072, depth 3, sigma_w^2 = 2, sigma_b^2 = 0.01, blocks as bench.py launches
    them (train block symmetric, test block against all train rows)."""
    xtr = nkdata.fc_rows(50000, 3072, nkdata.SEED_TRAIN).astype(np.float32)
    xte = nkdata.fc_rows(10000, 3072, nkdata.SEED_TEST).astype(np.float32)
    Xtr = torch.tensor(xtr, device="cuda")
    Xte = torch.tensor(xte, device="cuda")
    Ktr = h.fc_block(Xtr, Xtr, 2.0, 0.01, depth=3, symmetric=True)
    Kte = h.fc_block(Xte, Xtr, 2.0, 0.01, depth=3)
    h.sync_status()
    return xtr, xte, Ktr, Kte


def test_fc3_fullsize_sampled_entries(fc_full):
    xtr, xte, Ktr, Kte = fc_full
    rng = np.random.default_rng(11)
    ii = np.concatenate([[0, 49999, 777], rng.integers(0, 50000, 60)])
    jj = np.concatenate([[0, 49999, 777], rng.integers(0, 50000, 60)])
    kk = rng.integers(0, 10000, 60)
    got_tr = Ktr[torch.tensor(ii, device="cuda"), torch.tensor(jj, device="cuda")].double().cpu().numpy()
    got_te = Kte[torch.tensor(kk, device="cuda"), torch.tensor(jj[:60], device="cuda")].double().cpu().numpy()
    for n, (i, j) in enumerate(zip(ii, jj)):
        want = oracle.fc_nngp(xtr[i:i + 1].astype(np.float64), xtr[j:j + 1].astype(np.float64), 2.0, 0.01,
                              depth=3).item()
        assert abs(got_tr[n] - want) <= 1e-5 * abs(want), (i, j, got_tr[n], want)
    for n, (k, j) in enumerate(zip(kk, jj[:60])):
        want = oracle.fc_nngp(xte[k:k + 1].astype(np.float64), xtr[j:j + 1].astype(np.float64), 2.0, 0.01,
                              depth=3).item()
        assert abs(got_te[n] - want) <= 1e-5 * abs(want), (k, j, got_te[n], want)


def test_fc3_fullsize_properties_and_pcg(h, fc_full):
    """Symmetric and finite at full size; the mixed PCG solve of the 10 GB
    kernel reaches relative residual 1e-6, checked by an independent float64
    product on the device."""
    xtr, xte, Ktr, Kte = fc_full
    assert bool(torch.isfinite(Ktr).all()) and bool(torch.isfinite(Kte).all())
    for r0 in (0, 20000, 49000):
        blk = Ktr[r0:r0 + 1000]
        assert torch.equal(blk[:, r0:r0 + 1000], blk[:, r0:r0 + 1000].T)
        assert torch.equal(blk[:, :1000], Ktr[:1000, r0:r0 + 1000].T)
    Y = torch.tensor(nkdata.labels(50000, 10), device="cuda")
    A, its, rel = h.pcg_solve(Ktr, Y, -1e-4, precond="jacobi", prec="mixed", tol=1e-6, maxit=5000)
    lam = h.last_lambda()
    Kd = Ktr.double()
    r = Y - (Kd @ A + lam * A)
    del Kd
    rel_true = (r.norm(dim=0) / Y.norm(dim=0)).cpu().numpy()
    assert rel_true.max() <= 1e-6
    assert np.allclose(rel_true, rel, rtol=1e-3, atol=1e-9)
    assert abs(lam - 1e-4 * float(torch.diagonal(Ktr).double().sum()) / 50000) <= 1e-10 * lam


def _near_copies(n, d, eps, seed):
    """Rows x and x + eps z (both scaled to norm sqrt(d)): what data
    augmentation produces, and the case where the Gram is a sum of 3d
    products of one sign."""
    x = nkdata.fc_rows(n, d, seed=seed)
    z = np.random.default_rng(seed + 100).standard_normal((n, d))
    y = x + eps * z
    y *= np.sqrt(d) / np.linalg.norm(y, axis=1, keepdims=True)
    return x.astype(np.float32), y.astype(np.float32)


@pytest.mark.parametrize("eps", [1e-3, 1e-2])
def test_fc3_near_duplicate_rows(h, eps):
    """K(x, x + eps z) at d = 3072 within 1e-5 of the oracle: the tensor
    core's accumulator rounds toward zero, and for near copies every product
    has one sign; the kernel's order of K' and its two chunk accumulators keep
    the drift under the bar.  Also a symmetric block over [x; x + eps z], where
    the near copies sit off the diagonal."""
    xa, xb = _near_copies(256, 3072, eps, seed=5)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    K = h.fc_block(Xa, Xb, 2.0, 0.01, depth=3)
    h.sync_status()
    want = oracle.fc_nngp(xa.astype(np.float64), xb.astype(np.float64), 2.0, 0.01, depth=3).numpy()
    got = K.double().cpu().numpy()
    assert _maxrel(got, want) <= 1e-5
    # the near-copy pairs themselves (the diagonal of this block)
    assert float(np.max(np.abs(np.diag(got) - np.diag(want)) / np.abs(np.diag(want)))) <= 1e-5
    xs = np.concatenate([xa[:128], xb[:128]])
    Xs = torch.tensor(xs, device="cuda")
    Ks = h.fc_block(Xs, Xs, 2.0, 0.01, depth=3, symmetric=True)
    h.sync_status()
    wants = oracle.fc_nngp(xs.astype(np.float64), xs.astype(np.float64), 2.0, 0.01, depth=3).numpy()
    assert _maxrel(Ks.double().cpu().numpy(), wants) <= 1e-5


def test_fc_gram_near_duplicates_depth0(h):
    """depth 0 exposes the Gram itself: x . x' / d for near copies within
    8e-6 relative (the whole sum drifts one way; 6.3e-6 measured on GB300
    against 2.2e-5 predicted for one accumulator with the large products
    first)."""
    xa, xb = _near_copies(200, 3072, 1e-3, seed=6)
    K = h.fc_block(torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda"), 1.0, 0.0, depth=0)
    h.sync_status()
    want = xa.astype(np.float64) @ xb.astype(np.float64).T / 3072
    got = K.double().cpu().numpy()
    d = np.abs(np.diag(got) - np.diag(want)) / np.abs(np.diag(want))
    assert float(d.max()) <= 8e-6, float(d.max())


def test_fc_wait_limit_runs_out_and_the_handle_recovers(h):
    """A wait limit of 0 polls makes the first unmet mbarrier wait of the FC
    kernel give up: the launch returns, nk_sync_status reports
    NK_ERR_TIMEOUT, and with the default limit restored the next call on the
    same handle is correct.  No wait is left unbounded."""
    from paper_2303_05420_gb300._lib import NK_ERR_TIMEOUT, NkError

    x = nkdata.fc_rows(300, 3072, seed=4).astype(np.float32)
    X = torch.tensor(x, device="cuda")
    h.set_wait_limit(0)
    try:
        h.fc_block(X, X, 2.0, 0.01, depth=3, symmetric=True)
        with pytest.raises(NkError) as ei:
            h.sync_status()
        assert ei.value.status == NK_ERR_TIMEOUT
    finally:
        h.set_wait_limit(-1)
    K = h.fc_block(X, X, 2.0, 0.01, depth=3, symmetric=True)
    h.sync_status()
    want = oracle.fc_nngp(x.astype(np.float64), x.astype(np.float64), 2.0, 0.01, depth=3).numpy()
    assert _maxrel(K.double().cpu().numpy(), want) <= 1e-5
