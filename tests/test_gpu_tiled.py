"""GPU parity of the tiled fused form: MIXED blocks of 64x64 images (stage-0
tasks over row bands and shift groups, pooled stage-1 tensors in a ring of
global slots, one stage-1 task per pair), and queues that mix 64x64 and
32x32 blocks in one persistent launch.  Entries are checked against the
float64 oracle pair by pair and, for whole blocks, against the layer-wise
FP32 form (itself checked against the oracle in test_gpu_parity)."""

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


def _imgs(n, side, seed):
    x = nkdata.standardise(nkdata.images(n, 64, 3, seed, blur=True))[0]
    if side == 32:
        x = nkdata.downsample2(x)
    return x.astype(np.float32)


def _oracle_entry(convs, sb2, xa, xb):
    return float(oracle.kernels.myrtle_pair(oracle.Arch(convs), 2.0, sb2, torch.tensor(xa.astype(np.float64)),
                                            torch.tensor(xb.astype(np.float64))))


@pytest.mark.parametrize("convs,sb2", [((2, 1, 0), 0.0), ((2, 1, 0), 0.01), ((1,), 0.0), ((1, 1), 0.0)])
def test_tiled_64_matches_oracle(h, convs, sb2):
    x = _imgs(3, 64, 5)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, sb2)
    K = h.block(X, q, X, q, convs, 2.0, sb2, prec="mixed", a_range=(0, 2), b_range=(1, 3))
    h.sync_status()
    Kp = h.block(X, q, X, q, convs, 2.0, sb2, prec="plain_fp32", a_range=(0, 2), b_range=(1, 3))
    got, ref = K.double().cpu().numpy(), Kp.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-5
    for i, j in [(0, 0), (1, 1)]:
        want = _oracle_entry(convs, sb2, x[i], x[1 + j])
        assert abs(got[i, j] - want) <= 1e-5 * abs(want), (i, j, got[i, j], want)


def test_tiled_64_symmetric_block_reuses_slots(h):
    """300 pairs: far more than the slot ring holds, so every slot is cleared
    and reused many times; the mirror is exact."""
    convs, sb2 = (2, 1, 0), 0.0
    x = _imgs(24, 64, 7)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, sb2)
    K = h.block(X, q, X, q, convs, 2.0, sb2, prec="mixed", symmetric=True)
    h.sync_status()
    Kp = h.block(X, q, X, q, convs, 2.0, sb2, prec="plain_fp32", symmetric=True)
    got, ref = K.double().cpu().numpy(), Kp.double().cpu().numpy()
    assert np.array_equal(got, got.T)
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-5
    for i, j in [(0, 23), (11, 12), (23, 23)]:
        want = _oracle_entry(convs, sb2, x[i], x[j])
        assert abs(got[i, j] - want) <= 1e-5 * abs(want), (i, j)
    # a second call on the same handle (slots left clear by the first) agrees
    K2 = h.block(X, q, X, q, convs, 2.0, sb2, prec="mixed", symmetric=True)
    h.sync_status()
    assert np.max(np.abs(K2.double().cpu().numpy() - got) / np.abs(got)) <= 1e-6


def _mixed_tasks(h, convs, sb2):
    x64 = _imgs(9, 64, 11)
    x32 = _imgs(13, 32, 12)
    X64, X32 = torch.tensor(x64, device="cuda"), torch.tensor(x32, device="cuda")
    q64, q32 = h.self_diag(X64, convs, 2.0, sb2), h.self_diag(X32, convs, 2.0, sb2)
    tasks = [
        dict(Xa=X32, qa=q32, Xb=X32, qb=q32, symmetric=True),                           # 32 sym
        dict(Xa=X64, qa=q64, Xb=X64, qb=q64, a_range=(0, 6), b_range=(0, 6), symmetric=True),  # 64 sym
        dict(Xa=X32, qa=q32, Xb=X32, qb=q32, a_range=(10, 13), b_range=(0, 10)),          # 32 rect
        dict(Xa=X64, qa=q64, Xb=X64, qb=q64, a_range=(6, 9), b_range=(0, 6)),             # 64 rect
    ]
    return (x64, x32), tasks


@pytest.mark.parametrize("convs,sb2", [((2, 1, 0), 0.0), ((2, 1, 0), 0.01)])
def test_tiled_queue_mixes_64_and_32(h, convs, sb2):
    sets, tasks = _mixed_tasks(h, convs, sb2)
    outs = h.block_queue(tasks, convs, 2.0, sb2)
    h.sync_status()
    from paper_2303_05420_gb300.api import Handle

    h0 = Handle()
    h0.autotune_set(convs, 2.0, sb2, 32, 32, 0)
    for t, got in zip(tasks, outs):
        # 64x64: the tiled form alone; 32x32: the cluster super-plane kernel
        want = h0.block(t["Xa"], t["qa"], t["Xb"], t["qb"], convs, 2.0, sb2, prec="mixed",
                        a_range=t.get("a_range"), b_range=t.get("b_range"), symmetric=t.get("symmetric", False))
        g, w = got.double().cpu().numpy(), want.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.max(np.abs(g - w) / np.abs(w)) <= 1e-6
        if t.get("symmetric"):
            assert np.array_equal(g, g.T)
    h0.sync_status()
    for t, got in zip(tasks, outs):
        s = sets[0] if t["Xa"].shape[1] == 64 else sets[1]
        a0 = (t.get("a_range") or (0, 0))[0]
        b0 = (t.get("b_range") or (0, 0))[0]
        i, j = got.shape[0] - 1, 0
        want = _oracle_entry(convs, sb2, s[a0 + i], s[b0 + j])
        assert abs(float(got[i, j]) - want) <= 1e-5 * abs(want)


def test_tiled_queue_in_cuda_graph(h):
    convs, sb2 = (2, 1, 0), 0.0
    sets, tasks = _mixed_tasks(h, convs, sb2)
    ref = [o.clone() for o in h.block_queue(tasks, convs, 2.0, sb2)]
    outs = [torch.zeros_like(o) for o in ref]
    for t, o in zip(tasks, outs):
        t["out"] = o
    h.block_queue(tasks, convs, 2.0, sb2)  # warm-up outside the capture (workspace sized)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        h.block_queue(tasks, convs, 2.0, sb2)
    for o in outs:
        o.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    h.sync_status()
    for o, r in zip(outs, ref):
        assert torch.allclose(o, r, rtol=1e-6, atol=0)


def test_tiled_rejects(h):
    from paper_2303_05420_gb300._lib import NK_ERR_UNSUPPORTED, NkError

    x64 = torch.tensor(_imgs(2, 64, 3), device="cuda")
    x16 = torch.tensor(nkdata.downsample2(_imgs(2, 32, 4)).astype(np.float32), device="cuda")
    for convs in [(2, 1, 1), (3, 3, 3)]:
        q = h.self_diag(x64, convs, 2.0, 0.0)
        with pytest.raises(NkError) as ei:
            h.block(x64, q, x64, q, convs, 2.0, 0.0, prec="mixed")
        assert ei.value.status == NK_ERR_UNSUPPORTED
        with pytest.raises(NkError) as ei:
            h.block_queue([dict(Xa=x64, qa=q, Xb=x64, qb=q)], convs, 2.0, 0.0)
        assert ei.value.status == NK_ERR_UNSUPPORTED
    convs = (2, 1, 0)
    q64 = h.self_diag(x64, convs, 2.0, 0.0)
    q16 = h.self_diag(x16, convs, 2.0, 0.0)
    with pytest.raises(NkError) as ei:
        h.block_queue([dict(Xa=x64, qa=q64, Xb=x64, qb=q64), dict(Xa=x16, qa=q16, Xb=x16, qb=q16)], convs, 2.0,
                      0.0)
    assert ei.value.status == NK_ERR_UNSUPPORTED
