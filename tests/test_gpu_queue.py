"""GPU parity of the kernel-block queue (nk_block_queue): several MIXED
blocks of image sides 32, 16 and 8 in one persistent launch give the same
entries as separate nk_block calls and as the float64 oracle; the launch can
be captured in a CUDA graph and replayed; invalid and unsupported queues are
rejected before anything runs."""

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


def _sets():
    """32x32 images and their 2x2-average companions at 16x16 and 8x8 (the
    mixed-resolution queue of the 64x64 + 32x32 workload, one octave down)."""
    x32 = nkdata.standardise(nkdata.images(7, 32, 3, 0, blur=True))[0]
    x16 = nkdata.downsample2(nkdata.standardise(nkdata.images(9, 32, 3, 1, blur=True))[0])
    x8 = nkdata.downsample2(nkdata.downsample2(nkdata.standardise(nkdata.images(6, 32, 3, 2, blur=True))[0]))
    return [x.astype(np.float32) for x in (x32, x16, x8)]


def _tasks(h, convs, sb2):
    sets = _sets()
    X = [torch.tensor(x, device="cuda") for x in sets]
    q = [h.self_diag(x, convs, 2.0, sb2) for x in X]
    tasks = [
        dict(Xa=X[2], qa=q[2], Xb=X[2], qb=q[2], a_range=(1, 5), b_range=(0, 6)),          # 8x8
        dict(Xa=X[0], qa=q[0], Xb=X[0], qb=q[0], symmetric=True),                        # 32x32 sym
        dict(Xa=X[1], qa=q[1], Xb=X[1], qb=q[1], symmetric=True),                        # 16x16 sym
        dict(Xa=X[0], qa=q[0], Xb=X[0], qb=q[0], a_range=(5, 7), b_range=(0, 3)),          # 32x32 rect
        dict(Xa=X[1], qa=q[1], Xb=X[1], qb=q[1], a_range=(0, 9), b_range=(2, 9)),          # 16x16 rect
    ]
    return sets, X, q, tasks


@pytest.mark.parametrize("convs,sb2", [((2, 1, 0), 0.0), ((3, 3, 3), 0.01), ((2, 1, 1), 0.0)])
def test_queue_matches_blocks_and_oracle(h, convs, sb2):
    sets, X, q, tasks = _tasks(h, convs, sb2)
    outs = h.block_queue(tasks, convs, 2.0, sb2)
    h.sync_status()
    from paper_2303_05420_gb300.api import Handle

    h0 = Handle()
    # the cluster launch variant 0, as the queue uses (at 32x32 the default
    # of a fresh handle is the tiled form where the stage pattern has one)
    h0.autotune_set(convs, 2.0, sb2, 32, 32, 0)
    for t, got in zip(tasks, outs):
        want = h0.block(t["Xa"], t["qa"], t["Xb"], t["qb"], convs, 2.0, sb2, prec="mixed",
                        a_range=t.get("a_range"), b_range=t.get("b_range"),
                        symmetric=t.get("symmetric", False))
        g, w = got.double().cpu().numpy(), want.double().cpu().numpy()
        assert np.isfinite(g).all()
        assert np.max(np.abs(g - w) / np.abs(w)) <= 1e-6
        if t.get("symmetric"):
            assert np.array_equal(g, g.T)
    h0.sync_status()
    # sampled entries against the oracle (one per task)
    arch = oracle.Arch(convs)
    side = {32: 0, 16: 1, 8: 2}
    for t, got in zip(tasks, outs):
        s = sets[side[t["Xa"].shape[1]]]
        a0 = (t.get("a_range") or (0, 0))[0]
        b0 = (t.get("b_range") or (0, 0))[0]
        i, j = got.shape[0] - 1, 0
        xa = torch.tensor(s[a0 + i].astype(np.float64))
        xb = torch.tensor(s[b0 + j].astype(np.float64))
        want = float(oracle.kernels.myrtle_pair(arch, 2.0, sb2, xa, xb))
        assert abs(float(got[i, j]) - want) <= 1e-5 * abs(want)


def test_queue_in_cuda_graph(h):
    convs, sb2 = (2, 1, 0), 0.0
    sets, X, q, tasks = _tasks(h, convs, sb2)
    ref = [o.clone() for o in h.block_queue(tasks, convs, 2.0, sb2)]
    outs = [torch.zeros_like(o) for o in ref]
    for t, o in zip(tasks, outs):
        t["out"] = o
    h.block_queue(tasks, convs, 2.0, sb2)  # warm-up outside the capture
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


def test_queue_rejects(h):
    from paper_2303_05420_gb300._lib import NK_ERR_INVALID_ARG, NK_ERR_UNSUPPORTED, NkError

    # 64x64 images have the tiled form for (2,1,0) (test_gpu_tiled), not for (2,1,1)
    x64 = torch.zeros((2, 64, 64, 3), device="cuda")
    q64 = h.self_diag(x64 + 1.0, (2, 1, 1), 2.0, 0.0)
    with pytest.raises(NkError) as ei:
        h.block_queue([dict(Xa=x64, qa=q64, Xb=x64, qb=q64)], (2, 1, 1), 2.0, 0.0)
    assert ei.value.status == NK_ERR_UNSUPPORTED
    convs = (2, 1, 0)
    sets, X, q, tasks = _tasks(h, convs, 0.0)
    with pytest.raises(NkError) as ei:
        h.block_queue(tasks * 2, convs, 2.0, 0.0)
    assert ei.value.status == NK_ERR_INVALID_ARG
    bad = dict(tasks[1])
    bad["b_range"] = (0, 3)  # symmetric with unequal ranges
    with pytest.raises(NkError) as ei:
        h.block_queue([bad], convs, 2.0, 0.0)
    assert ei.value.status == NK_ERR_INVALID_ARG
    assert h.block_queue([], convs, 2.0, 0.0) == []


def test_64x64_plain_path_matches_oracle(h):
    """64x64 images (the larger problem of the mixed-resolution workload) in
    the layer-wise FP32 form, here one row of a 2 x 3 block against the oracle
    pair by pair (the tiled fused form is checked against this form)."""
    convs = (2, 1, 0)
    x = nkdata.standardise(nkdata.images(3, 64, 3, 5, blur=True))[0].astype(np.float32)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, 0.0)
    K = h.block(X, q, X, q, convs, 2.0, 0.0, prec="plain_fp32", a_range=(0, 1), b_range=(0, 3))
    h.sync_status()
    arch = oracle.Arch(convs)
    for j in range(3):
        want = float(oracle.kernels.myrtle_pair(arch, 2.0, 0.0, torch.tensor(x[0].astype(np.float64)),
                                                torch.tensor(x[j].astype(np.float64))))
        assert abs(float(K[0, j]) - want) <= 1e-5 * abs(want), (j, float(K[0, j]), want)
