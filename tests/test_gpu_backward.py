"""GPU parity of the adjoint (nk_block_backward) and the autograd op.

The oracle's gradients (torch autograd through the float64 definition,
itself pinned by fourth-order central differences in test_oracle_solve_grad)
are the reference.  Every component is compared on its own:
|got - want| <= tol * max(|want|, floor), with floor = 1e-3 of the largest
component of that gradient (a component a thousand times smaller than the
largest is a sum whose terms cancel to that level, so its FP32 rounding is
measured against the terms, not against the small result).  tol = 1e-9 for
the FP64 adjoint and 1e-4 for the FP32 adjoint (the benchmark's bar for
gradients).
"""

import numpy as np
import pytest
import torch

import nkdata
import oracle
from oracle.kernels import myrtle_layers_pair, myrtle_self_q

pytestmark = pytest.mark.gpu
F64 = torch.float64


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    return Handle()


def _imgs(n, hw, seed):
    x = nkdata.images(n, hw, 3, seed, blur=True)
    return nkdata.standardise(x)[0].astype(np.float32)


def _oracle_grads(convs, sw2, sb2, xa, xb, dK, symmetric):
    arch = oracle.Arch(convs)
    Xa = torch.tensor(xa.astype(np.float64), requires_grad=True)
    Xb = Xa if symmetric else torch.tensor(xb.astype(np.float64), requires_grad=True)
    s = torch.tensor(sw2, dtype=F64, requires_grad=True)
    b = torch.tensor(sb2, dtype=F64, requires_grad=True)
    qa = [myrtle_self_q(arch, s, b, Xa[i]) for i in range(Xa.shape[0])]
    qb = qa if symmetric else [myrtle_self_q(arch, s, b, Xb[j]) for j in range(Xb.shape[0])]
    L = 0.0
    for i in range(Xa.shape[0]):
        for j in range(Xb.shape[0]):
            k, _, _ = myrtle_layers_pair(arch, s, b, Xa[i], Xb[j], qa[i], qb[j])
            L = L + float(dK[i, j]) * k
    L.backward()
    gb = None if symmetric else Xb.grad.numpy()
    return Xa.grad.numpy(), gb, float(s.grad), float(b.grad)


FLOOR = 1e-3


def _rel(got, want):
    """Largest element-wise relative error, each component against
    max(|want|, FLOOR * max |want|)."""
    den = np.maximum(np.abs(want), FLOOR * np.max(np.abs(want)))
    return float(np.max(np.abs(got - want) / den))


@pytest.mark.parametrize("convs,sb2,hw", [((2, 1, 0), 0.0, 8), ((3, 3, 3), 0.01, 8), ((2, 1, 1), 0.05, 16),
                                          ((1,), 0.1, 8)])
@pytest.mark.parametrize("bprec", ["plain_fp64", "plain_fp32"])
@pytest.mark.parametrize("symmetric", [False, True])
def test_backward_matches_oracle_autograd(h, convs, sb2, hw, bprec, symmetric):
    xa = _imgs(3, hw, 0)
    xb = xa if symmetric else _imgs(2, hw, 1)
    rng = np.random.default_rng(7)
    dK = rng.standard_normal((xa.shape[0], xb.shape[0]))
    want_a, want_b, want_s, want_b2 = _oracle_grads(convs, 2.0, sb2, xa, xb, dK, symmetric)
    fp64 = bprec == "plain_fp64"
    dt = torch.float64 if fp64 else torch.float32
    Xa = torch.tensor(xa, device="cuda")
    Xb = Xa if symmetric else torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2)
    qb = qa if symmetric else h.self_diag(Xb, convs, 2.0, sb2)
    dXa = torch.zeros(Xa.shape, dtype=dt, device="cuda")
    dXb = dXa if symmetric else torch.zeros(Xb.shape, dtype=dt, device="cuda")
    dsw2 = torch.zeros(1, dtype=F64, device="cuda")
    dsb2 = torch.zeros(1, dtype=F64, device="cuda")
    dKt = torch.tensor(dK, dtype=dt, device="cuda")
    h.block_backward(Xa, qa, Xb, qb, convs, 2.0, sb2, dKt, dXa, dXb, dsw2, dsb2, prec=bprec,
                     symmetric=symmetric)
    h.sync_status()
    tol = 1e-9 if fp64 else 1e-4
    assert _rel(dXa.double().cpu().numpy(), want_a) <= tol
    if not symmetric:
        assert _rel(dXb.double().cpu().numpy(), want_b) <= tol
    assert abs(float(dsw2) - want_s) <= tol * abs(want_s)
    if sb2 > 0 or abs(want_b2) > 0:
        assert abs(float(dsb2) - want_b2) <= tol * max(abs(want_b2), 1e-12)


def test_backward_accumulates(h):
    convs = (2, 1, 0)
    x = _imgs(3, 8, 2)
    X = torch.tensor(x, device="cuda")
    q = h.self_diag(X, convs, 2.0, 0.01)
    dK = torch.ones((3, 3), dtype=F64, device="cuda")
    d1 = torch.zeros(X.shape, dtype=F64, device="cuda")
    s1 = torch.zeros(1, dtype=F64, device="cuda")
    b1 = torch.zeros(1, dtype=F64, device="cuda")
    h.block_backward(X, q, X, q, convs, 2.0, 0.01, dK, d1, None, s1, b1, prec="plain_fp64")
    d2, s2, b2 = d1.clone(), s1.clone(), b1.clone()
    h.block_backward(X, q, X, q, convs, 2.0, 0.01, dK, d2, None, s2, b2, prec="plain_fp64")
    h.sync_status()
    assert torch.allclose(d2, 2 * d1, rtol=1e-12, atol=0)
    assert torch.allclose(s2, 2 * s1, rtol=1e-12) and torch.allclose(b2, 2 * b1, rtol=1e-12)


# the FP64 case: its smallest image-gradient components (at the floor) agree
# to about 1.4e-6, FP64 round-off amplified by the ridge solve; 1e-5 is still
# ten times under the gradient bar of 1e-4
@pytest.mark.parametrize("bprec,tol", [("plain_fp64", 1e-5), ("plain_fp32", 1e-4)])
def test_krr_loss_gradients_through_autograd(h, bprec, tol):
    """Kernel-ridge support-set loss (Myrtle-10, 3 support x 4 target images):
    gradients w.r.t. sigma_w^2, sigma_b^2 and the support pixels through the
    autograd op match the oracle's."""
    from paper_2303_05420_gb300.api import nngp_block

    convs = (3, 3, 3)
    rng = np.random.default_rng(nkdata.SEED_SUPPORT)
    xs = rng.standard_normal((3, 8, 8, 3)).astype(np.float32)
    xt = rng.standard_normal((4, 8, 8, 3)).astype(np.float32)
    ys = nkdata.labels(3, 10)
    yt = nkdata.labels(4, 10, seed=9)
    sw2, sb2, lam = 2.0, 0.01, 0.05
    L0, g_sw, g_sb, g_x = oracle.krr_loss_and_grads(oracle.Arch(convs), sw2, sb2, xs.astype(np.float64), ys,
                                                    xt.astype(np.float64), yt, lam)
    fwd = "plain_fp64" if bprec == "plain_fp64" else "mixed"
    Xs = torch.tensor(xs, device="cuda", requires_grad=True)
    Xt = torch.tensor(xt, device="cuda")
    s = torch.tensor(sw2, dtype=F64, device="cuda", requires_grad=True)
    b = torch.tensor(sb2, dtype=F64, device="cuda", requires_grad=True)
    Kss = nngp_block(Xs, Xs, s, b, convs, h, symmetric=True, prec=fwd, bprec=bprec).double()
    Kts = nngp_block(Xt, Xs, s, b, convs, h, prec=fwd, bprec=bprec).double()
    A = torch.linalg.solve(Kss + lam * torch.eye(3, dtype=F64, device="cuda"),
                           torch.tensor(ys, device="cuda"))
    L = 0.5 * ((Kts @ A - torch.tensor(yt, device="cuda")) ** 2).mean()
    L.backward()
    assert abs(float(L.detach()) - L0) <= tol * abs(L0)
    assert abs(float(s.grad) - g_sw) <= tol * abs(g_sw)
    assert abs(float(b.grad) - g_sb) <= tol * abs(g_sb)
    assert _rel(Xs.grad.double().cpu().numpy(), g_x.numpy()) <= tol


@pytest.mark.parametrize("symmetric", [False, True])
def test_backward_myrtle10_32x32(h, symmetric):
    """The gradient workload's network and image size: Myrtle-10 (3,3,3) on
    32x32 images, 2 support x 2 target images, FP32 adjoint against the
    oracle's autograd gradients element by element."""
    convs, sb2 = (3, 3, 3), 0.01
    xa = _imgs(2, 32, 3)
    xb = xa if symmetric else _imgs(2, 32, 4)
    rng = np.random.default_rng(8)
    dK = rng.standard_normal((2, 2))  # a symmetric block counts dK[i][j] and dK[j][i] for entry (i, j)
    want_a, want_b, want_s, want_b2 = _oracle_grads(convs, 2.0, sb2, xa, xb, dK, symmetric)
    Xa = torch.tensor(xa, device="cuda")
    Xb = Xa if symmetric else torch.tensor(xb, device="cuda")
    qa = h.self_diag(Xa, convs, 2.0, sb2)
    qb = qa if symmetric else h.self_diag(Xb, convs, 2.0, sb2)
    dXa = torch.zeros(Xa.shape, dtype=torch.float32, device="cuda")
    dXb = dXa if symmetric else torch.zeros(Xb.shape, dtype=torch.float32, device="cuda")
    dsw2 = torch.zeros(1, dtype=F64, device="cuda")
    dsb2 = torch.zeros(1, dtype=F64, device="cuda")
    dKt = torch.tensor(dK, dtype=torch.float32, device="cuda")
    h.block_backward(Xa, qa, Xb, qb, convs, 2.0, sb2, dKt, dXa, dXb, dsw2, dsb2, prec="plain_fp32",
                     symmetric=symmetric)
    h.sync_status()
    assert _rel(dXa.double().cpu().numpy(), want_a) <= 1e-4
    if not symmetric:
        assert _rel(dXb.double().cpu().numpy(), want_b) <= 1e-4
    assert abs(float(dsw2) - want_s) <= 1e-4 * abs(want_s)
    assert abs(float(dsb2) - want_b2) <= 1e-4 * abs(want_b2)


@pytest.mark.parametrize("hw,na,nb", [(32, 5, 6), (64, 1, 2)])
def test_backward_tensor_core_seed(h, hw, na, nb):
    """FP32 adjoints at 32x32 and 64x64 take the first layer's stored
    pre-activation from the patch Gram on the tensor cores (seed_gemm.cu).
    5 x 6 pairs at 32x32 are 960 GEMM tiles, more than the 4-stage operand
    ring and the two accumulators hold per CTA; the gradients are checked
    element by element against the oracle's autograd."""
    convs, sb2 = (2, 1, 0), 0.01
    xa, xb = _imgs(na, hw, 5), _imgs(nb, hw, 6)
    rng = np.random.default_rng(9)
    dK = rng.standard_normal((na, nb))
    want_a, want_b, want_s, want_b2 = _oracle_grads(convs, 2.0, sb2, xa, xb, dK, False)
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa, qb = h.self_diag(Xa, convs, 2.0, sb2), h.self_diag(Xb, convs, 2.0, sb2)
    dXa = torch.zeros(Xa.shape, dtype=torch.float32, device="cuda")
    dXb = torch.zeros(Xb.shape, dtype=torch.float32, device="cuda")
    dsw2 = torch.zeros(1, dtype=F64, device="cuda")
    dsb2 = torch.zeros(1, dtype=F64, device="cuda")
    dKt = torch.tensor(dK, dtype=torch.float32, device="cuda")
    h.block_backward(Xa, qa, Xb, qb, convs, 2.0, sb2, dKt, dXa, dXb, dsw2, dsb2, prec="plain_fp32")
    h.sync_status()
    assert _rel(dXa.double().cpu().numpy(), want_a) <= 1e-4
    assert _rel(dXb.double().cpu().numpy(), want_b) <= 1e-4
    assert abs(float(dsw2) - want_s) <= 1e-4 * abs(want_s)
    assert abs(float(dsb2) - want_b2) <= 1e-4 * abs(want_b2)


def test_backward_wait_limit_runs_out_and_the_handle_recovers(h):
    """A wait limit of 0 polls makes the mbarrier waits of the adjoint's
    tensor-core first layer (seed_gemm.cu) give up: the call returns,
    nk_sync_status reports NK_ERR_TIMEOUT, and with the default limit
    restored the next call on the same handle matches the oracle.  Each CTA
    still waits, with a fixed bound, for the loads it issued before it exits,
    so no wait is left unbounded."""
    from paper_2303_05420_gb300._lib import NK_ERR_TIMEOUT, NkError

    convs, sb2 = (2, 1, 0), 0.01
    xa, xb = _imgs(2, 32, 11), _imgs(2, 32, 12)
    dK = np.random.default_rng(13).standard_normal((2, 2))
    Xa, Xb = torch.tensor(xa, device="cuda"), torch.tensor(xb, device="cuda")
    qa, qb = h.self_diag(Xa, convs, 2.0, sb2), h.self_diag(Xb, convs, 2.0, sb2)
    dKt = torch.tensor(dK, dtype=torch.float32, device="cuda")
    h.sync_status()

    def run():
        dXa = torch.zeros(Xa.shape, dtype=torch.float32, device="cuda")
        dXb = torch.zeros(Xb.shape, dtype=torch.float32, device="cuda")
        dsw2 = torch.zeros(1, dtype=F64, device="cuda")
        dsb2 = torch.zeros(1, dtype=F64, device="cuda")
        h.block_backward(Xa, qa, Xb, qb, convs, 2.0, sb2, dKt, dXa, dXb, dsw2, dsb2, prec="plain_fp32")
        return dXa, dXb, dsw2, dsb2

    h.set_wait_limit(0)
    try:
        run()
        with pytest.raises(NkError) as ei:
            h.sync_status()
        assert ei.value.status == NK_ERR_TIMEOUT
    finally:
        h.set_wait_limit(-1)
    dXa, dXb, dsw2, dsb2 = run()
    h.sync_status()
    want_a, want_b, want_s, want_b2 = _oracle_grads(convs, 2.0, sb2, xa, xb, dK, False)
    assert _rel(dXa.double().cpu().numpy(), want_a) <= 1e-4
    assert _rel(dXb.double().cpu().numpy(), want_b) <= 1e-4
    assert abs(float(dsw2) - want_s) <= 1e-4 * abs(want_s)
    assert abs(float(dsb2) - want_b2) <= 1e-4 * abs(want_b2)
