"""Parity at the headline size, in the launch configuration bench.py times.

2048 train + 512 test 32x32x3 images (the benchmark's generator), Myrtle-5
(2,1,0), sigma_w^2 = 2, sigma_b^2 = 0, after nk_autotune: the full train block
(symmetric) and test block on the GPU; sampled entries against the float64
oracle one by one (train diagonal, train off-diagonal, test); properties at
full size: finite, positive, symmetric, positive semi-definite in float64;
the MIXED PCG solve reaches relative residual 1e-6 against the float32 K
upcast to float64.
"""

import numpy as np
import pytest
import torch

import nkdata
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def headline():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_05420_gb300.api import Handle

    p = nkdata.image_problem(2048, 512, 32, n_classes=10, blur=True)
    x = np.concatenate([p.x_train, p.x_test]).astype(np.float32)
    h = Handle()
    X = torch.tensor(x, device="cuda")
    convs = (2, 1, 0)
    h.autotune(convs, 2.0, 0.0, 32, 32, 3)
    q = h.self_diag(X, convs, 2.0, 0.0)
    Ktr = h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", a_range=(0, 2048), b_range=(0, 2048),
                  symmetric=True)
    Kte = h.block(X, q, X, q, convs, 2.0, 0.0, prec="mixed", a_range=(2048, 2560), b_range=(0, 2048))
    h.sync_status()
    return h, x, p, Ktr, Kte


def test_sampled_entries_match_oracle(headline):
    h, x, p, Ktr, Kte = headline
    arch = oracle.Arch((2, 1, 0))
    xs = torch.tensor(x.astype(np.float64))
    samples = [("tr", 0, 0), ("tr", 7, 7), ("tr", 3, 2047), ("tr", 1500, 611), ("tr", 1024, 1025),
               ("te", 0, 0), ("te", 511, 2047), ("te", 100, 1234)]
    Kt, Ke = Ktr.cpu().numpy(), Kte.cpu().numpy()
    qcache = {}

    def q_of(i):
        if i not in qcache:
            qcache[i] = oracle.myrtle_self_q(arch, 2.0, 0.0, xs[i])
        return qcache[i]

    for which, i, j in samples:
        ia = i if which == "tr" else 2048 + i
        want, _, _ = oracle.kernels.myrtle_layers_pair(arch, 2.0, 0.0, xs[ia], xs[j], q_of(ia), q_of(j))
        got = Kt[i, j] if which == "tr" else Ke[i, j]
        assert abs(float(got) - float(want)) <= 1e-5 * abs(float(want)), (which, i, j, got, float(want))


def test_fullsize_properties(headline):
    h, x, p, Ktr, Kte = headline
    Kt = Ktr.double().cpu().numpy()
    assert np.isfinite(Kt).all() and np.isfinite(Kte.cpu().numpy()).all()
    assert (Kt > 0).all()
    assert np.array_equal(Kt, Kt.T)
    ev = np.linalg.eigvalsh(Kt)
    assert ev.min() >= -1e-6 * ev.max()  # float32 entries: PSD up to their rounding


def test_fullsize_pcg(headline):
    h, x, p, Ktr, Kte = headline
    Y = torch.tensor(p.y_train, device="cuda")
    A, its, rel = h.pcg_solve(Ktr, Y, -1e-4, precond="jacobi", prec="mixed", tol=1e-6, maxit=20000)
    Kt = Ktr.double().cpu().numpy()
    lam = h.last_lambda()
    assert abs(lam - 1e-4 * np.trace(Kt) / 2048) <= 1e-12 * lam
    r = p.y_train - (Kt + lam * np.eye(2048)) @ A.cpu().numpy()
    rel_true = np.linalg.norm(r, axis=0) / np.linalg.norm(p.y_train, axis=0)
    assert rel_true.max() <= 1e-6
    assert np.allclose(rel_true, rel, rtol=1e-3, atol=1e-9)


def test_fullsize_pcg_pivchol(headline):
    """The paper's preconditioner on the headline block: relative residual
    1e-6 in far fewer iterations than Jacobi."""
    h, x, p, Ktr, Kte = headline
    Y = torch.tensor(p.y_train, device="cuda")
    _, it_j, _ = h.pcg_solve(Ktr, Y, -1e-4, precond="jacobi", prec="plain_fp64", tol=1e-6, maxit=20000)
    h.pcg_set_rank(100)
    A, its, rel = h.pcg_solve(Ktr, Y, -1e-4, precond="pivchol", prec="mixed", tol=1e-6, maxit=20000)
    Kt = Ktr.double().cpu().numpy()
    lam = h.last_lambda()
    r = p.y_train - (Kt + lam * np.eye(2048)) @ A.cpu().numpy()
    rel_true = np.linalg.norm(r, axis=0) / np.linalg.norm(p.y_train, axis=0)
    assert rel_true.max() <= 1e-6
    _, it_p64, _ = h.pcg_solve(Ktr, Y, -1e-4, precond="pivchol", prec="plain_fp64", tol=1e-6, maxit=20000)
    assert it_p64 < it_j / 2, (it_p64, it_j)


def _sym_pair(idx, n):
    """(i, j) of upper-triangle pair number idx in the row-major order the
    kernels walk (row i holds pairs (i, i), (i, i + 1), ..., (i, n - 1))."""
    i = 0
    while idx >= n - i:
        idx -= n - i
        i += 1
    return i, i + idx


def test_fullsize_contiguous_subblocks(headline):
    """Contiguous 16 x 16 sub-blocks of the full-size blocks, entry by entry:
    one crossing the train block's diagonal at its end, one in its interior,
    and the last rows and columns of the test block."""
    h, x, p, Ktr, Kte = headline
    arch = oracle.Arch((2, 1, 0))
    xd = x.astype(np.float64)
    Kt, Ke = Ktr.double().cpu().numpy(), Kte.double().cpu().numpy()
    cases = [(Kt, slice(2032, 2048), slice(2032, 2048), xd[2032:2048], xd[2032:2048]),
             (Kt, slice(1000, 1016), slice(1100, 1116), xd[1000:1016], xd[1100:1116]),
             (Ke, slice(496, 512), slice(2032, 2048), xd[2048 + 496:2560], xd[2032:2048])]
    for K, ri, cj, xa, xb in cases:
        want = oracle.myrtle_block(arch, 2.0, 0.0, xa, xb).numpy()
        got = K[ri, cj]
        err = float(np.max(np.abs(got - want) / np.abs(want)))
        assert err <= 1e-5, (ri, cj, err)


def test_fullsize_item_order_positions(headline):
    """Pairs at the start, middle and end of the train block's item order,
    and pairs one and two slot-ring lengths apart (the 32x32 launch of two
    CTAs per SM keeps 154 slots; pairs g and g + 154 share one)."""
    h, x, p, Ktr, Kte = headline
    arch = oracle.Arch((2, 1, 0))
    xs = torch.tensor(x.astype(np.float64))
    G = 2048 * 2049 // 2
    idx = [0, 1, 2, G // 2, G // 2 + 1, G - 2, G - 1, 100000, 100000 + 154, 100000 + 308]
    Kt = Ktr.cpu().numpy()
    for g in idx:
        i, j = _sym_pair(g, 2048)
        qi = oracle.myrtle_self_q(arch, 2.0, 0.0, xs[i])
        qj = oracle.myrtle_self_q(arch, 2.0, 0.0, xs[j])
        want, _, _ = oracle.kernels.myrtle_layers_pair(arch, 2.0, 0.0, xs[i], xs[j], qi, qj)
        assert abs(float(Kt[i, j]) - float(want)) <= 1e-5 * abs(float(want)), (g, i, j, Kt[i, j], float(want))
