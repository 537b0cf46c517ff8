"""Pins for the oracle's Myrtle NNGP recursion (Appendix A, Myrtle listing).

* brute force: an independent loop-by-loop implementation (plain Python,
  math.acos) on 2x2x1 and 4x4x1 images;
* identity activation: the network is linear, so the kernel is built from
  explicit shift, pooling and averaging matrices (a different computation
  from the oracle's padded 4-D slicing);
* 1x1 images: the CNN kernel reduces to the FC kernel (exactly for 1x1
  filters; with 3x3 filters each hidden layer carries sigma_w^2 / 9);
* symmetry, positive semi-definiteness, joint flip / transpose / channel
  permutation invariance and degree-1 homogeneity (sigma_b^2 = 0);
* the self-variances are the diagonal of the self kernel tensor.
"""

import itertools
import math

import numpy as np
import pytest
import torch

from oracle import Arch, fc_nngp, myrtle_block, myrtle_pair, myrtle_self_q
from oracle.kernels import myrtle_layers_pair

F64 = torch.float64


# ---------------------------------------------------------------- brute force

def _bf_map(K, q1, q2):
    s = math.sqrt(q1 * q2)
    if s == 0.0:
        return 0.0
    c = max(-1.0, min(1.0, K / s))
    th = math.acos(c)
    return s / (2 * math.pi) * (math.sin(th) + (math.pi - th) * math.cos(th))


def _bf_forward(convs, sw2, sb2, x, xp):
    """Loop-by-loop Myrtle kernel.  x, xp: nested lists [H][W][C]."""
    H, W, C = len(x), len(x[0]), len(x[0][0])

    def input_cov(a, b):
        return {(i, j, k, l): sum(a[i][j][c] * b[k][l][c] for c in range(C)) / C
                for i in range(H) for j in range(W) for k in range(H) for l in range(W)}

    def conv(T, h, w):
        out = {}
        for (i, j, k, l) in T:
            acc = 0.0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    a, b, cc, d = i + dy, j + dx, k + dy, l + dx
                    if 0 <= a < h and 0 <= b < w and 0 <= cc < h and 0 <= d < w:
                        acc += T[(a, b, cc, d)]
            out[(i, j, k, l)] = sw2 / 9.0 * acc + sb2
        return out

    def pool(T, h, w):
        out = {}
        for I in range(h // 2):
            for J in range(w // 2):
                for K_ in range(h // 2):
                    for L in range(w // 2):
                        s = 0.0
                        for a in (0, 1):
                            for b in (0, 1):
                                for cc in (0, 1):
                                    for d in (0, 1):
                                        s += T[(2 * I + a, 2 * J + b, 2 * K_ + cc, 2 * L + d)]
                        out[(I, J, K_, L)] = s / 16.0
        return out

    def run(a, b, qa=None, qb=None):
        T = input_cov(a, b)
        h, w = H, W
        used = []
        li = 0
        for s, n in enumerate(convs):
            if s > 0:
                T = pool(T, h, w)
                h, w = h // 2, w // 2
            for _ in range(n):
                Kp = conv(T, h, w)
                if qa is None:
                    q1 = {(i, j): Kp[(i, j, i, j)] for i in range(h) for j in range(w)}
                    q2 = q1
                else:
                    q1, q2 = qa[li], qb[li]
                used.append(q1)
                T = {key: _bf_map(v, q1[key[:2]], q2[key[2:]]) for key, v in Kp.items()}
                li += 1
        mean = sum(T.values()) / len(T)
        return sw2 * mean + sb2, used

    _, qa = run(x, x)
    _, qb = run(xp, xp)
    val, _ = run(x, xp, qa, qb)
    return val


@pytest.mark.parametrize("hw,convs", [(2, (2, 1)), (4, (1, 1, 1)), (4, (2, 1, 0))])
def test_brute_force(hw, convs):
    rng = np.random.default_rng(11)
    x = rng.standard_normal((hw, hw, 1))
    xp = rng.standard_normal((hw, hw, 1))
    for sw2, sb2 in [(2.0, 0.0), (1.3, 0.07)]:
        want = _bf_forward(convs, sw2, sb2, x.tolist(), xp.tolist())
        got = float(myrtle_pair(Arch(convs), sw2, sb2, torch.tensor(x), torch.tensor(xp)))
        assert abs(got - want) <= 1e-13 * abs(want), (got, want)


# ----------------------------------------------- identity activation: matrices

def _shift(h, w, dy, dx):
    T = np.zeros((h * w, h * w))
    for i in range(h):
        for j in range(w):
            a, b = i + dy, j + dx
            if 0 <= a < h and 0 <= b < w:
                T[i * w + j, a * w + b] = 1.0
    return T


def _poolmat(h, w):
    P = np.zeros(((h // 2) * (w // 2), h * w))
    for I in range(h // 2):
        for J in range(w // 2):
            for a in (0, 1):
                for b in (0, 1):
                    P[I * (w // 2) + J, (2 * I + a) * w + 2 * J + b] = 0.25
    return P


def _linear_kernel(convs, sw2, sb2, x, xp):
    h, w, C = x.shape
    K = x.reshape(h * w, C) @ xp.reshape(h * w, C).T / C
    for s, n in enumerate(convs):
        if s > 0:
            P = _poolmat(h, w)
            K = P @ K @ P.T
            h, w = h // 2, w // 2
        shifts = [_shift(h, w, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        for _ in range(n):
            K = sw2 / 9.0 * sum(T @ K @ T.T for T in shifts) + sb2
    return sw2 * K.mean() + sb2


@pytest.mark.parametrize("convs", [(2, 1, 0), (1, 2, 1), (3, 3, 3)])
def test_identity_activation_closed_form(convs):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((8, 8, 3))
    xp = rng.standard_normal((8, 8, 3))
    want = _linear_kernel(convs, 1.7, 0.05, x, xp)
    got = float(myrtle_pair(Arch(convs, act="identity"), 1.7, 0.05, torch.tensor(x), torch.tensor(xp)))
    assert abs(got - want) <= 1e-12 * abs(want)


# --------------------------------------------------------- 1x1 images vs FC

def test_one_by_one_reduces_to_fc():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, 1, 1, 7))
    flat = X.reshape(5, 7)
    for sw2, sb2 in [(2.0, 0.01), (0.8, 0.3)]:
        # 1x1 filters: exact equality with FC3
        cnn = myrtle_block(Arch((3,), filt=1), sw2, sb2, X, X)
        fc = fc_nngp(flat, flat, sw2, sb2, depth=3)
        assert torch.allclose(cnn, fc, rtol=1e-13, atol=0)
    # 3x3 filters on 1x1 images: only the centre tap is live, so each hidden
    # layer carries sigma_w^2 / 9; with sigma_b^2 = 0 the kernel is then
    # (1/9)^3 times the FC3 kernel (every map is 1-homogeneous).
    cnn = myrtle_block(Arch((3,), filt=3), 2.0, 0.0, X, X)
    fc = fc_nngp(flat, flat, 2.0, 0.0, depth=3)
    assert torch.allclose(cnn, fc / 9.0 ** 3, rtol=1e-13, atol=0)


# ------------------------------------------------ symmetry, PSD, invariances

@pytest.fixture(scope="module")
def eight_by_eight():
    rng = np.random.default_rng(7)
    return torch.tensor(rng.standard_normal((6, 8, 8, 3)))


@pytest.mark.parametrize("convs", [(2, 1, 0), (1, 1, 1)])
def test_symmetry_and_psd(eight_by_eight, convs):
    X = eight_by_eight
    K = myrtle_block(Arch(convs), 2.0, 0.01, X, X)
    assert torch.allclose(K, K.T, rtol=1e-13, atol=0)
    ev = torch.linalg.eigvalsh(K)
    assert float(ev.min()) >= -1e-12 * float(ev.abs().max())
    Kab = myrtle_block(Arch(convs), 2.0, 0.01, X[:2], X[2:])
    Kba = myrtle_block(Arch(convs), 2.0, 0.01, X[2:], X[:2])
    assert torch.allclose(Kab, Kba.T, rtol=1e-13, atol=0)


def test_joint_invariances_and_homogeneity(eight_by_eight):
    arch = Arch((2, 1, 0))
    x, xp = eight_by_eight[0], eight_by_eight[1]
    base = float(myrtle_pair(arch, 2.0, 0.02, x, xp))
    ops = [lambda t: t.flip(0), lambda t: t.flip(1), lambda t: t.transpose(0, 1),
           lambda t: t[:, :, [2, 0, 1]]]
    for op in ops:
        v = float(myrtle_pair(arch, 2.0, 0.02, op(x).contiguous(), op(xp).contiguous()))
        assert abs(v - base) <= 1e-13 * abs(base)
    # one-sided flip is NOT an invariance (guards against a transposed operand)
    v = float(myrtle_pair(arch, 2.0, 0.02, x.flip(0).contiguous(), xp))
    assert abs(v - base) > 1e-6 * abs(base)
    # sigma_b^2 = 0: K(a x, b x') = a b K(x, x')
    k0 = float(myrtle_pair(arch, 2.0, 0.0, x, xp))
    k1 = float(myrtle_pair(arch, 2.0, 0.0, 2.5 * x, 0.3 * xp))
    assert abs(k1 - 0.75 * k0) <= 1e-13 * abs(k0)


def test_self_q_is_diagonal_of_self_tensor(eight_by_eight):
    arch = Arch((2, 1, 1))
    x = eight_by_eight[3]
    qs = myrtle_self_q(arch, 2.0, 0.01, x)
    _, _, pre = myrtle_layers_pair(arch, 2.0, 0.01, x, x)
    for q, K in zip(qs, pre):
        h, w = q.shape
        d = torch.diagonal(K.reshape(h * w, h * w)).reshape(h, w)
        assert torch.equal(q, d)
    # K(x, x) evaluated as a cross pair with those q equals the self value
    kself, _, _ = myrtle_layers_pair(arch, 2.0, 0.01, x, x)
    kcross, _, _ = myrtle_layers_pair(arch, 2.0, 0.01, x, x, qs, qs)
    assert abs(float(kself) - float(kcross)) <= 1e-14 * abs(float(kself))
    # the diagonal of every self pre-activation layer: at c = 1 the map gives q/2
    q1 = qs[0]
    K2 = pre[1]
    h, w = q1.shape
    # q_2(p) = sw2/9 sum_delta q_1(p+delta)/2 + sb2 (only diagonal terms feed the diagonal)
    pad = torch.nn.functional.pad(q1 / 2, (1, 1, 1, 1))
    want = 2.0 / 9.0 * sum(pad[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
                           for dy in (-1, 0, 1) for dx in (-1, 0, 1)) + 0.01
    assert torch.allclose(torch.diagonal(K2.reshape(h * w, h * w)).reshape(h, w), want,
                          rtol=1e-13, atol=0)
