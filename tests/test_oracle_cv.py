"""Pins for the oracle's CV8 NNGP (the CV8 listing: conv 3x3 SAME + ReLU
layers, Flatten, Dense readout), none of which re-types its formula.

* Offset-0 recursion: the diagonal stencil moves both pixels of a pair by the
  same offset, so the offset p' - p never changes, and the Flatten readout
  reads only the p = p' entries; a plain-loop recursion that carries ONLY the
  H x W diagonal (and the self-variances of each image) must give the same
  value as the full (H W)^2 tensor the oracle carries.
* 1x1 images with 1x1 filters: the network is the fully-connected ReLU
  network of the same depth, so the kernel equals the FC NNGP exactly.
* Monte Carlo: finite CNNs with one hidden layer and a Flatten readout
  (pre-activations exactly Gaussian at any width): the readout covariance,
  given the hidden layer in closed form, averages to the oracle within
  sampling error.
* Symmetry and positive semi-definiteness of a Gram block.
"""

import math

import numpy as np
import torch

from nkdata import SEED_MC
from oracle import cv_block, cv_pair, fc_nngp

F64 = torch.float64


def _relu_map_scalar(K, q1, q2):
    s = math.sqrt(q1 * q2)
    if s == 0.0:
        return 0.0
    c = max(-1.0, min(1.0, K / s))
    t = math.acos(c)
    return s / (2.0 * math.pi) * (math.sin(t) + (math.pi - t) * c)


def _diag_only(sw2, sb2, x, xp, depth):
    """CV NNGP carrying only the diagonal K_l(p, p) of the pair and of each
    image with itself (plain loops, scalars)."""
    H, W, C = x.shape

    def conv(D):
        out = [[0.0] * W for _ in range(H)]
        for i in range(H):
            for j in range(W):
                acc = 0.0
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        u, v = i + dy, j + dx
                        if 0 <= u < H and 0 <= v < W:
                            acc += D[u][v]
                out[i][j] = sw2 / 9.0 * acc + sb2
        return out

    def cov(a, b):
        return [[sum(float(a[i, j, c]) * float(b[i, j, c]) for c in range(C)) / C for j in range(W)]
                for i in range(H)]

    D, Qa, Qb = cov(x, xp), cov(x, x), cov(xp, xp)
    for _ in range(depth):
        D, Qa, Qb = conv(D), conv(Qa), conv(Qb)
        D = [[_relu_map_scalar(D[i][j], Qa[i][j], Qb[i][j]) for j in range(W)] for i in range(H)]
        Qa = [[_relu_map_scalar(Qa[i][j], Qa[i][j], Qa[i][j]) for j in range(W)] for i in range(H)]
        Qb = [[_relu_map_scalar(Qb[i][j], Qb[i][j], Qb[i][j]) for j in range(W)] for i in range(H)]
    return sw2 * sum(sum(r) for r in D) / (H * W) + sb2


def test_cv_full_tensor_equals_offset0_recursion():
    rng = np.random.default_rng(SEED_MC + 21)
    x = torch.tensor(rng.standard_normal((5, 5, 3)))
    xp = torch.tensor(rng.standard_normal((5, 5, 3)))
    for depth, sb2 in [(1, 0.0), (3, 0.1), (8, 0.01)]:
        got = float(cv_pair(2.0, sb2, x, xp, depth=depth))
        want = _diag_only(2.0, sb2, x.numpy(), xp.numpy(), depth)
        assert abs(got - want) <= 1e-13 * abs(want), (depth, got, want)


def test_cv_1x1_images_equal_fc_nngp():
    rng = np.random.default_rng(SEED_MC + 22)
    X = rng.standard_normal((4, 1, 1, 6))
    want = fc_nngp(X.reshape(4, 6), X.reshape(4, 6), 2.0, 0.01, depth=8)
    got = cv_block(X, X, 2.0, 0.01, depth=8, filt=1)
    assert torch.allclose(got, want, rtol=1e-13, atol=0)


def test_cv_monte_carlo_one_hidden_layer():
    rng = np.random.default_rng(SEED_MC + 23)
    X = torch.tensor(rng.standard_normal((3, 4, 4, 2)))
    sw2, sb2 = 2.0, 0.1
    want = cv_block(X, X, sw2, sb2, depth=1)
    gen = torch.Generator().manual_seed(SEED_MC + 24)
    B, H, W, C = X.shape
    x0 = X.permute(0, 3, 1, 2)
    width, draws = 1024, 96
    covs = []
    for _ in range(draws):
        w = torch.randn(width, C, 3, 3, dtype=F64, generator=gen) * math.sqrt(sw2 / (C * 9))
        b = torch.randn(width, dtype=F64, generator=gen) * math.sqrt(sb2)
        h = torch.relu(torch.nn.functional.conv2d(x0, w, b, padding=1)).reshape(B, -1)  # Flatten
        covs.append(sw2 / h.shape[1] * h @ h.T + sb2)  # Dense readout, fan_in = width H W
    covs = torch.stack(covs)
    mean = covs.mean(0)
    se = covs.std(0) / math.sqrt(draws)
    assert float(((mean - want).abs() / se).max()) < 4.5, (mean, want, se)
    assert float(((mean - want).abs() / want.abs()).max()) < 0.01


def test_cv_block_symmetric_psd():
    rng = np.random.default_rng(SEED_MC + 25)
    X = torch.tensor(rng.standard_normal((4, 4, 4, 3)))
    K = cv_block(X, X, 2.0, 0.01, depth=8)
    assert torch.allclose(K, K.T, rtol=1e-13)
    assert float(torch.linalg.eigvalsh(K).min()) >= -1e-13 * float(K.abs().max())
