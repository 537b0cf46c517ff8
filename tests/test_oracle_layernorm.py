"""Pins for the oracle's LayerNorm option (Arch(norm="layer"): a layer norm
over pixels and channels of each image between each conv and its activation,
as in the tuned Myrtle listing), none of which re-types its formula.

* Monte Carlo: finite CNNs with one hidden layer, an explicit layer norm of
  each image's hidden representation (mean and variance over channels and
  pixels), ReLU, global average pool and a Dense readout; the readout
  covariance given the hidden layer averages to the oracle within four
  standard errors plus an O(1/n) allowance (the empirical normaliser of a
  finite layer fluctuates around its limit).
* Scale invariance: with sb2 = 0 a layer norm removes the scale of each
  image, so K(a x, x') = K(x, x') exactly for a > 0, while the network
  without it is degree-1 homogeneous in each image.
* Identity activation, one conv layer: the NTK with the norm is the NTK
  without it divided by sqrt(m m'), m the mean over pixels of each image's
  conv-output variance (the normaliser is a deterministic per-image scale
  in the limit).
"""

import math

import numpy as np
import torch

from nkdata import SEED_MC
from oracle import Arch, myrtle_block, myrtle_ntk_block, myrtle_self_q

F64 = torch.float64


def test_layernorm_monte_carlo_one_hidden_layer():
    rng = np.random.default_rng(SEED_MC + 31)
    X = torch.tensor(rng.standard_normal((3, 4, 4, 2)))
    sw2, sb2 = 2.0, 0.1
    want = myrtle_block(Arch((1,), norm="layer"), sw2, sb2, X, X)
    gen = torch.Generator().manual_seed(SEED_MC + 32)
    B, H, W, C = X.shape
    x0 = X.permute(0, 3, 1, 2)
    width, draws = 2048, 64
    covs = []
    for _ in range(draws):
        w = torch.randn(width, C, 3, 3, dtype=F64, generator=gen) * math.sqrt(sw2 / (C * 9))
        b = torch.randn(width, dtype=F64, generator=gen) * math.sqrt(sb2)
        h = torch.nn.functional.conv2d(x0, w, b, padding=1)  # [B, n, H, W]
        mu = h.mean(dim=(1, 2, 3), keepdim=True)
        var = ((h - mu) ** 2).mean(dim=(1, 2, 3), keepdim=True)
        g = torch.relu((h - mu) / torch.sqrt(var)).mean(dim=(2, 3))  # layer norm, ReLU, GAP
        covs.append(sw2 / width * g @ g.T + sb2)
    covs = torch.stack(covs)
    mean = covs.mean(0)
    se = covs.std(0) / math.sqrt(draws)
    err = (mean - want).abs()
    assert bool((err <= 4 * se + 4.0 / width * want.abs()).all()), (mean, want, se)
    assert float((err / want.abs()).max()) < 0.01
    # the norm changes the kernel (the same networks without it differ)
    assert float((myrtle_block(Arch((1,)), sw2, sb2, X, X) - want).abs().max()) > 0.05


def test_layernorm_scale_invariance():
    rng = np.random.default_rng(SEED_MC + 33)
    x = torch.tensor(rng.standard_normal((1, 4, 4, 3)))
    xp = torch.tensor(rng.standard_normal((1, 4, 4, 3)))
    for convs in [(1,), (2, 1, 0)]:
        ln, plain = Arch(convs, norm="layer"), Arch(convs)
        k1 = myrtle_block(ln, 2.0, 0.0, x, xp)
        k3 = myrtle_block(ln, 2.0, 0.0, 3.0 * x, xp)
        assert torch.allclose(k1, k3, rtol=1e-13, atol=0)
        p1 = myrtle_block(plain, 2.0, 0.0, x, xp)
        p3 = myrtle_block(plain, 2.0, 0.0, 3.0 * x, xp)
        assert torch.allclose(p3, 3.0 * p1, rtol=1e-12, atol=0)


def test_layernorm_ntk_identity_one_layer():
    rng = np.random.default_rng(SEED_MC + 34)
    X = torch.tensor(rng.standard_normal((3, 4, 4, 2)))
    sw2, sb2 = 2.0, 0.1
    _, T_ln = myrtle_ntk_block(Arch((1,), act="identity", norm="layer"), sw2, sb2, X, X)
    K0, T0 = myrtle_ntk_block(Arch((1,), act="identity"), sw2, sb2, X, X)
    m = torch.stack([myrtle_self_q(Arch((1,), act="identity"), sw2, sb2, x)[0].mean() for x in X])
    # readout: K = sw2 mean Kt + sb2 and Theta = K + sw2 mean Theta_t, with Kt, Theta_t scaled by 1/sqrt(m m')
    s = torch.sqrt(m[:, None] * m[None, :])
    Kt_mean = (K0 - sb2) / sw2
    Tt_mean = (T0 - K0) / sw2
    want = (sw2 * Kt_mean / s + sb2) + sw2 * Tt_mean / s
    assert torch.allclose(T_ln, want, rtol=1e-12, atol=0)
