"""Pins for the oracle's neural tangent kernel (the Myrtle NTK, the first
widening of the hot path).

* Identity activation with sigma_b^2 = 0: the network is linear and every
  weight layer contributes the same term, so Theta = (L + 1) K for L conv
  layers plus the readout (a closed form independent of the recursion's
  bookkeeping).
* Monte Carlo: the empirical NTK sum_theta df(x)/dtheta df(x')/dtheta of
  finite random networks in the NTK parameterisation (standard-normal
  parameters scaled in the forward pass), gradients by torch autograd.  With
  one hidden layer its expectation is the limit at any width (the hidden
  pre-activations are Gaussian and the readout weights independent); deeper
  networks carry an O(1/n) bias, allowed as 4/n of the value on top of four
  standard errors at widths 32 and 256.
* Symmetry, positive semi-definiteness of the Theta Gram, degree-1
  homogeneity in each image with sigma_b^2 = 0, and K equal to the NNGP
  oracle.
"""

import numpy as np
import pytest
import torch

from nkdata import SEED_MC
from oracle import Arch, myrtle_block, myrtle_ntk_block

F64 = torch.float64


def _empirical_ntk(convs, sw2, sb2, X, width, gen):
    """One draw: the empirical NTK Gram [B, B] of a random network."""
    B, H, W, C = X.shape
    layers = []
    cin = C
    for s, n in enumerate(convs):
        for _ in range(n):
            w = torch.randn(width, cin, 3, 3, dtype=F64, generator=gen).requires_grad_()
            b = torch.randn(width, dtype=F64, generator=gen).requires_grad_()
            layers.append((s, w, b, cin))
            cin = width
    wo = torch.randn(cin, dtype=F64, generator=gen).requires_grad_()
    bo = torch.randn((), dtype=F64, generator=gen).requires_grad_()
    params = [p for (_, w, b, _) in layers for p in (w, b)] + [wo, bo]

    def f(x):
        h = x.permute(2, 0, 1)[None]
        stage = 0
        for s, w, b, ci in layers:
            while stage < s:
                h = torch.nn.functional.avg_pool2d(h, 2)
                stage += 1
            h = torch.nn.functional.conv2d(h, w * np.sqrt(sw2 / (ci * 9)), b * np.sqrt(sb2), padding=1)
            h = torch.relu(h)
        while stage < len(convs) - 1:
            h = torch.nn.functional.avg_pool2d(h, 2)
            stage += 1
        g = h.mean(dim=(2, 3))[0]
        return (wo * g).sum() * np.sqrt(sw2 / cin) + bo * np.sqrt(sb2)

    grads = []
    for a in range(B):
        gs = torch.autograd.grad(f(X[a]), params)
        grads.append(torch.cat([g.reshape(-1) for g in gs]))
    G = torch.stack(grads)
    return G @ G.T


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(SEED_MC + 1)
    return torch.tensor(rng.standard_normal((3, 4, 4, 2)))


@pytest.mark.parametrize("convs", [(1,), (2, 1, 0), (3, 3, 3)])
def test_ntk_identity_activation_closed_form(tiny, convs):
    arch = Arch(convs, act="identity")
    K, T = myrtle_ntk_block(arch, 2.0, 0.0, tiny, tiny)
    L = sum(convs)
    assert torch.allclose(T, (L + 1) * K, rtol=1e-12, atol=0)


def test_ntk_k_is_the_nngp_and_properties(tiny):
    arch = Arch((2, 1, 0))
    K, T = myrtle_ntk_block(arch, 2.0, 0.1, tiny, tiny)
    assert torch.allclose(K, myrtle_block(arch, 2.0, 0.1, tiny, tiny), rtol=1e-12)
    assert torch.allclose(T, T.T, rtol=1e-12)
    assert float(torch.linalg.eigvalsh(T).min()) >= -1e-12 * float(T.abs().max())
    assert bool((T > K).all())  # every hidden layer adds a non-negative term
    _, T2 = myrtle_ntk_block(arch, 2.0, 0.0, 1.5 * tiny[:1], 0.5 * tiny[1:])
    _, T1 = myrtle_ntk_block(arch, 2.0, 0.0, tiny[:1], tiny[1:])
    assert torch.allclose(T2, 0.75 * T1, rtol=1e-11)


def test_ntk_monte_carlo_one_hidden_layer(tiny):
    sw2, sb2 = 2.0, 0.1
    _, want = myrtle_ntk_block(Arch((1,)), sw2, sb2, tiny, tiny)
    gen = torch.Generator().manual_seed(SEED_MC)
    draws = torch.stack([_empirical_ntk((1,), sw2, sb2, tiny, 512, gen) for _ in range(96)])
    mean = draws.mean(0)
    se = draws.std(0) / np.sqrt(draws.shape[0])
    assert float(((mean - want).abs() / se).max()) < 4.5, (mean, want, se)
    assert float(((mean - want).abs() / want.abs()).max()) < 0.02


@pytest.mark.slow
def test_ntk_monte_carlo_myrtle5_pattern_converges(tiny):
    sw2, sb2 = 2.0, 0.1
    convs = (2, 1, 0)
    _, want = myrtle_ntk_block(Arch(convs), sw2, sb2, tiny, tiny)
    gen = torch.Generator().manual_seed(SEED_MC + 7)
    for width, draws in [(32, 96), (256, 96)]:
        d = torch.stack([_empirical_ntk(convs, sw2, sb2, tiny, width, gen) for _ in range(draws)])
        mean = d.mean(0)
        se = d.std(0) / np.sqrt(draws)
        err = (mean - want).abs()
        # sampling error plus an O(1/n) finite-width bias
        assert bool((err <= 4 * se + 4.0 / width * want.abs()).all()), (width, mean, want, se)
