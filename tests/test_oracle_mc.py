"""Monte Carlo pin: the oracle kernel is the covariance of wide random networks.

Finite networks are sampled with the parameterisation of the Appendix A
listings (stax defaults): weights N(0, sigma_w^2 / fan_in) with fan_in =
C_in * 3 * 3, biases N(0, sigma_b^2), SAME zero padding, ReLU, 2x2 average
pools, global average pool and a Dense readout.  The readout expectation is
taken exactly given the last hidden layer, E[f f' | g] = sigma_w^2 / n
sum_c GAP(g_c) GAP(g'_c) + sigma_b^2, so only hidden layers are sampled.

* One hidden layer: the pre-activations are exactly Gaussian at any width, so
  the empirical mean must match the oracle within sampling error alone.
* Deeper (the Myrtle-5 stage pattern (2, 1, 0) on 4x4 images, every pool and
  border exercised): finite width adds an O(1/n) bias, so the error must be
  within 4 standard errors plus an O(1/n) allowance and must shrink with width.
"""

import numpy as np
import pytest
import torch

from oracle import Arch, myrtle_block
from nkdata import SEED_MC

F64 = torch.float64


def _sample_cov(convs, sw2, sb2, X, width, draws, chunk, gen):
    """Per-draw readout covariance matrices [draws, B, B]."""
    B, H, W, C = X.shape
    x0 = X.permute(0, 3, 1, 2)  # NCHW
    out = []
    done = 0
    while done < draws:
        D = min(chunk, draws - done)
        h = x0.repeat(1, D, 1, 1)  # [B, D*C, H, W]
        cin = C
        first = True
        for s, n in enumerate(convs):
            if s > 0:
                h = torch.nn.functional.avg_pool2d(h, 2)
            for _ in range(n):
                w = torch.randn(D * width, cin, 3, 3, dtype=F64, generator=gen) * np.sqrt(sw2 / (cin * 9))
                b = torch.randn(D * width, dtype=F64, generator=gen) * np.sqrt(sb2)
                h = torch.nn.functional.conv2d(h, w, b, padding=1, groups=D)
                h = torch.relu(h)
                cin = width
                first = False
        g = h.mean(dim=(2, 3)).reshape(B, D, width)  # GAP
        cov = sw2 / width * torch.einsum("adn,bdn->dab", g, g) + sb2
        out.append(cov)
        done += D
    return torch.cat(out, 0)


@pytest.fixture(scope="module")
def tiny_images():
    rng = np.random.default_rng(SEED_MC)
    return torch.tensor(rng.standard_normal((4, 4, 4, 2)))


def test_mc_one_hidden_layer_exact(tiny_images):
    X = tiny_images
    sw2, sb2 = 2.0, 0.1
    want = myrtle_block(Arch((1,)), sw2, sb2, X, X)
    gen = torch.Generator().manual_seed(SEED_MC)
    covs = _sample_cov((1,), sw2, sb2, X, width=4096, draws=64, chunk=16, gen=gen)
    mean = covs.mean(0)
    se = covs.std(0) / np.sqrt(covs.shape[0])
    z = ((mean - want).abs() / se).max()
    assert float(z) < 4.5, (mean, want, se)
    # tight in absolute terms too
    assert float(((mean - want).abs() / want.abs()).max()) < 0.01


@pytest.mark.slow
def test_mc_myrtle5_pattern_converges_with_width(tiny_images):
    X = tiny_images
    sw2, sb2 = 2.0, 0.1
    convs = (2, 1, 0)
    want = myrtle_block(Arch(convs), sw2, sb2, X, X)
    gen = torch.Generator().manual_seed(SEED_MC + 1)
    errs = []
    for width, draws in [(64, 1600), (512, 200)]:
        covs = _sample_cov(convs, sw2, sb2, X, width=width, draws=draws, chunk=100, gen=gen)
        mean = covs.mean(0)
        se = covs.std(0) / np.sqrt(covs.shape[0])
        err = (mean - want).abs()
        allowance = 4 * se + 4.0 * sum(convs) / width * want.abs()
        assert bool((err <= allowance).all()), (width, err, allowance)
        errs.append(float((err / want.abs()).max()))
    # the finite-width bias shrinks with width
    assert errs[1] < errs[0]
    assert errs[1] < 0.02
